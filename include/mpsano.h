/*
 * mpsano.h -- C ABI of the B300 (sm_103a) MPS-ANO-VQC feature-extraction path.
 *
 * What it computes (arxiv 2607.10280):
 *   p x p image -> one qubit per pixel on a row-major chain (Sec. II.B)
 *   -> encoding / entangling circuit (Sec. II.B, Eq. 2)
 *   -> matrix product state with SVD truncation to bond dimension chi (Sec. II.B, Eq. 3)
 *   -> all 16 two-qubit Pauli expectations of image-local pairs, the Pauli cache
 *      (Sec. II.C, Eq. 4-5)
 *   -> adaptive-observable features q = sum_alpha c_alpha <P_alpha> (Eq. 1, 4, 5)
 *   -> linear reconstruction y = W q + b (Eq. 6).
 *
 * Conventions shared by every call
 *   - Qubit k is pixel (k / p, k % p).  Pauli index alpha = 4a + b with I,X,Y,Z = 0..3,
 *     P_a on the lower chain index of the pair.
 *   - Pair order per image: horizontal (r,c)-(r,c+1) row-major by the left pixel,
 *     then vertical (r,c)-(r+1,c) row-major by the top pixel, then (pair set HVD only)
 *     diagonal (r,c)-(r+1,c+1) and anti-diagonal (r,c+1)-(r+1,c), each row-major.
 *   - "device" pointers are CUDA global-memory addresses on the batch's device;
 *     "host" pointers are ordinary CPU memory.  The caller owns every pointer it
 *     passes; the library owns only what a mps_batch holds.
 *   - Every call returns an mps_status.  Argument errors are detected on the host
 *     and returned synchronously; nothing is launched in that case.  Work is
 *     enqueued asynchronously on the batch's stream.  Errors raised by device code
 *     (bounded waits, bounds checks) are recorded in a device status word and are
 *     returned by the next mps_sync() on that batch.  mps_last_error() gives a
 *     thread-local message for the last non-OK status.  Nothing throws across
 *     the ABI.
 */
#ifndef MPSANO_H
#define MPSANO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MPS_OK = 0,
    MPS_ERR_INVALID_ARG = 1,  /* bad size, pointer or enum value */
    MPS_ERR_OOM = 2,          /* device allocation failed */
    MPS_ERR_CUDA = 3,         /* a CUDA runtime call failed */
    MPS_ERR_TIMEOUT = 4,      /* a bounded device wait gave up */
    MPS_ERR_UNSUPPORTED = 5,  /* valid request outside what the library supports */
    MPS_ERR_NOT_READY = 6,    /* e.g. Pauli cache requested before a circuit ran */
    MPS_ERR_DEVICE = 7        /* a device-side check failed (see mps_last_error) */
} mps_status;

/* Arithmetic of the path.
 *   MPS_FP64         complex128 everywhere (the plain FP64 path).
 *   MPS_MIXED        complex64 wherever no singular value is discarded: gates, exact
 *                    QR splits, operator products, environments and Pauli
 *                    contractions.  An image whose circuit truncates lossily (keeps
 *                    chi < rank at some cut) runs its whole circuit on a complex128
 *                    state -- sequential truncation amplifies the rounding of a
 *                    complex64 state far beyond 1e-5 (measured up to 4e-3 at chi = 2,
 *                    7x7, L = 4) -- and the final MPS is rounded to complex64 for the
 *                    environment and Pauli kernels.  Every Pauli entry then stays
 *                    within 1e-5 of the FP64 result.
 *   MPS_MIXED_ORTH64 as MPS_MIXED, and the QR/LQ factorisations of the complex64
 *                    circuits also in FP64.
 *   MPS_MIXED_FAST   complex64 state also through lossy truncations (FP64 only for
 *                    the Gram matrix, the eigenvalues near the cut and the
 *                    re-orthogonalisation of the kept vectors): faster, but its error
 *                    in the truncated regime is NOT bounded by 1e-5; kept to measure
 *                    what the FP64 state of MPS_MIXED costs. */
typedef enum { MPS_FP64 = 0, MPS_MIXED = 1, MPS_MIXED_ORTH64 = 2, MPS_MIXED_FAST = 3 } mps_precision;

/* Circuit family.
 *   MPS_ANSATZ_LADDER  R_Y(pi x_k) once, then L x [R_Y(alpha_{l,k}) then R_Z(beta_{l,k})
 *                      on every qubit, CNOT(k -> k+1) for k = 0..n-2 in order].
 *   MPS_ANSATZ_PAPER   L x [H, R_Y(2 pi x_k - pi) (Eq. 2) on every qubit, CNOTs on bonds
 *                      (0,1),(2,3),... then (1,2),(3,4),..., each sub-layer ascending];
 *                      Sec. II.B. */
typedef enum { MPS_ANSATZ_LADDER = 0, MPS_ANSATZ_PAPER = 1 } mps_ansatz;

/* Pair set (Sec. II.C): horizontal + vertical neighbours (2p(p-1) pairs), or also
 * both diagonals (2p(p-1) + 2(p-1)^2 pairs: 156 at p = 7). */
typedef enum { MPS_PAIRS_HV = 0, MPS_PAIRS_HVD = 1 } mps_pair_set;

/* Largest accepted bond cap, and largest bond dimension the kernels hold.  Bonds up
 * to 32 run with their workspaces in shared memory; bonds of 64 and 128 run the same
 * kernels with one 256-thread (circuit) or 128-thread (Pauli cache) team per image and
 * the workspaces in global memory, allocated by the library (slower; the paper's
 * large-chi sweep). */
#define MPS_CHI_LIMIT 4096
#define MPS_BOND_LIMIT 128

typedef struct mps_batch mps_batch;

typedef struct {
    int32_t ansatz;              /* mps_ansatz */
    int32_t L;                   /* layers for every image, >= 0 (ignored if L_per_image) */
    const int32_t* L_per_image;  /* host [n_images] or NULL */
    const double* params;        /* device [L_max][params_n][2] angles (alpha, beta) in
                                    radians, LADDER only (NULL for PAPER); image i uses
                                    params[l][k][.] for l < L_i, k < n_i */
    int32_t params_n;            /* qubit stride of params, >= max n_i */
} mps_circuit;

/* Create a batch of n_images independent MPS (Sec. II.B, Eq. 3).
 *   p        host [n_images], image sides, 2 <= p_i <= 16 (n_i = p_i^2 qubits)
 *   chi      host [n_images] bond caps, or NULL to use chi_all for every image
 *   chi_all  bond cap when chi == NULL, 1 <= chi <= MPS_CHI_LIMIT.  Any chi is a cap:
 *            bonds only grow to min(chi, 2 D_left, 2 D_right) (e.g. at most 2^L for
 *            the ladder), and the kernels hold bonds up to MPS_BOND_LIMIT; a circuit
 *            that would need more returns MPS_ERR_UNSUPPORTED from mps_apply_circuit.
 *            Sites are padded for bonds up to min(chi, 2^floor(n/2), 32); a circuit that
 *            needs a larger bond lays the batch out again with a larger padding in
 *            mps_apply_circuit (that call waits for the stream and may allocate).  The
 *            pair set with diagonals is built for bonds up to 32.
 *   prec     mps_precision
 *   stream   cudaStream_t (NULL = legacy default stream) used by every later call
 *   out      receives the handle
 * The library allocates the MPS arena and its workspace on the current device
 * (about sum_i n_i * D_i^2 * 2 complex values, D_i the largest bond image i can
 * reach).  Returns MPS_ERR_OOM if that allocation fails. */
mps_status mps_create_batch(int32_t n_images, const int32_t* p, const int32_t* chi,
                            int32_t chi_all, int32_t prec, void* stream, mps_batch** out);

/* Give an existing batch a new list of images (same precision and stream), reusing
 * its device memory when the new layout fits and growing it otherwise.  Waits for
 * the batch's queued work first.  Arguments as in mps_create_batch.  A circuit must
 * be applied again before mps_pauli_cache.  Refused arguments (MPS_ERR_INVALID_ARG)
 * leave the batch unchanged; a reshape that fails later (MPS_ERR_OOM, MPS_ERR_CUDA)
 * leaves it allocated but unusable: mps_apply_circuit, mps_bond_dims and
 * mps_discarded_weight return MPS_ERR_NOT_READY until a reshape succeeds. */
mps_status mps_reshape_batch(mps_batch* batch, int32_t n_images, const int32_t* p, const int32_t* chi,
                             int32_t chi_all);

/* Allocate now, for the batch's current layout, every device buffer that a later
 * mps_apply_circuit may need: the left environments of operator-product images, and
 * under MPS_MIXED / MPS_MIXED_ORTH64 the complex128 sites of truncating chains, plus
 * gate tables for up to max(L_max, n_images) rows.  Afterwards mps_apply_circuit with
 * at most L_max layers, on this layout or a smaller one set by mps_reshape_batch,
 * allocates nothing (a serving loop then never stalls on cudaMalloc).  Waits for the
 * batch's stream if it grows a buffer.  MPS_ERR_OOM if an allocation fails. */
mps_status mps_reserve(mps_batch* batch, int32_t L_max);

/* Release a batch (stream-ordered: waits for its queued work first). NULL is a no-op. */
mps_status mps_destroy_batch(mps_batch* batch);

/* Run the circuit on every image (Sec. II.B): reset to |0...0>, apply the gate list,
 * and after every two-qubit gate truncate the bond to chi at the orthogonality
 * centre (keep the largest min(chi, 2D_left, 2D_right) singular values, renormalise).
 * A ladder circuit in which nothing is truncated, with 1 <= L <= 4 and 2^L within the
 * image's chi and site padding, is built exactly without any factorisation (the CNOT
 * ladder as a bond-2 operator, see mps_set_layer_pipeline): its MPS has bond 2^L at
 * every inner cut and is not left-canonical; the Pauli cache then contracts left
 * environments as well.  Same state, represented differently (mps_bond_dims).
 *   pixels  device, float64, packed [sum_i n_i] in image order, values in [0, 1]
 *   circ    host, see mps_circuit
 * Asynchronous.  A call that fails after its argument checks (MPS_ERR_UNSUPPORTED for
 * a circuit whose bond exceeds the image's padding, MPS_ERR_OOM, MPS_ERR_CUDA) leaves
 * no circuit on the batch: mps_pauli_cache returns MPS_ERR_NOT_READY until a call
 * succeeds. */
mps_status mps_apply_circuit(mps_batch* batch, const double* pixels, const mps_circuit* circ);

/* Pauli cache (Sec. II.C, Eq. 5): for every image-local pair and every alpha,
 * <P_a (x) P_b> / <psi|psi>.
 *   pair_set      mps_pair_set
 *   out           device, caller-owned, [sum_i m_i][16]; float64 for MPS_FP64,
 *                 float32 otherwise
 *   pair_offsets  host [n_images + 1] (may be NULL): receives the prefix sums of m_i
 * Returns MPS_ERR_NOT_READY if no circuit has run on the batch.  Asynchronous. */
mps_status mps_pauli_cache(mps_batch* batch, int32_t pair_set, void* out, int64_t* pair_offsets);

/* ANO features and linear reconstruction (Sec. II.A, II.C; Eq. 1, 4, 5, 6) for a batch
 * of images that share one pair layout of m pairs.
 *   pauli        device [n_images][m][16], float32 (pauli_f64 = 0) or float64 (= 1);
 *                1 <= n_images <= 2^31 - 1, m >= 1 (MPS_ERR_INVALID_ARG otherwise)
 *   abd          device float32 [m][16]: A[6] real off-diagonal, B[6] imaginary
 *                off-diagonal of H_q for (k,l) = (0,1),(0,2),(0,3),(1,2),(1,3),(2,3),
 *                D[4] diagonal; c_{q,alpha} = Tr(H_q P_alpha)/4 (Eq. 4)
 *   W, bias      device float32 [out_dim][m] and [out_dim]; W may be NULL (no linear
 *                layer, out ignored); bias may be NULL (zero)
 *   features     device float32 [n_images][m], q_q = sum_alpha c_{q,alpha} <P_alpha>
 *   out          device float32 [n_images][out_dim], y = W q + b
 *   stream       cudaStream_t
 * The linear layer runs on the tcgen05 tensor cores with a three-term TF32 split
 * (FP32-level accuracy).  Asynchronous. */
mps_status ano_features(const void* pauli, int32_t pauli_f64, int64_t n_images, int32_t m,
                        const float* abd, const float* W, const float* bias, int32_t out_dim,
                        float* features, float* out, void* stream);

/* Wait for the device and report whether a bounded wait inside the tensor-core
 * linear layer of ano_features gave up since the last call (MPS_ERR_TIMEOUT; the
 * flag is then cleared).  Setting the environment variable MPSANO_LINEAR=fp32
 * makes ano_features use a plain FP32 CUDA-core GEMM instead. */
mps_status ano_status(void);

/* ---- Training on cached Pauli expectations (Sec. II.C-D) ----
 * The Pauli cache depends on the image only, so it is computed once; a training
 * step then updates the observable parameters (A, B, D) and the linear layer
 * (W, b) from the cache alone.  The loss is the MSE term of Eq. 7,
 *   L = mse_weight * mean_{i,o} (y_hat[i][o] - y[i][o])^2,  y_hat = W q + b,
 * (the LPIPS term of Eq. 7 needs a pretrained network and is not part of this
 * library), and two Adam optimizers (Kingma and Ba, with bias correction) update
 * (A, B, D) and (W, b) with their own learning rates. */
typedef struct {
    float lr_abd;      /* learning rate of the (A, B, D) optimizer */
    float lr_linear;   /* learning rate of the (W, b) optimizer */
    float beta1;       /* first-moment decay, 0 <= beta1 < 1 (0.9) */
    float beta2;       /* second-moment decay, 0 <= beta2 < 1 (0.999) */
    float eps;         /* > 0, added to sqrt(v_hat) (1e-8) */
    float mse_weight;  /* lambda_MSE of Eq. 7 */
} ano_adam;

/* Floats of device workspace that ano_train_step needs (-1 on bad sizes).  Layout,
 * in floats: features [n_images][m] at 0, then d L / d y_hat [n_images][out_dim],
 * d L / d q [n_images][m], the gradient [m*16 + out_dim*m + out_dim] of
 * (abd, W, b) in that order, then FP64 scratch and the split-K partial tiles of
 * the two backward GEMMs. */
int64_t ano_train_workspace_floats(int64_t n_images, int32_t m, int32_t out_dim);

/* One full-batch training step, asynchronous on `stream`:
 *   pauli, pauli_f64   device Pauli cache [n_images*m][16] (FP32, or FP64 if pauli_f64)
 *   abd                device [m][16] observable parameters, updated in place
 *   W, bias            device [out_dim][m] and [out_dim], updated in place
 *   targets            device [n_images][out_dim] ground truth y
 *   adam_moments       device [2][m*16 + out_dim*m + out_dim] first then second
 *                      moments of (abd, W, b); caller-owned, zero before step 1
 *   step               Adam step number t >= 1 (bias correction 1 - beta^t)
 *   hp                 host hyper-parameters
 *   workspace          device, ano_train_workspace_floats() floats, 8-byte aligned
 *   loss               device double: the loss at the parameters before the update
 * The gradients are left in the workspace.  The three GEMMs (y_hat, d L / d q,
 * d L / d W) run on the tcgen05 tensor cores (3-term TF32 split); batch reductions
 * accumulate in FP64 in a fixed order, so a step is bit-reproducible.  Errors:
 * MPS_ERR_INVALID_ARG for NULL pointers, non-positive sizes, step < 1, beta
 * outside [0, 1), eps <= 0 or a misaligned workspace; a failed tensor-core wait is
 * reported by ano_status. */
mps_status ano_train_step(const void* pauli, int32_t pauli_f64, int64_t n_images, int32_t m, float* abd,
                          float* W, float* bias, int32_t out_dim, const float* targets, float* adam_moments,
                          int32_t step, const ano_adam* hp, float* workspace, double* loss, void* stream);

/* ---- diagnostics and control ------------------------------------------------ */

/* Wait for the batch's stream and return the first device-side error, if any. */
mps_status mps_sync(mps_batch* batch);

/* Thread-local text of the last non-OK status (never NULL). */
const char* mps_last_error(void);

/* Number of pairs of a p x p image for a pair set: 2p(p-1), plus 2(p-1)^2 for HVD. */
int64_t mps_pair_count(int32_t p, int32_t pair_set);

/* Copy bond dimensions to the host: out [sum_i (n_i + 1)], image i's block holds
 * D_0 = 1, D_1, ..., D_{n_i} = 1 (D_k = left bond of site k; 2^L at every inner cut
 * for an image built as an operator product, see mps_apply_circuit).  Synchronous. */
mps_status mps_bond_dims(mps_batch* batch, int32_t* out);

/* Copy per-image discarded weight sum_steps sum(dropped sigma^2)/sum(sigma^2) of
 * the last circuit to the host, out [n_images].  Synchronous. */
mps_status mps_discarded_weight(mps_batch* batch, double* out);

/* How mps_apply_circuit would run one image, computed on the host alone (no device
 * work; usable without a GPU).  out [4], host:
 *   out[0] route: 0 operator product (nothing truncates, 1 <= L <= 4, 2^L <= chi, bond
 *          2^L at every inner cut), 1 layer-pipelined (ladder, nothing truncates,
 *          L <= 4), 2 sequential kernel in the batch's precision, 3 sequential kernel on
 *          a complex128 state (a lossy truncation under MPS_MIXED / MPS_MIXED_ORTH64)
 *   out[1] largest bond of the image's MPS
 *   out[2] 1 if some step keeps fewer singular values than the rank (lossy), else 0
 *   out[3] site padding (power of two) the image gets in a batch
 * with layer_pipeline as set by mps_set_layer_pipeline.  MPS_ERR_INVALID_ARG for bad
 * arguments, MPS_ERR_UNSUPPORTED (out filled) when the bond exceeds MPS_BOND_LIMIT. */
mps_status mps_plan_image(int32_t p, int32_t L, int32_t chi, int32_t ansatz, int32_t prec,
                          int32_t layer_pipeline, int32_t* out);

/* Kernels this library has launched since it was loaded (all batches). */
uint64_t mps_launch_count(void);

/* Launch-shape knobs used by the autotuner (0 leaves a knob unchanged).
 *   images_per_cta   images per CTA of the circuit kernel when it runs one warp per
 *                    image, 1..8
 *   circuit_threads  threads that share one image in the circuit kernel: 32, 64 or 128
 *                    (64: the mixed path at bond bucket 16 without truncation; 128:
 *                    the complex128 truncation chains up to bond 16, which then use the
 *                    SM's four FP64 pipes for one image, for latency when few images
 *                    run at once; elsewhere one warp per image runs)
 *   pauli_threads    threads that share one (image, grid column) unit of the Pauli
 *                    kernel: 32, 64 or 128 (the pair set with diagonals always runs
 *                    with 64)
 * images_per_cta and pauli_threads leave every result bit-identical; circuit_threads
 * changes the summation order inside the QR splits (results agree to rounding). */
mps_status mps_set_launch_shape(mps_batch* batch, int32_t images_per_cta, int32_t circuit_threads,
                                int32_t pauli_threads);

/* Fast paths for ladder circuits (enable != 0: on, the default), chosen per image.
 * An image whose ladder circuit truncates nowhere (min(2 D_left, 2 D_right) <= chi at
 * every two-qubit gate) with 1 <= L <= 4:
 *  - if 2^L <= min(chi, site padding, 16): operator product.  The ladder of CNOTs maps
 *    |x_0 x_1 ...> to the prefix parities |x_0, x_0^x_1, ...>; as an operator its
 *    bond carries the running parity, so each layer (one-qubit gates, then the
 *    ladder) doubles every bond by copying entries, and every site tensor is built
 *    on its own (exact, no factorisation; bond 2^L; not left-canonical);
 *  - else: layer pipelining, one warp per layer; layer l applies its gate at bond k
 *    as soon as layer l-1 has finished bond k+1 (Sec. II.B's gate order is kept for
 *    every qubit), every split exact, the MPS equal to the sequential sweep's.
 * Other circuits, and every circuit with enable = 0, run the sequential sweep.  Takes
 * effect at the next mps_apply_circuit. */
mps_status mps_set_layer_pipeline(mps_batch* batch, int32_t enable);

/* Half-structured sites (enable != 0: on, the default).  A ladder circuit built as an
 * operator product leaves every site but the last with A[l][s][r] = 0 unless r lies
 * in half s of the right bond (the last layer's parity bit is the top bit of the
 * right index and equals the output bit); the environment and Pauli kernels then
 * contract over that half only.  The skipped terms are exact zeros, so results are
 * bit-identical with enable = 0 (the dense contractions), which exists to check
 * exactly that.  Takes effect at the next mps_apply_circuit. */
mps_status mps_set_half_structure(mps_batch* batch, int32_t enable);

/* Block solve in FP64 truncations (enable != 0: on, the default).  A truncation at
 * the orthogonality centre (Sec. II.B) keeps the span of the chi largest eigenvectors
 * of the Gram matrix of theta; the basis inside that span is a gauge of the new bond.
 * When FP64 Rayleigh quotients of the FP32-started eigenvectors place the cut in a gap
 * wider than 1e-5 of the largest eigenvalue, FP64 Jacobi then rotates only pairs with
 * one kept and one dropped direction.  With enable = 0 every FP64 truncation runs the
 * full FP64 eigen-decomposition; the truncated states agree to rounding, and the
 * switch exists to check exactly that.  Takes effect at the next mps_apply_circuit. */
mps_status mps_set_block_truncation(mps_batch* batch, int32_t enable);

/* Pauli-cache kernel choice under the mixed precisions at bonds up to 16:
 *   MPS_PAULI_COLUMN  one team per (image, grid column) walking the column, after
 *                     separate right and left environment chains;
 *   MPS_PAULI_SWEEP   one CTA per image walking its chain from the last site to the
 *                     first, carrying the right environment and the closings of every
 *                     pair still open (Sec. II.C, Eq. 5), so each transfer through a
 *                     site is one stacked product over all of them;
 *   MPS_PAULI_AUTO    (default) the sweep for batches of equal-size images whose sites
 *                     are all half-structured (operator-product ladder circuits), the
 *                     column walk otherwise (it measured faster on dense sites and on
 *                     mixed sizes).
 * The two kernels accumulate every sum in the same order: the results are
 * bit-identical.  A sweep that would not fit a block's shared memory runs the column
 * walk.  Takes effect at the next mps_pauli_cache. */
#define MPS_PAULI_COLUMN 0
#define MPS_PAULI_SWEEP 1
#define MPS_PAULI_AUTO 2
mps_status mps_set_pauli_sweep(mps_batch* batch, int32_t mode);

/* Real-element environment and Pauli kernels for a real state (enable != 0: on, the
 * default).  The paper ansatz's gates (H, R_Y(2 pi x - pi), CNOT) are real, so its state
 * is real in every amplitude; under the mixed precisions the environment and Pauli
 * kernels then contract real matrices (a quarter of the multiply-adds), and every Pauli
 * with one Y is exactly zero.  enable = 0 runs the complex kernels (results agree to
 * rounding).  Takes effect at the next mps_apply_circuit. */
mps_status mps_set_real_arithmetic(mps_batch* batch, int32_t enable);

/* Per-launch timing with CUDA events recorded on the batch's stream around each
 * kernel the batch launches (enable != 0 turns it on; off by default). */
mps_status mps_set_timing(mps_batch* batch, int32_t enable);

/* Sum of the recorded launch durations since the last call, per kernel kind
 * (0 circuit, 1 environments: right, and left for images whose ladder circuit ran
 * as an operator product, 2 Pauli cache): ms [3], launches [3].
 * Synchronises the batch's stream, then clears the records. */
mps_status mps_kernel_times(mps_batch* batch, double* ms, int64_t* launches);

/* ---- Pauli cache without device allocation ------------------------------------
 * The paper has no counterpart to this call; it exists for callers that cannot
 * allocate device memory themselves or through this library:
 *   - plug-ins inside a host application whose GPU memory is owned by another
 *     allocator or a fixed pool, where an extra cudaMalloc fails or breaks that
 *     application's accounting;
 *   - processes whose framework reserves the whole GPU at start-up, so that any
 *     later cudaMalloc runs out of memory;
 *   - latency-bound serving loops, where cudaMalloc/cudaFree can synchronise the
 *     device and stall every stream.
 * It computes the same Pauli cache as mps_create_batch + mps_apply_circuit +
 * mps_pauli_cache for n_images images of one size, MPS_MIXED precision (a circuit
 * that truncates lossily runs on a complex128 state, as there), the ladder ansatz
 * and the horizontal + vertical pair set, using the same kernels.  All working
 * memory (site tensors, their complex128 copies for a truncating circuit, the
 * workspace of a truncation at bond 32, environments, bond dimensions, per-image
 * records, the status word) lives in one fixed array inside this library's device
 * memory (about 62 MiB, held on every GPU that loads the library until the process
 * exits).
 *   n_images  1..64
 *   p, chi, L image side 2..16, bond cap 1..32, layers >= 0
 *   pixels    device float64 [n_images][p*p], values in [0, 1]
 *   params    device float64 [>= L][params_n][2] angles, params_n >= p*p (may be NULL if L == 0)
 *   out       device float32 [n_images][2p(p-1)][16], caller-owned
 *   status    device int32, caller-owned, or NULL: receives, in stream order after the
 *             Pauli cache, the first device-side error of this call (0 = none; 1 = a
 *             bond exceeded the padding the host sized, 3 = a step the kernel does not
 *             support), which the kernels record instead of writing out of bounds
 *   stream    cudaStream_t
 * Limits: with ld the smallest power of two >= 4 that holds the largest bond the
 * circuit reaches, n_images * p^2 * 2 * ld^2 * 8 bytes <= 12 MiB of site storage and
 * n_images * p^2 * ld^2 * 8 bytes <= 6 MiB of environments (e.g. up to 62 images of
 * 7x7 at chi = 16, L = 4), and L * p^2 <= 16384.  Larger requests return
 * MPS_ERR_INVALID_ARG with a message.
 * No cudaMalloc, cudaFree or other allocating routine is called.  The first call on a
 * device looks up the array's device address with that device current; make that
 * first call before any stream capture.  Every call reuses the same array and
 * overwrites the previous call's contents (per-call state, the status word included,
 * is cleared at its start), so calls that overlap on the GPU -- on different streams
 * or from different threads -- race and corrupt each other: keep them on one stream.
 * Asynchronous on stream. */
mps_status mps_pauli_cache_noalloc(int32_t n_images, int32_t p, int32_t chi, int32_t L,
                                   const double* pixels, const double* params, int32_t params_n,
                                   float* out, int32_t* status, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* MPSANO_H */
