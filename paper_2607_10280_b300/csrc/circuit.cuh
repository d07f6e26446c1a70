// Circuit kernel: one warp owns one image's MPS (Sec. II.B, Eq. 3) for the whole
// circuit.  The warp sweeps the chain left to right applying the two-qubit gates
// in their fixed order; the orthogonality centre travels with the sweep.  Each
// two-qubit step forms theta = A_k A_{k+1} on the fly (with the one-qubit gates of
// the layer folded into the load of A_{k+1}), applies the gate as a row/column
// permutation (CNOT) and splits theta back into two sites:
//
//   * min(M, N) <= chi (nothing to truncate): exact split.  N <= M: Householder
//     QR, A_k = Q, A_{k+1} = R.  M < N: A_k = I_M, A_{k+1} = theta.  The state is
//     the one the SVD split would give, in another gauge of the new bond.
//   * Each CNOT at most doubles the Schmidt rank across its cut, so after c CNOTs
//     the rank is at most 2^c and a split keeps at most cap = min(chi, 2^c).
//     min(M, N) > cap = 2^c <= chi: theta has rank <= cap, and a Householder QR
//     with column pivoting stopped after cap steps splits it exactly up to
//     rounding, in any gauge (the paper ansatz's odd-bond sub-layer needs it).
//   * min(M, N) > cap = chi < 2^c: SVD truncation at the orthogonality centre.  Gram matrix of
//     the smaller side in FP64; cyclic Jacobi eigensolver (FP64 path: in FP64;
//     mixed path: in FP32 on the rounded Gram, the eigenvalues near the cut refined
//     as FP64 Rayleigh quotients, and solved again in FP64 when the gap at the cut
//     is below 1e-3 of the largest); keep the chi largest, A_k = U_chi (re-orthogonalised by an FP64
//     Householder QR unless it came from an FP64 solve of the left Gram),
//     A_{k+1} = U_chi^H theta rescaled to unit norm.
//
// Before a pass in which some step truncates, a right-to-left LQ sweep moves the
// centre to the first site of the pass so that every truncation happens at the
// true orthogonality centre (the sites to its right are right-orthonormal).
// Passes without truncation skip that sweep: their splits are exact in any gauge.
// After the last pass the MPS is left-canonical with the centre at site n-1,
// which is the form the Pauli kernel expects.
//
// Shared memory is private to each warp; the kernel has no block-wide barriers.
#pragma once
#include "common.cuh"
#include "linalg.cuh"

namespace mpsano {

constexpr int MAX_QUBITS = 256;  // p <= 16

// Per-warp shared-memory layout.  CHI bounds every bond the images reach.
// With TRUNC the site buffers (cur, nxt, rb) share one region with the FP64 Gram
// matrix and eigenvectors (G, V) of the SVD truncation: theta is formed from cur and
// nxt before G is written, rb serves only the exact centre moves, and the new centre
// is written to cur (inside G) only after the last read of U (held in G), from V.
// That keeps the FP64 Gram and eigenvector workspace of a bond-32 truncation at about
// 205 KB; with the FP64 basis W of the refined eigen-decomposition (REFINE) the layout
// grows to about 270 KB, which launch_circuit places in global memory.
template <typename T, typename TQ, int CHI, bool TRUNC>
struct CircuitLayout {
    static constexpr int CS = CHI + 1;              // row stride of a site: element (l,s,r) at (2l+s)*CS + r
    static constexpr int SITE = 2 * CHI * CS;       // complex elements of a site buffer
    static constexpr int LDM = 2 * CHI + 1;         // column stride of theta (column-major)
    static constexpr int THETA = 2 * CHI * LDM;
    static constexpr int K = 2 * CHI;               // largest Gram matrix
    static constexpr int LDK = K + 1;
    static constexpr size_t SITES_BYTES = sizeof(cx<T>) * (2 * SITE + CHI * CS);
    static constexpr size_t GV_BYTES = TRUNC ? 2 * sizeof(cx<double>) * K * LDK : 0;
    static constexpr size_t REGION = ((SITES_BYTES > GV_BYTES ? SITES_BYTES : GV_BYTES) + 15) & ~size_t(15);
    static constexpr size_t off_cur = 0;
    static constexpr size_t off_nxt = off_cur + sizeof(cx<T>) * SITE;
    static constexpr size_t off_rb = off_nxt + sizeof(cx<T>) * SITE;
    static constexpr size_t off_gram = 0;
    static constexpr size_t off_vec = off_gram + (TRUNC ? sizeof(cx<double>) * K * LDK : 0);
    static constexpr size_t off_th = REGION;
    static constexpr size_t off_tau = off_th + sizeof(cx<TQ>) * THETA;
    static constexpr size_t off_bd = off_tau + sizeof(cx<TQ>) * K;
    static constexpr size_t off_cn = off_bd + sizeof(int) * (MAX_QUBITS + 1);   // CNOTs per cut
    static constexpr size_t off_perm = off_cn + sizeof(int) * (MAX_QUBITS + 1);  // pivoted QR
    static constexpr size_t off_cnorm = (off_perm + sizeof(int) * K + 15) & ~size_t(15);
    static constexpr size_t off_cz = off_cnorm + sizeof(TQ) * K;                  // zero rows of cur
    static constexpr size_t off_taud = (off_cz + sizeof(int) + 15) & ~size_t(15);
    static constexpr size_t off_lam = off_taud + (TRUNC ? sizeof(cx<double>) * K : 0);
    static constexpr size_t off_ord = off_lam + (TRUNC ? sizeof(double) * K : 0);
    static constexpr size_t off_red = (off_ord + (TRUNC ? sizeof(int) * K : 0) + 15) & ~size_t(15);
    static constexpr size_t off_flag = off_red + sizeof(double) * 8;   // team reductions (<= 256 threads)
    // FP64 truncation: the eigen-decomposition starts from FP32 Jacobi vectors, made
    // orthonormal in FP64 in the buffer W (see svd_truncate); from bond 32 on the layout
    // exceeds a block's shared memory and the kernel runs on a global-memory workspace
    static constexpr bool REFINE = TRUNC && sizeof(TQ) == 8;
    static constexpr size_t off_w = (off_flag + sizeof(int) + 15) & ~size_t(15);
    static constexpr size_t bytes = (off_w + (REFINE ? sizeof(cx<double>) * K * LDK : 0) + 15) & ~size_t(15);
    // the new centre (in cur) is written from V, so the two must not overlap
    static_assert(!TRUNC || off_cur + sizeof(cx<T>) * SITE <= off_vec, "cur must lie within the Gram buffer");
};

// The 2x2 one-qubit gate applied to site k at the start of a layer.
template <typename T>
struct Gate1 { cx<T> u00, u01, u10, u11; };

// One-qubit gate of (layer, site k) from the table written by gate_table_kernel:
// ladder ansatz gates[(layer * gn + k) * 4 + e], paper ansatz gates[(img * gn + k) * 4 + e]
// (the paper layer gate depends on the pixel, not on the layer).
template <typename T>
__device__ __forceinline__ Gate1<T> table_gate(const cx<T>* gates, int gn, int ansatz, int layer, int img, int k) {
    const cx<T>* g = gates + ((size_t)(ansatz == 0 ? layer : img) * gn + k) * 4;
    Gate1<T> u;
    u.u00 = g[0]; u.u01 = g[1]; u.u10 = g[2]; u.u11 = g[3];
    return u;
}

// Gate table in FP64, rounded to the state type once per launch.
//   ladder: entry (layer, k) = R_Z(beta_{layer,k}) R_Y(alpha_{layer,k})
//   paper:  entry (img, k)   = R_Y(2 pi x_k - pi) H   (Eq. 2)
template <typename T>
__global__ void gate_table_kernel(int ansatz, int rows, int gn, const double* __restrict__ params, int params_n,
                                  const ImageMeta* __restrict__ meta, const double* __restrict__ pixels,
                                  cx<T>* __restrict__ gates) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= rows * gn) return;
    const int row = t / gn, k = t % gn;
    double u[8];
    if (ansatz == 0) {
        const double a = params[((size_t)row * params_n + k) * 2 + 0];
        const double b = params[((size_t)row * params_n + k) * 2 + 1];
        double sa, ca, sb, cb;
        sincos(0.5 * a, &sa, &ca);
        sincos(0.5 * b, &sb, &cb);
        // e^{-ib/2} = (cb, -sb), e^{ib/2} = (cb, sb), R_Y(a) = [[ca, -sa], [sa, ca]]
        u[0] = cb * ca;  u[1] = -sb * ca;
        u[2] = -cb * sa; u[3] = sb * sa;
        u[4] = cb * sa;  u[5] = sb * sa;
        u[6] = cb * ca;  u[7] = sb * ca;
    } else {
        const ImageMeta m = meta[row];
        const double x = k < m.n ? pixels[m.pixel_off + k] : 0.0;
        double sn, c;
        sincos(0.5 * (2.0 * M_PI * x - M_PI), &sn, &c);
        const double h = 0.70710678118654752440;
        u[0] = h * (c - sn); u[1] = 0.0;   // [c -s; s c] [1 1; 1 -1] / sqrt 2
        u[2] = h * (c + sn); u[3] = 0.0;
        u[4] = h * (sn + c); u[5] = 0.0;
        u[6] = h * (sn - c); u[7] = 0.0;
    }
    cx<T>* g = gates + (size_t)t * 4;
    for (int e = 0; e < 4; ++e) g[e] = mk<T>(T(u[2 * e]), T(u[2 * e + 1]));
}

// Global site (Dl x 2 x Dr, padded [ld][2][ld]) -> shared site buffer, optionally
// applying a one-qubit gate on the physical index.
template <typename T, int CS, int NTHR>
__device__ __forceinline__ void load_site(cx<T>* dst, const cx<T>* src, int ld, int Dl, int Dr,
                                          const Gate1<T>* g, int lane) {
    team_for_2d<NTHR>(Dl, Dr, lane, [&](int l, int r) {
        const cx<T> a0 = src[(2 * l) * ld + r], a1 = src[(2 * l + 1) * ld + r];
        if (g) {
            dst[(2 * l) * CS + r] = cdot2(g->u00, a0, g->u01, a1);
            dst[(2 * l + 1) * CS + r] = cdot2(g->u10, a0, g->u11, a1);
        } else {
            dst[(2 * l) * CS + r] = a0;
            dst[(2 * l + 1) * CS + r] = a1;
        }
    });
}

template <typename T, int CS, int NTHR>
__device__ __forceinline__ void store_site(cx<T>* dst, const cx<T>* src, int ld, int Dl, int Dr, int lane) {
    team_for_2d<NTHR>(2 * Dl, Dr, lane, [&](int row, int r) { dst[row * ld + r] = src[row * CS + r]; });
}

template <typename T, int CS, int NTHR>
__device__ __forceinline__ void apply_gate_smem(cx<T>* site, int Dl, int Dr, const Gate1<T>& g, int lane) {
    team_for_2d<NTHR>(Dl, Dr, lane, [&](int l, int r) {
        const cx<T> a0 = site[(2 * l) * CS + r], a1 = site[(2 * l + 1) * CS + r];
        site[(2 * l) * CS + r] = cdot2(g.u00, a0, g.u01, a1);
        site[(2 * l + 1) * CS + r] = cdot2(g.u10, a0, g.u11, a1);
    });
}

template <typename T, typename TQ, int CHI, bool TRUNC, int NTHR>
struct CircuitTeam {
    using Lay = CircuitLayout<T, TQ, CHI, TRUNC>;
    static constexpr int CS = Lay::CS, LDM = Lay::LDM, LDK = Lay::LDK;

    cx<T>* cur;   // centre tensor of the sweep
    cx<T>* nxt;   // next site
    cx<T>* rb;    // small triangular factor
    cx<TQ>* th;   // theta, column-major M x N, rows (l,s), columns (t,r)
    cx<TQ>* tau;
    int* bd;      // bd[k] = left bond of site k, k = 0..n
    int* cn;      // cn[k] = CNOTs applied so far across the cut left of site k
    int* perm;    // column order of a pivoted QR
    TQ* cnorm;    // its column norms
    // cur = R of a QR split is upper triangular, so its rows (l, s = 0) with l >= D_m
    // of the next step are zero: *czp holds that D_m (NOZ: no known zero rows).  zr:
    // rows (l, 0), l >= zr, left out of this step's theta (zr = Dl: none).
    static constexpr int NOZ = 1 << 30;
    int* czp;
    int zr;
    cx<double>* G;
    cx<double>* V;
    cx<double>* W;   // FP64 eigenvector basis of the refined eigen-decomposition (Lay::REFINE)
    cx<double>* taud;
    double* lam;
    int* ord;
    double* red;  // team reductions
    int* flag;    // team broadcast
    int lane, n, chi, ld;
    int keep;     // singular values an SVD truncation keeps
    bool block_trunc;   // FP64 truncations may use the block solve (META_FULL_EIGH clear)
    cx<T>* sites;        // this image's site 0 in the arena
    double discarded;
    int* status;

    __device__ cx<T>* site_ptr(int k) const { return sites + (size_t)k * (2 * ld * ld); }

    // ---- theta = cur(Dl x 2 x Dm) nxt(Dm x 2 x Dr), CNOT(control = left) folded in ----
    // theta = cur nxt with the structurally zero rows of cur left out when
    // allow_compact: compact row q is (l, s) = (q / 2, q % 2) for q < 2 zr, then
    // (zr + q - 2 zr, 1); the QR of the compact theta needs 2 Dr <= Dl + zr rows.
    __device__ void form_theta(int Dl, int Dm, int Dr, bool cnot, bool allow_compact = false) {
        const int N = 2 * Dr;
        int z = *czp < Dl ? *czp : Dl;
        if (!(allow_compact && z < Dl && N <= Dl + z)) z = Dl;
        zr = z;
        const int M = Dl + z;
        team_for_2d<NTHR>(M, N, lane, [&](int q, int c) {
            const int row = q < 2 * z ? q : 2 * (q - z) + 1;    // (l, s) -> 2 l + s
            const int s = row & 1;
            int t = c >= Dr ? 1 : 0;
            const int r = c - t * Dr;
            if (cnot && s) t ^= 1;
            cx<T> acc0 = czero<T>(), acc1 = czero<T>();
            const cx<T>* a = cur + row * CS;
            const cx<T>* b = nxt + t * CS + r;
            int m = 0;
            for (; m + 1 < Dm; m += 2) {
                cmac(acc0, a[m], b[2 * m * CS]);
                cmac(acc1, a[m + 1], b[2 * (m + 1) * CS]);
            }
            if (m < Dm) cmac(acc0, a[m], b[2 * m * CS]);
            th[c * LDM + q] = cvt<TQ>(acc0 + acc1);
        });
        tsync<NTHR>();
        if (lane == 0) *czp = NOZ;   // consumed; a QR split sets it again
    }

    // Householder QR of theta (M x N, N <= M) in place; R (N x N) reshaped (N, 2, Dr)
    // becomes the new centre; the reflectors and tau stay in th / tau.
    __device__ void qr_to_cur(int M, int N, int Dr) {
        team_qr<NTHR>(th, LDM, M, N, tau, red, lane);
        team_for_2d<NTHR>(N, N, lane, [&](int i, int c) {
            const int t = c >= Dr ? 1 : 0, r = c - t * Dr;
            const cx<TQ> v = (i <= c) ? th[c * LDM + i] : czero<TQ>();
            cur[(2 * i + t) * CS + r] = cvt<T>(v);
        });
        tsync<NTHR>();
    }

    // The explicit Q (M x K) of the reflectors in th / tau, stored as site k; with
    // compaction (z < Dl) compact row q goes to row 2 l + s and the left-out rows
    // (l, 0), l >= z, are zero.
    __device__ void q_to_site(int k, int M, int K, int Dl, int z) {
        cx<T>* dst = site_ptr(k);
        team_form_q<NTHR>(th, LDM, M, K, tau, lane);
        team_for_2d<NTHR>(M, K, lane, [&](int q, int c) {
            const int row = q < 2 * z ? q : 2 * (q - z) + 1;
            dst[row * ld + c] = cvt<T>(th[c * LDM + q]);
        });
        team_for_2d<NTHR>(Dl - z, K, lane, [&](int i, int c) { dst[2 * (z + i) * ld + c] = czero<T>(); });
        tsync<NTHR>();
    }

    // Exact split (nothing dropped).  N <= M: Householder QR, A_k = Q (M x N),
    // cur = R (N x N) reshaped (N, 2, Dr).  M < N: A_k = I_M, cur = theta reshaped
    // (M, 2, Dr).  Returns the new bond dimension.
    __device__ int split_exact(int k, int Dl, int Dr) {
        const int M = 2 * Dl, N = 2 * Dr;
        if (N <= M) {
            qr_to_cur(Dl + zr, N, Dr);
            if (lane == 0) *czp = Dr;
            q_to_site(k, Dl + zr, N, Dl, zr);
            return N;
        }
        cx<T>* dst = site_ptr(k);
        team_for_2d<NTHR>(M, M, lane, [&](int row, int c) { dst[row * ld + c] = mk<T>(T(row == c ? 1 : 0), T(0)); });
        team_for_2d<NTHR>(M, N, lane, [&](int i, int c) {
            const int t = c >= Dr ? 1 : 0, r = c - t * Dr;
            cur[(2 * i + t) * CS + r] = cvt<T>(th[c * LDM + i]);
        });
        tsync<NTHR>();
        return M;
    }

    // ---- split theta (M x N) into site k (written to global) and cur (new centre) ----
    // cap: most singular values the split may keep, min(chi, 2^c) with c the CNOTs
    // that have crossed this cut (each at most doubles the Schmidt rank).
    // min(M, N) <= cap: exact QR / identity split.  Otherwise exact_cap (cap = 2^c
    // <= chi, so theta has rank <= cap): rank-revealing split by pivoted QR, which
    // drops only rounding noise.  Otherwise (cap = chi < 2^c) an SVD truncation to
    // chi; the caller has moved the orthogonality centre here first.
    // Returns the new bond dimension.
    __device__ int split(int k, int Dl, int Dr, int cap, bool exact_cap) {
        const int M = 2 * Dl, N = 2 * Dr;
        const int mn = M < N ? M : N;
        if (mn <= cap) return split_exact(k, Dl, Dr);
        if (exact_cap) return rank_split(k, M, N, Dr, cap);
        if constexpr (TRUNC) {
            keep = cap;
            return svd_truncate(k, Dl, Dr);
        } else {
            raise_status(status, DEV_BAD_SHAPE);
            return cap;
        }
    }

    // Rank-revealing split of theta (M x N, rank <= cap < min(M, N)): pivoted QR
    // stopped after cap reflectors, A_k = Q (M x cap), cur = R P^T (cap x N)
    // reshaped (cap, 2, Dr).  The discarded rows of R are rounding noise.
    __device__ int rank_split(int k, int M, int N, int Dr, int cap) {
        team_qrcp<NTHR>(th, LDM, M, N, cap, tau, perm, cnorm, red, lane);
        team_for_2d<NTHR>(cap, N, lane, [&](int i, int c) {
            const int oc = perm[c];
            const int t = oc >= Dr ? 1 : 0, r = oc - t * Dr;
            const cx<TQ> v = (i <= c) ? th[c * LDM + i] : czero<TQ>();
            cur[(2 * i + t) * CS + r] = cvt<T>(v);
        });
        tsync<NTHR>();
        q_to_site(k, M, cap, M / 2, M / 2);
        return cap;
    }

    // SVD truncation of theta (M x N) to keep singular values, min(M, N) > keep.
    __device__ int svd_truncate(int k, int Dl, int Dr) {
        const int M = 2 * Dl, N = 2 * Dr;
        const bool left = M <= N;      // Gram of the row space (M x M) or column space (N x N)
        const int K = left ? M : N;
        // G = theta theta^H (left) or theta^H theta, accumulated in FP64
        team_for_upper<NTHR>(K, lane, [&](int i, int j) {   // G[i][j], column-major store G[j*LDK + i]
            cx<double> acc = czero<double>();
            if (left) {
                for (int c = 0; c < N; ++c)
                    cmac(acc, cvt<double>(th[c * LDM + i]), conj(cvt<double>(th[c * LDM + j])));
            } else {
                for (int r = 0; r < M; ++r)
                    cmac_cj(acc, cvt<double>(th[i * LDM + r]), cvt<double>(th[j * LDM + r]));
            }
            G[j * LDK + i] = acc;
            G[i * LDK + j] = conj(acc);
        });
        tsync<NTHR>();
        // Eigen-decomposition of G.  FP64 path: Jacobi in FP64 in place (diag(G) = sigma^2,
        // V = eigenvectors).  Mixed path: Jacobi in FP32 on a rounded copy (in the V
        // buffer), sigma^2 near the cut refined as FP64 Rayleigh quotients v_i^H G v_i of
        // the FP64 Gram, and the kept vectors re-orthogonalised in FP64 below.
        cx<float>* G32 = reinterpret_cast<cx<float>*>(V);
        cx<float>* V32 = G32 + K * LDK;
        // rank the eigenvalues lam (descending, ties by index) into ord
        auto rank_lam = [&]() {
            for (int i = lane; i < K; i += NTHR) {
                const double li = lam[i];
                int rank = 0;
                for (int j = 0; j < K; ++j) rank += (lam[j] > li) || (lam[j] == li && j < i);
                ord[rank] = i;
            }
            tsync<NTHR>();
        };
        bool fp64_vectors = sizeof(TQ) == 8;
        bool cross = false;   // the refined solve decoupled the kept part only
        const cx<double>* Vd = V;   // FP64 eigenvectors (columns), when fp64_vectors
        if constexpr (sizeof(TQ) == 8) {
            if constexpr (Lay::REFINE) {
                // The same FP64 eigen-decomposition as a Jacobi solve from scratch, at a
                // fraction of its FP64 work: FP32 Jacobi on the rounded Gram gives
                // vectors accurate to ~eps_32; they are made orthonormal in FP64 (Cholesky
                // QR: their Gram matrix is I + O(eps_32), so R is perfectly conditioned),
                // G becomes W^H G W in FP64, and FP64 Jacobi started from W (v_given)
                // only has to remove off-diagonal entries of size ~eps_32 lambda_1 (two
                // rotating sweeps instead of six to eight; clusters of eigenvalues below
                // FP32 resolution are resolved by the same sweeps).
                team_for_2d<NTHR>(K, K, lane, [&](int c, int r) { G32[c * LDK + r] = cvt<float>(G[c * LDK + r]); });
                tsync<NTHR>();
                team_jacobi_eigh<NTHR, float>(G32, V32, LDK, K, lane, 40, red);
                tsync<NTHR>();
                team_for_2d<NTHR>(K, K, lane, [&](int c, int r) { W[c * LDK + r] = cvt<double>(V32[c * LDK + r]); });
                tsync<NTHR>();
                // C = W^H W (upper triangle, column-major in the V buffer), then C = R^H R
                cx<double>* C = V;
                team_for_upper<NTHR>(K, lane, [&](int i, int j) {
                    cx<double> acc = czero<double>();
                    for (int r = 0; r < K; ++r) cmac_cj(acc, W[i * LDK + r], W[j * LDK + r]);
                    C[j * LDK + i] = acc;
                });
                tsync<NTHR>();
                for (int k = 0; k < K; ++k) {
                    // 1/sqrt in one call (rsqrt, within about an ulp): the pivot is
                    // 1 + O(eps_32), far from any range rsqrt treats specially
                    const double inv = rsqrt(C[k * LDK + k].re);
                    const double d = C[k * LDK + k].re * inv;
                    tsync<NTHR>();
                    for (int j = k + lane; j < K; j += NTHR)
                        C[j * LDK + k] = j == k ? mk<double>(d, 0.0) : inv * C[j * LDK + k];
                    if (lane == 0) taud[k] = mk<double>(inv, 0.0);
                    tsync<NTHR>();
                    team_for_upper<NTHR>(K - 1 - k, lane, [&](int ii, int jj) {
                        const int i = k + 1 + ii, j = k + 1 + jj;
                        cmsub(C[j * LDK + i], conj(C[i * LDK + k]), C[j * LDK + k]);
                    });
                    tsync<NTHR>();
                }
                // W <- W R^{-1}, row by row (forward substitution over the columns).  A
                // group of GS lanes takes a row (GS * K <= NTHR, GS <= 32), each lane the
                // terms m = g (mod GS) of every column's sum, combined by xor-shuffles, so
                // that no lane of a warp idles when K < NTHR.
                {
                    int GS = 1;
                    while (GS < 32 && 2 * GS * K <= NTHR) GS *= 2;
                    const int g = lane & (GS - 1), groups = NTHR / GS;
                    for (int r0 = 0; r0 < K; r0 += groups) {
                        const int r = r0 + lane / GS;
                        const bool live = r < K;
                        for (int c = 0; c < K; ++c) {
                            cx<double> part = czero<double>();
                            if (live)
                                for (int m = g; m < c; m += GS) cmac(part, W[m * LDK + r], C[c * LDK + m]);
                            for (int o = GS >> 1; o > 0; o >>= 1) {
                                part.re += __shfl_xor_sync(0xffffffffu, part.re, o);
                                part.im += __shfl_xor_sync(0xffffffffu, part.im, o);
                            }
                            if (live && g == 0) W[c * LDK + r] = taud[c].re * (W[c * LDK + r] - part);
                            __syncwarp();
                        }
                    }
                }
                tsync<NTHR>();
                // G <- W^H (G W), through T = G W in the V buffer
                cx<double>* Tm = V;
                team_for_2d<NTHR>(K, K, lane, [&](int c, int r) {
                    cx<double> acc = czero<double>();
                    for (int m = 0; m < K; ++m) cmac(acc, G[m * LDK + r], W[c * LDK + m]);
                    Tm[c * LDK + r] = acc;
                });
                tsync<NTHR>();
                // W^H G W is Hermitian: the upper triangle, mirrored
                team_for_upper<NTHR>(K, lane, [&](int i, int j) {
                    cx<double> acc = czero<double>();
                    for (int r = 0; r < K; ++r) cmac_cj(acc, W[i * LDK + r], Tm[j * LDK + r]);
                    if (i == j) acc.im = 0.0;
                    G[j * LDK + i] = acc;
                    G[i * LDK + j] = conj(acc);
                });
                tsync<NTHR>();
                // diag(G) now holds FP64 Rayleigh quotients of the FP32 vectors (error
                // ~eps_32 lambda_1 at worst, inside a cluster).  Where they put the cut in a
                // gap wider than 1e-5 lambda_1 that split is certain, and FP64 Jacobi only
                // has to decouple the kept from the dropped directions (team_jacobi_cross:
                // the rotations inside either part change nothing a truncation uses);
                // otherwise the full FP64 eigen-decomposition ranks them.
                for (int i = lane; i < K; i += NTHR) lam[i] = G[i * LDK + i].re;
                tsync<NTHR>();
                rank_lam();
                cross = block_trunc && lam[ord[keep - 1]] - lam[ord[keep]] >= 1e-5 * lam[ord[0]];
                if (cross) team_jacobi_cross<NTHR, double>(G, W, LDK, K, ord, keep, lane, 40, red);
                else team_jacobi_eigh<NTHR, double>(G, W, LDK, K, lane, 40, red, true);
                Vd = W;
            } else {
                team_jacobi_eigh<NTHR, double>(G, V, LDK, K, lane, 40, red);
            }
            tsync<NTHR>();
            for (int i = lane; i < K; i += NTHR) lam[i] = G[i * LDK + i].re;
            tsync<NTHR>();
            // after the block solve ord keeps its split (kept part first)
            if (!cross) rank_lam();
        } else {
            team_for_2d<NTHR>(K, K, lane, [&](int c, int r) { G32[c * LDK + r] = cvt<float>(G[c * LDK + r]); });
            tsync<NTHR>();
            team_jacobi_eigh<NTHR, float>(G32, V32, LDK, K, lane, 40, red);
            tsync<NTHR>();
            // lambda from the FP32 Jacobi (absolute error ~ eps_32 lambda_1) ranks the
            // vectors.  Only near the cut can that ranking or the tie test below need
            // more: the vectors whose eigenvalue lies within 2e-3 lambda_1 of the cut get
            // lambda = v^H G v in FP64 (Rayleigh quotients of the FP64 Gram, error
            // ~ eps_32^2 lambda_1); elsewhere FP64 work on this part is 1/58 of FP32.
            for (int i = lane; i < K; i += NTHR) lam[i] = (double)G32[i * LDK + i].re;
            tsync<NTHR>();
            rank_lam();
            {
                const double l1 = lam[ord[0]];
                const double lc = 0.5 * (lam[ord[keep - 1]] + lam[ord[keep]]);
                if (lam[ord[keep - 1]] - lam[ord[keep]] < 2e-3 * l1) {
                    for (int i = lane; i < K; i += NTHR) {
                        if (fabs(lam[i] - lc) > 2e-3 * l1) continue;
                        cx<double> acc = czero<double>();
                        const cx<float>* v = V32 + i * LDK;
                        for (int r = 0; r < K; ++r) {
                            cx<double> gv = czero<double>();
                            for (int c = 0; c < K; ++c) cmac(gv, G[c * LDK + r], cvt<double>(v[c]));
                            cmac_cj(acc, cvt<double>(v[r]), gv);
                        }
                        lam[i] = acc.re;
                    }
                    tsync<NTHR>();
                    rank_lam();
                }
            }
            // Near a tie at the cut the FP32 eigenvectors mix the kept and the dropped
            // directions at the FP32 rounding level; there the eigenproblem is solved
            // again in FP64 (G still holds the FP64 Gram, V is free for FP64 vectors).
            // A tie between negligible eigenvalues (lambda_keep <= 1e-12 lambda_1)
            // needs no redo: whichever of those directions is kept, the state moves
            // by at most sqrt(2 lambda_keep / lambda_1) <= 1.5e-6 of its norm.
            const double gap = lam[ord[keep - 1]] - lam[ord[keep]];
            if (gap < 1e-3 * lam[ord[0]] && lam[ord[keep - 1]] > 1e-12 * lam[ord[0]]) {
                team_jacobi_eigh<NTHR, double>(G, V, LDK, K, lane, 40, red);
                tsync<NTHR>();
                for (int i = lane; i < K; i += NTHR) lam[i] = G[i * LDK + i].re;
                tsync<NTHR>();
                rank_lam();
                fp64_vectors = true;
            }
        }
        // discarded weight of this step
        double tot = 0.0, drop = 0.0;
        for (int i = lane; i < K; i += NTHR) {
            const double w = lam[ord[i]] > 0.0 ? lam[ord[i]] : 0.0;
            tot += w;
            if (i >= keep) drop += w;
        }
        tot = team_sum<NTHR>(tot, red, lane);
        drop = team_sum<NTHR>(drop, red, lane);
        if (tot > 0.0) discarded += drop / tot;
        tsync<NTHR>();
        const int D = keep;
        // U_chi (M x D, FP64) into the Gram buffer
        cx<double>* U = G;
        auto vec = [&](int c, int r) -> cx<double> {
            if (fp64_vectors) return Vd[ord[c] * LDK + r];
            return cvt<double>(V32[ord[c] * LDK + r]);
        };
        if (left) {
            team_for_2d<NTHR>(D, M, lane, [&](int c, int r) { U[c * LDK + r] = vec(c, r); });
            tsync<NTHR>();
            if (!fp64_vectors) {
                // FP32 eigenvectors -> orthonormal to FP64 rounding
                team_qr<NTHR>(U, LDK, M, D, taud, red, lane);
                team_form_q<NTHR>(U, LDK, M, D, taud, lane);
            }
        } else {
            // X = theta V_chi (M x D), then U = Q of its FP64 Householder QR
            team_for_2d<NTHR>(D, M, lane, [&](int c, int r) {
                cx<double> acc = czero<double>();
                for (int j = 0; j < N; ++j) cmac(acc, cvt<double>(th[j * LDM + r]), vec(c, j));
                U[c * LDK + r] = acc;
            });
            tsync<NTHR>();
            team_qr<NTHR>(U, LDK, M, D, taud, red, lane);
            team_form_q<NTHR>(U, LDK, M, D, taud, lane);
        }
        // A_k = U (Dl x 2 x D)
        cx<T>* dst = site_ptr(k);
        team_for_2d<NTHR>(M, D, lane, [&](int row, int c) { dst[row * ld + c] = cvt<T>(U[c * LDK + row]); });
        // cur = U^H theta (D x N), FP64 accumulation, then unit Frobenius norm
        double nrm = 0.0;
        team_for_2d<NTHR>(D, N, lane, [&](int i, int c) {
            cx<double> acc = czero<double>();
            for (int r = 0; r < M; ++r) cmac_cj(acc, U[i * LDK + r], cvt<double>(th[c * LDM + r]));
            nrm += norm2(acc);
            V[c * LDK + i] = acc;   // V is free now
        });
        nrm = team_sum<NTHR>(nrm, red, lane);
        tsync<NTHR>();
        const double inv = nrm > 0.0 ? 1.0 / sqrt(nrm) : 0.0;
        team_for_2d<NTHR>(D, N, lane, [&](int i, int c) {
            const int t = c >= Dr ? 1 : 0, r = c - t * Dr;
            cur[(2 * i + t) * CS + r] = cvt<T>(inv * V[c * LDK + i]);
        });
        tsync<NTHR>();
        return D;
    }

    // Exact centre move one site right: cur (Dl x 2 x Dm) = Q R, site k = Q,
    // cur <- R * nxt.  Returns the new bond min(2 Dl, Dm).
    __device__ int move_right(int k, int Dl, int Dm, int Dr) {
        const int M = 2 * Dl, N = Dm;
        if (lane == 0) *czp = NOZ;
        team_for_2d<NTHR>(M, N, lane, [&](int row, int c) { th[c * LDM + row] = cvt<TQ>(cur[row * CS + c]); });
        tsync<NTHR>();
        team_qr<NTHR>(th, LDM, M, N, tau, red, lane);
        const int Kd = M < N ? M : N;
        team_for_2d<NTHR>(Kd, N, lane, [&](int i, int c) { rb[i * CS + c] = cvt<T>(i <= c ? th[c * LDM + i] : czero<TQ>()); });
        tsync<NTHR>();
        team_form_q<NTHR>(th, LDM, M, Kd, tau, lane);
        cx<T>* dst = site_ptr(k);
        team_for_2d<NTHR>(M, Kd, lane, [&](int row, int c) { dst[row * ld + c] = cvt<T>(th[c * LDM + row]); });
        // cur(i, t, r) = sum_m R(i, m) nxt(m, t, r)
        team_for_2d<NTHR>(Kd, 2 * Dr, lane, [&](int i, int tr) {
            const int t = tr >= Dr ? 1 : 0, r = tr - t * Dr;
            cx<T> acc = czero<T>();
            for (int m = i; m < N; ++m) cmac(acc, rb[i * CS + m], nxt[(2 * m + t) * CS + r]);
            cur[(2 * i + t) * CS + r] = acc;
        });
        tsync<NTHR>();
        return Kd;
    }

    // Exact centre move one site left (LQ): site k (held in cur, Dl x 2 x Dr) = L Q,
    // site k = Q, cur <- site_{k-1} L.  Returns the new bond min(Dl, 2 Dr).
    __device__ int move_left(int k, int Dlm, int Dl, int Dr) {
        const int M = 2 * Dr, N = Dl;   // A^H is (2 Dr) x Dl
        if (lane == 0) *czp = NOZ;
        team_for_2d<NTHR>(N, M, lane, [&](int l, int sr) {
            const int s = sr >= Dr ? 1 : 0, r = sr - s * Dr;
            th[l * LDM + sr] = conj(cvt<TQ>(cur[(2 * l + s) * CS + r]));
        });
        tsync<NTHR>();
        team_qr<NTHR>(th, LDM, M, N, tau, red, lane);
        const int Kd = M < N ? M : N;
        team_for_2d<NTHR>(Kd, N, lane, [&](int i, int c) {
            rb[i * CS + c] = cvt<T>(i <= c ? th[c * LDM + i] : czero<TQ>());   // R'(i, c)
        });
        tsync<NTHR>();
        team_form_q<NTHR>(th, LDM, M, Kd, tau, lane);
        // site k = Q'^H : (Kd x 2 x Dr), element (m, s, r) = conj(Q'(s*Dr + r, m))
        cx<T>* dst = site_ptr(k);
        team_for_2d<NTHR>(Kd, M, lane, [&](int m, int sr) {
            const int s = sr >= Dr ? 1 : 0, r = sr - s * Dr;
            dst[(2 * m + s) * ld + r] = conj(cvt<T>(th[m * LDM + sr]));
        });
        tsync<NTHR>();
        // cur <- site_{k-1} (Dlm x 2 x Dl) times L = R'^H (Dl x Kd)
        load_site<T, CS, NTHR>(nxt, site_ptr(k - 1), ld, Dlm, Dl, nullptr, lane);
        tsync<NTHR>();
        team_for_2d<NTHR>(2 * Dlm, Kd, lane, [&](int row, int m) {
            cx<T> acc = czero<T>();
            for (int l = m; l < Dl; ++l) cmac_cj(acc, rb[m * CS + l], nxt[row * CS + l]);
            cur[row * CS + m] = acc;
        });
        tsync<NTHR>();
        return Kd;
    }
};

// Largest Schmidt rank after c CNOTs across a cut (operator Schmidt rank 2 each).
__device__ __forceinline__ int rank_bound(int c) { return c >= 30 ? (1 << 30) : (1 << c); }

// Pass description: bonds first..n-2; at bond k a CNOT if (k - first) % stride == 0
// (ladder: stride 1), otherwise an exact centre move.  gates_on_load applies the
// layer's one-qubit gates as the sites are loaded.  fresh: the state is the
// initial product state (its normalised sites are already right-orthonormal).
template <typename T, typename TQ, int CHI, bool TRUNC, int NTHR>
__device__ bool run_pass(CircuitTeam<T, TQ, CHI, TRUNC, NTHR>& w, int first, int stride, int ansatz,
                         const cx<T>* gates, int gn, int img, int layer, bool gates_on_load, bool fresh) {
    constexpr int CS = CircuitTeam<T, TQ, CHI, TRUNC, NTHR>::CS;
    const int n = w.n, lane = w.lane;
    int* bd = w.bd;
    // does any step of this pass truncate lossily (keep chi < min(M, N) with chi
    // below the rank bound 2^c of its cut)?  Bond dimensions only; thread 0.
    int* cn = w.cn;
    if (lane == 0) {
        int trunc = 0;
        int dl = bd[first];
        for (int k = first; k < n - 1; ++k) {
            if ((k - first) % stride == 0) {
                const int m = 2 * dl, nn = 2 * bd[k + 2];
                const int mn = m < nn ? m : nn;
                const int rb = rank_bound(cn[k + 1] + 1);
                if (mn > w.chi && rb > w.chi) trunc = 1;
                const int cap = rb < w.chi ? rb : w.chi;
                dl = mn < cap ? mn : cap;
            } else {
                const int m = 2 * dl;
                dl = m < bd[k + 1] ? m : bd[k + 1];
            }
        }
        *w.flag = trunc;
    }
    tsync<NTHR>();
    const int trunc = *w.flag;
    tsync<NTHR>();
    if (trunc && TRUNC && !fresh) {
        // right-to-left LQ sweep: centre from n-1 (held in cur) to `first`
        for (int k = n - 1; k > first; --k) {
            const int nb = w.move_left(k, bd[k - 1], bd[k], bd[k + 1]);
            if (lane == 0) bd[k] = nb;
            tsync<NTHR>();
        }
    } else {
        // the centre stays where it is; the pass starts from the stored site `first`
        load_site<T, CS, NTHR>(w.cur, w.site_ptr(first), w.ld, bd[first], bd[first + 1], nullptr, lane);
        if (lane == 0) *w.czp = CircuitTeam<T, TQ, CHI, TRUNC, NTHR>::NOZ;
        tsync<NTHR>();
    }
    if (gates_on_load) {
        const Gate1<T> g = table_gate<T>(gates, gn, ansatz, layer, img, first);
        apply_gate_smem<T, CS, NTHR>(w.cur, bd[first], bd[first + 1], g, lane);
        tsync<NTHR>();
    }
    for (int k = first; k < n - 1; ++k) {
        const int Dl = bd[k], Dm = bd[k + 1], Dr = bd[k + 2];
        if (gates_on_load) {
            const Gate1<T> g = table_gate<T>(gates, gn, ansatz, layer, img, k + 1);
            load_site<T, CS, NTHR>(w.nxt, w.site_ptr(k + 1), w.ld, Dm, Dr, &g, lane);
        } else {
            load_site<T, CS, NTHR>(w.nxt, w.site_ptr(k + 1), w.ld, Dm, Dr, nullptr, lane);
        }
        tsync<NTHR>();
        int nb;
        if ((k - first) % stride == 0) {
            const int c = cn[k + 1] + 1;
            const int rb = rank_bound(c);
            const int cap = rb < w.chi ? rb : w.chi;
            w.form_theta(Dl, Dm, Dr, true, 2 * Dr <= cap);
            nb = w.split(k, Dl, Dr, cap, rb <= w.chi);
            if (lane == 0) cn[k + 1] = c;
        } else {
            nb = w.move_right(k, Dl, Dm, Dr);
        }
        if (nb > CHI || nb > w.ld) {  // never expected: the host sizes CHI and ld from a dry run
            raise_status(w.status, DEV_BOND_OVERFLOW);
            return false;
        }
        if (lane == 0) bd[k + 1] = nb;
        tsync<NTHR>();
    }
    store_site<T, CS, NTHR>(w.site_ptr(n - 1), w.cur, w.ld, bd[n - 1], bd[n], lane);
    tsync<NTHR>();
    return true;
}

// Persistent kernel: every team of NTHR threads takes images from a work queue
// (an atomic counter over `order`, which the host sorts by descending cost so that
// the longest chains start first) until the queue is empty.  NTHR = 32: a CTA holds
// blockDim/32 independent teams (no block barriers); NTHR > 32: a CTA is one team.
// `queue` must be zero at launch.
template <typename T, typename TQ, int CHI, bool TRUNC, int NTHR>
__global__ void __launch_bounds__(NTHR == 32 ? 256 : NTHR, NTHR == 32 ? 1 : 1024 / NTHR / 2) circuit_kernel(
    const ImageMeta* __restrict__ meta, int n_images, const int32_t* __restrict__ order, int* queue,
    const double* __restrict__ pixels, const cx<T>* __restrict__ gates, int gn, int ansatz,
    cx<T>* __restrict__ arena, int32_t* __restrict__ bonds_out,
    double* __restrict__ discarded_out, int* status, unsigned char* __restrict__ gws) {
    using Lay = CircuitLayout<T, TQ, CHI, TRUNC>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int team = threadIdx.x / NTHR, lane = threadIdx.x % NTHR;
    // per-team workspace: shared memory, or (gws != NULL: bonds above 32, whose
    // workspace exceeds a block's shared memory) a slice of global memory that the host
    // sized as gridDim.x * blockDim.x / NTHR teams
    unsigned char* base = (gws ? gws + (size_t)blockIdx.x * (blockDim.x / NTHR) * Lay::bytes : smem_raw)
                          + (size_t)team * Lay::bytes;
    CircuitTeam<T, TQ, CHI, TRUNC, NTHR> w;
    w.cur = reinterpret_cast<cx<T>*>(base + Lay::off_cur);
    w.nxt = reinterpret_cast<cx<T>*>(base + Lay::off_nxt);
    w.rb = reinterpret_cast<cx<T>*>(base + Lay::off_rb);
    w.th = reinterpret_cast<cx<TQ>*>(base + Lay::off_th);
    w.tau = reinterpret_cast<cx<TQ>*>(base + Lay::off_tau);
    w.bd = reinterpret_cast<int*>(base + Lay::off_bd);
    w.cn = reinterpret_cast<int*>(base + Lay::off_cn);
    w.perm = reinterpret_cast<int*>(base + Lay::off_perm);
    w.cnorm = reinterpret_cast<TQ*>(base + Lay::off_cnorm);
    w.czp = reinterpret_cast<int*>(base + Lay::off_cz);
    w.zr = 0;
    w.G = reinterpret_cast<cx<double>*>(base + Lay::off_gram);
    w.V = reinterpret_cast<cx<double>*>(base + Lay::off_vec);
    w.W = Lay::REFINE ? reinterpret_cast<cx<double>*>(base + Lay::off_w) : nullptr;
    w.taud = reinterpret_cast<cx<double>*>(base + Lay::off_taud);
    w.lam = reinterpret_cast<double*>(base + Lay::off_lam);
    w.ord = reinterpret_cast<int*>(base + Lay::off_ord);
    w.red = reinterpret_cast<double*>(base + Lay::off_red);
    w.flag = reinterpret_cast<int*>(base + Lay::off_flag);
    w.lane = lane;
    w.status = status;

    for (;;) {
        if (lane == 0) *w.flag = atomicAdd(queue, 1);
        tsync<NTHR>();
        const int slot = *w.flag;
        tsync<NTHR>();
        if (slot >= n_images) return;
        const int img = order ? order[slot] : slot;
        const ImageMeta mt = meta[img];
        w.n = mt.n;
        w.chi = mt.chi < CHI ? mt.chi : CHI;
        w.ld = mt.ld;
        w.sites = arena + mt.site_off;
        w.block_trunc = (mt.flags & META_FULL_EIGH) == 0;
        w.discarded = 0.0;
        const double* px = pixels + mt.pixel_off;
        const int n = mt.n;

        // |0...0> then the encoding R_Y(pi x) (ladder); every bond is 1
        for (int k = lane; k <= n; k += NTHR) { w.bd[k] = 1; w.cn[k] = 0; }
        for (int k = lane; k < n; k += NTHR) {
            cx<T>* s = w.site_ptr(k);
            T sn = T(0), cs = T(1);
            if (ansatz == 0) encode_amplitudes(px[k], &sn, &cs);
            s[0] = mk<T>(cs, T(0));
            s[w.ld] = mk<T>(sn, T(0));
        }
        tsync<NTHR>();
        bool ok = true;
        for (int layer = 0; ok && layer < mt.L; ++layer) {
            if (ansatz == 0) {
                ok = run_pass<T, TQ, CHI, TRUNC, NTHR>(w, 0, 1, ansatz, gates, gn, img, layer, true, layer == 0);
            } else {
                ok = run_pass<T, TQ, CHI, TRUNC, NTHR>(w, 0, 2, ansatz, gates, gn, img, layer, true, layer == 0);
                if (ok && n > 2)
                    ok = run_pass<T, TQ, CHI, TRUNC, NTHR>(w, 1, 2, ansatz, gates, gn, img, layer, false, false);
            }
        }
        // A pass ends with the centre at n-1.  The paper ansatz's second pass leaves
        // site 0 as written by the first pass (left-orthonormal), so the whole chain is
        // left-canonical either way.
        for (int k = lane; k <= n; k += NTHR) bonds_out[mt.bond_off + k] = w.bd[k];
        if (lane == 0) discarded_out[img] = w.discarded;
        tsync<NTHR>();
    }
}


// ---------------------------------------------------------------------------
// Layer-pipelined circuit kernel: ladder ansatz, no step truncates, L <= 4.
//
// One CTA per image and one warp per layer.  Layer j's step at bond k runs in
// super-step t = k + 2j, so it starts once layer j-1 has finished its steps at
// bonds k and k+1: sites k and k+1 then hold exactly what the sequential sweep
// would hand to layer j, and the gates still pending in layer j-1 (bonds >= k+2)
// act on other qubits.  Every split of a pass without truncation is exact (QR or
// identity), so no step needs the orthogonality centre; each step also runs the
// same arithmetic as in circuit_kernel, so the two kernels give the same state.
// A CTA barrier ends every super-step (no spin waits).
//
// After layer l of a ladder every bond is at most 2^l (one CNOT crosses each cut
// per layer), so layer l's buffers are sized for a left bond <= CL = min(2^l, CHI)
// and middle/right bonds <= CLR = min(2^(l-1), CHI); a step whose bonds exceed
// them raises DEV_BOND_OVERFLOW before touching the buffers.
constexpr int WAVE_LAYERS = 4;

template <typename T, typename TQ, int CL, int CLR>
struct WaveBuf {
    static constexpr int CS = CL + 1, LDM = 2 * CL + 1;
    static constexpr size_t off_cur = 0;
    static constexpr size_t off_nxt = off_cur + sizeof(cx<T>) * 2 * CL * CS;
    // two theta / reflector buffers and two tau buffers (alternating super-steps), and
    // per buffer a record (k, M, N, Q pending)
    static constexpr size_t TH_BYTES = (sizeof(cx<TQ>) * 2 * CLR * LDM + 15) & ~size_t(15);
    static constexpr size_t TAU_BYTES = (sizeof(cx<TQ>) * 2 * CLR + 15) & ~size_t(15);
    static constexpr size_t off_th = (off_nxt + sizeof(cx<T>) * 2 * CLR * CS + 15) & ~size_t(15);
    static constexpr size_t off_tau = off_th + 2 * TH_BYTES;
    static constexpr size_t off_rec = off_tau + 2 * TAU_BYTES;   // 2 x (k, M, N, pending, zr, Dl), then cz
    static constexpr size_t bytes = (off_rec + 13 * sizeof(int) + 15) & ~size_t(15);   // next layer 16-aligned
};

template <int CHI, int J> struct WaveDims;
template <typename T, typename TQ, int CL, int CLR>
constexpr bool wave_buf_aligned() {
    return WaveBuf<T, TQ, CL, CLR>::bytes % 16 == 0 && WaveBuf<T, TQ, CL, CLR>::off_th % 16 == 0 &&
           WaveBuf<T, TQ, CL, CLR>::off_tau % 16 == 0 && WaveBuf<T, TQ, CL, CLR>::off_nxt % 16 == 0;
}

// Layers 0..2 share one buffer shape, sized for layer 2, so that one compiled step
// (one call site) serves all three and the kernel's code stays small for the
// instruction cache; loops run to the actual bonds, so the arithmetic is the same.
template <int CHI, int J> struct WaveDims {
    static constexpr int JJ = J < 2 ? 2 : J;
    static constexpr int CL = (2 << JJ) < CHI ? (2 << JJ) : CHI;
    static constexpr int CLR = (1 << JJ) < CHI ? (1 << JJ) : CHI;
};

template <typename T, typename TQ, int CHI>
struct WaveLayout {
    static constexpr size_t off_bd = 0;                                  // MAX_QUBITS + 1 bonds
    static constexpr size_t off_w0 = (sizeof(int) * (MAX_QUBITS + 1) + 15) & ~size_t(15);
    static constexpr size_t b0 = WaveBuf<T, TQ, WaveDims<CHI, 0>::CL, WaveDims<CHI, 0>::CLR>::bytes;
    static constexpr size_t b1 = WaveBuf<T, TQ, WaveDims<CHI, 1>::CL, WaveDims<CHI, 1>::CLR>::bytes;
    static constexpr size_t b2 = WaveBuf<T, TQ, WaveDims<CHI, 2>::CL, WaveDims<CHI, 2>::CLR>::bytes;
    static constexpr size_t b3 = WaveBuf<T, TQ, WaveDims<CHI, 3>::CL, WaveDims<CHI, 3>::CLR>::bytes;
    static constexpr size_t off_w1 = off_w0 + b0, off_w2 = off_w1 + b1, off_w3 = off_w2 + b2;
    static_assert(b0 == b1 && b1 == b2, "layers 0..2 share one buffer shape (buffer j at off_w0 + j * b0)");
    static constexpr size_t bytes = off_w3 + b3;
    static_assert(off_w0 % 16 == 0 && off_w1 % 16 == 0 && off_w2 % 16 == 0 && off_w3 % 16 == 0,
                  "layer buffers must stay 16-byte aligned");
};

// One step (bond k) of layer `layer` for the warp that owns it.  Returns false
// (after raising the status) when a bond exceeds the layer's buffers.
template <typename T, typename TQ, int CL, int CLR>
__device__ bool wave_step(unsigned char* buf, int t, int* bd, int k, int n, int ld, cx<T>* sites,
                          const cx<T>* gates, int gn, int layer, bool defer_q, int lane, int* status) {
    using B = WaveBuf<T, TQ, CL, CLR>;
    constexpr int CS = B::CS;
    CircuitTeam<T, TQ, CL, false, 32> w;
    w.cur = reinterpret_cast<cx<T>*>(buf + B::off_cur);
    w.nxt = reinterpret_cast<cx<T>*>(buf + B::off_nxt);
    w.th = reinterpret_cast<cx<TQ>*>(buf + B::off_th + (t & 1) * B::TH_BYTES);
    w.tau = reinterpret_cast<cx<TQ>*>(buf + B::off_tau + (t & 1) * B::TAU_BYTES);
    int* rec = reinterpret_cast<int*>(buf + B::off_rec) + 6 * (t & 1);
    w.rb = nullptr; w.G = nullptr; w.V = nullptr; w.W = nullptr; w.taud = nullptr; w.lam = nullptr; w.ord = nullptr;
    w.red = nullptr; w.flag = nullptr;
    w.bd = bd;
    w.cn = nullptr;
    w.perm = nullptr;
    w.cnorm = nullptr;
    w.czp = reinterpret_cast<int*>(buf + B::off_rec) + 12;
    w.zr = 0;
    w.lane = lane;
    w.n = n;
    w.chi = CL;
    w.ld = ld;
    w.sites = sites;
    w.block_trunc = true;
    w.discarded = 0.0;
    w.status = status;
    const int Dl = bd[k], Dm = bd[k + 1], Dr = bd[k + 2];
    const int nb = 2 * Dl < 2 * Dr ? 2 * Dl : 2 * Dr;
    if (Dl > CL || Dm > CLR || Dr > CLR || nb > CL || nb > ld) {
        raise_status(status, DEV_BOND_OVERFLOW);
        return false;
    }
    if (k == 0) {
        // the pass starts from the stored site 0 with the layer's one-qubit gate
        if (lane == 0) *w.czp = CircuitTeam<T, TQ, CL, false, 32>::NOZ;
        load_site<T, CS, 32>(w.cur, w.site_ptr(0), ld, Dl, Dm, nullptr, lane);
        __syncwarp();
        const Gate1<T> g = table_gate<T>(gates, gn, 0, layer, 0, 0);
        apply_gate_smem<T, CS, 32>(w.cur, Dl, Dm, g, lane);
        __syncwarp();
    }
    const Gate1<T> g = table_gate<T>(gates, gn, 0, layer, 0, k + 1);
    load_site<T, CS, 32>(w.nxt, w.site_ptr(k + 1), ld, Dm, Dr, &g, lane);
    __syncwarp();
    w.form_theta(Dl, Dm, Dr, true, true);
    if (defer_q && 2 * Dr <= 2 * Dl) {
        // QR only; warp 0 forms this site's Q from the reflectors next super-step
        w.qr_to_cur(Dl + w.zr, 2 * Dr, Dr);
        if (lane == 0) {
            *w.czp = Dr;
            rec[0] = k; rec[1] = Dl + w.zr; rec[2] = 2 * Dr; rec[3] = 1; rec[4] = w.zr; rec[5] = Dl;
        }
    } else {
        w.split_exact(k, Dl, Dr);   // no ladder step exceeds its rank bound
    }
    if (k == n - 2) {
        store_site<T, CS, 32>(w.site_ptr(n - 1), w.cur, ld, nb, Dr, lane);
    }
    __syncwarp();
    if (lane == 0) bd[k + 1] = nb;
    return true;
}

// The Q factor a layer's warp left pending in reflector buffer `slot` (see
// wave_step), formed and stored by warp 0.
template <typename T, typename TQ, int CL, int CLR>
__device__ void wave_deferred_q(unsigned char* buf, int slot, int ld, cx<T>* sites, int lane) {
    using B = WaveBuf<T, TQ, CL, CLR>;
    int* rec = reinterpret_cast<int*>(buf + B::off_rec) + 6 * slot;
    if (!rec[3]) return;
    CircuitTeam<T, TQ, CL, false, 32> w;
    w.th = reinterpret_cast<cx<TQ>*>(buf + B::off_th + slot * B::TH_BYTES);
    w.tau = reinterpret_cast<cx<TQ>*>(buf + B::off_tau + slot * B::TAU_BYTES);
    w.lane = lane;
    w.ld = ld;
    w.sites = sites;
    w.q_to_site(rec[0], rec[1], rec[2], rec[5], rec[4]);
    if (lane == 0) rec[3] = 0;
}

template <typename T, typename TQ, int CHI>
__global__ void __launch_bounds__(32 * WAVE_LAYERS, 8) circuit_wave_kernel(
    const ImageMeta* __restrict__ meta, int n_images, const int32_t* __restrict__ order,
    const double* __restrict__ pixels, const cx<T>* __restrict__ gates, int gn,
    cx<T>* __restrict__ arena, int32_t* __restrict__ bonds_out, double* __restrict__ discarded_out,
    int* status) {
    using Lay = WaveLayout<T, TQ, CHI>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int slot = blockIdx.x;
    if (slot >= n_images) return;
    const int img = order ? order[slot] : slot;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const ImageMeta mt = meta[img];
    const int n = mt.n, ld = mt.ld;
    cx<T>* sites = arena + mt.site_off;
    int* bd = reinterpret_cast<int*>(smem_raw + Lay::off_bd);
    const double* px = pixels + mt.pixel_off;
    // |0...0> then the encoding R_Y(pi x); every bond is 1
    for (int k = threadIdx.x; k <= n; k += blockDim.x) bd[k] = 1;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        cx<T>* s = sites + (size_t)k * (2 * ld * ld);
        T sn, cs;
        encode_amplitudes(px[k], &sn, &cs);
        s[0] = mk<T>(cs, T(0));
        s[ld] = mk<T>(sn, T(0));
    }
    const int L = mt.L < WAVE_LAYERS ? mt.L : WAVE_LAYERS;
    const int last = L - 1;
    // the last layer's sites feed no later layer: its Q factors are formed by warp 0
    // (the cheapest layer) one super-step later, off the last layer's critical path
    const bool defer = L >= 2;
    if (threadIdx.x < 13) {
        reinterpret_cast<int*>(smem_raw + Lay::off_w0 + WaveBuf<T, TQ, WaveDims<CHI, 0>::CL, WaveDims<CHI, 0>::CLR>::off_rec)[threadIdx.x] = 0;
        reinterpret_cast<int*>(smem_raw + Lay::off_w1 + WaveBuf<T, TQ, WaveDims<CHI, 1>::CL, WaveDims<CHI, 1>::CLR>::off_rec)[threadIdx.x] = 0;
        reinterpret_cast<int*>(smem_raw + Lay::off_w2 + WaveBuf<T, TQ, WaveDims<CHI, 2>::CL, WaveDims<CHI, 2>::CLR>::off_rec)[threadIdx.x] = 0;
        reinterpret_cast<int*>(smem_raw + Lay::off_w3 + WaveBuf<T, TQ, WaveDims<CHI, 3>::CL, WaveDims<CHI, 3>::CLR>::off_rec)[threadIdx.x] = 0;
    }
    __syncthreads();
    const int supersteps = (L > 0 && n > 1) ? (n - 1) + 2 * (L - 1) + (defer ? 1 : 0) : 0;
    for (int t = 0; t < supersteps; ++t) {
        const int k = t - 2 * warp;
        bool ok = true;
        if (warp < L && k >= 0 && k < n - 1) {
            const bool dq = defer && warp == last;
            if (warp < 3)
                ok = wave_step<T, TQ, WaveDims<CHI, 2>::CL, WaveDims<CHI, 2>::CLR>(
                    smem_raw + Lay::off_w0 + warp * Lay::b0, t, bd, k, n, ld, sites, gates, gn, warp, dq, lane, status);
            else
                ok = wave_step<T, TQ, WaveDims<CHI, 3>::CL, WaveDims<CHI, 3>::CLR>(
                    smem_raw + Lay::off_w3, t, bd, k, n, ld, sites, gates, gn, 3, dq, lane, status);
        }
        if (defer && warp == 0 && t >= 1) {
            if (last < 3)
                wave_deferred_q<T, TQ, WaveDims<CHI, 2>::CL, WaveDims<CHI, 2>::CLR>(
                    smem_raw + Lay::off_w0 + last * Lay::b0, (t - 1) & 1, ld, sites, lane);
            else
                wave_deferred_q<T, TQ, WaveDims<CHI, 3>::CL, WaveDims<CHI, 3>::CLR>(
                    smem_raw + Lay::off_w3, (t - 1) & 1, ld, sites, lane);
        }
        // global writes of this super-step become visible to the other warps here
        if (__syncthreads_or(ok ? 0 : 1)) break;
    }
    for (int k = threadIdx.x; k <= n; k += blockDim.x) bonds_out[mt.bond_off + k] = bd[k];
    if (threadIdx.x == 0) discarded_out[img] = 0.0;
}

}  // namespace mpsano
