// Host-side batch handle shared by the translation units of the library.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "common.cuh"
#include "mpsano.h"

struct mps_batch {
    int B = 0;
    int prec = MPS_MIXED;
    cudaStream_t stream = nullptr;
    int ld_max = 1;
    int n_max = 0;
    size_t elem = 8;                       // bytes per complex element of the state
    std::vector<mpsano::ImageMeta> meta_h;
    std::vector<int32_t> p_h, chi_h;       // the layout's image sides and bond caps
    std::vector<int32_t> units_h;          // (image, column) pairs of the Pauli kernel
    int n_units = 0;                       // = units_h.size() / 2 when units_h is used
    mpsano::ImageMeta* meta_d = nullptr;
    mpsano::ImageMeta* meta_pinned = nullptr;
    int32_t* units_d = nullptr;
    void* arena = nullptr;                 // sites
    void* renv = nullptr;                  // right environments
    int64_t renv_stride = 0;               // complex elements per image
    void* lenv = nullptr;                  // left environments (operator-product ladder images), as renv
    size_t cap_lenv = 0;
    bool any_lenv = false;                 // some image of the last circuit is flagged META_LENV
    bool all_half = false;                 // every image of the last circuit is flagged META_HALF
    void* norms = nullptr;
    int32_t* bonds_d = nullptr;
    double* discarded_d = nullptr;
    int* status_d = nullptr;
    int64_t total_pairs_hv = 0, total_pairs_hvd = 0;
    int64_t total_bonds = 0;
    bool circuit_done = false;
    bool layout_ok = false;                // device buffers match the host layout
    bool meta_dirty = false;               // meta_h changed since its last upload
    void* gates = nullptr;                 // one-qubit gate table of the last circuit
    size_t gates_bytes = 0;
    // complex128 state of the images whose circuit truncates lossily under the mixed
    // precisions (their chain runs in FP64 and is rounded into `arena` at its end), and
    // the FP64 gate table that chain reads
    void* arena64 = nullptr;
    size_t cap_arena64 = 0;
    void* gates64 = nullptr;
    size_t gates64_bytes = 0;
    int n_chain64 = 0;                     // images of the last circuit that took the FP64 chain
    // global-memory workspace of the kernels for bonds above 32 (their per-team buffers
    // exceed a block's shared memory)
    void* gws = nullptr;
    size_t cap_gws = 0;
    bool gws_fixed = false;                // gws is caller-provided scratch: never (re)allocate it
    int gate_n = 0;                        // qubit stride of the gate table
    bool gates_owned = true;               // false when gates points into static scratch
    int circuit_threads = 32;              // threads per image in the circuit kernel
    bool layer_pipeline = true;            // layer-pipelined kernel where it applies
    bool half_structure = true;            // exploit half-structured sites (META_HALF)
    bool block_truncation = true;          // FP64 truncations may use the block solve (else META_FULL_EIGH)
    bool real = false;                     // the last circuit's state is real (paper ansatz)
    bool real_allowed = true;              // real-element kernels for real states (mps_set_real_arithmetic)
    int pauli_sweep = MPS_PAULI_AUTO;      // Pauli-cache kernel choice (mps_set_pauli_sweep)
    int L_max = 0;                         // most layers of any image in the last circuit
    // images of the next circuit launch: run_order[0 .. run_count), and whether the
    // layer-pipelined kernel runs them
    const int32_t* run_order = nullptr;
    int run_count = 0;
    bool use_wave = false;
    std::vector<int32_t> cost_order;       // all images by descending cost
    std::vector<int32_t> order_h;          // the order last uploaded to order_d
    int32_t* order_d = nullptr;            // circuit work queue: images by descending cost
    int32_t* order_pinned = nullptr;       // staging of order_d
    int32_t* units_pinned = nullptr;       // staging of units_d
    int64_t need_sites = 0;                // complex elements of site storage of the layout
    // allocated capacities in bytes (buffers grow, never shrink, across re-layouts)
    size_t cap_meta = 0, cap_meta_pinned = 0, cap_units = 0, cap_arena = 0, cap_renv = 0, cap_norms = 0,
           cap_bonds = 0, cap_disc = 0, cap_status = 0, cap_queue = 0, cap_order = 0, cap_order_pinned = 0,
           cap_units_pinned = 0;
    int* queue_d = nullptr;                // circuit work-queue counter
    int chi_tpl = 0;                       // kernel CHI bucket of the last circuit
    int images_per_cta = 2;
    int pauli_warps = 2;
    // optional per-launch event timing (mps_set_timing / mps_kernel_times)
    bool timing = false;
    struct TimedLaunch { int kind; cudaEvent_t start, stop; };
    std::vector<TimedLaunch> timed;
    std::vector<cudaEvent_t> event_pool;
};

namespace mpsano {

// Record a thread-local error message and return st.
mps_status fail(mps_status st, const char* fmt, ...);
// Count one kernel launch (reported by mps_launch_count).
void count_launch();
// Kernel kinds reported by mps_kernel_times.
enum KernelKind { KIND_CIRCUIT = 0, KIND_RENV = 1, KIND_PAULI = 2, KIND_COUNT = 3 };
// Record a start event for a timed launch on the batch stream (no-op unless timing).
void timing_begin(mps_batch* b, int kind);
void timing_end(mps_batch* b);
// Opt-in shared-memory limit per block on the current device.
int smem_optin_limit();
// Y(r, o) = sum_k X(r, k) W(o, k) + bias[o] on the tensor cores (strided operands,
// see linear_tc_kernel); failures of its bounded waits surface through ano_status.
// With partial != NULL and k_split > 1, K is split over linear_tc_splits(K, k_split)
// CTAs per tile whose partial tiles (planes of rows x out_dim floats in `partial`)
// are then summed in a fixed order.
mps_status launch_linear_tc(const float* X, int64_t xs_r, int64_t xs_k, int rows, int K, const float* W,
                            int64_t ws_o, int64_t ws_k, const float* bias, int out_dim, float* Y,
                            cudaStream_t s, int k_split = 1, float* partial = nullptr);
int linear_tc_splits(int K, int k_split);

mps_status launch_circuit_fp64_t0(mps_batch* b, int chi_tpl, const double* px, int ansatz);
mps_status launch_circuit_fp64_t1(mps_batch* b, int chi_tpl, const double* px, int ansatz);
inline mps_status launch_circuit_fp64(mps_batch* b, int chi_tpl, bool trunc, const double* px, int ansatz) {
    return trunc ? launch_circuit_fp64_t1(b, chi_tpl, px, ansatz) : launch_circuit_fp64_t0(b, chi_tpl, px, ansatz);
}
mps_status launch_circuit_mixed_t0(mps_batch* b, int chi_tpl, const double* px, int ansatz);
mps_status launch_circuit_mixed_t1(mps_batch* b, int chi_tpl, const double* px, int ansatz);
inline mps_status launch_circuit_mixed(mps_batch* b, int chi_tpl, bool trunc, const double* px, int ansatz) {
    return trunc ? launch_circuit_mixed_t1(b, chi_tpl, px, ansatz) : launch_circuit_mixed_t0(b, chi_tpl, px, ansatz);
}
mps_status launch_circuit_orth64_t0(mps_batch* b, int chi_tpl, const double* px, int ansatz);
mps_status launch_circuit_orth64_t1(mps_batch* b, int chi_tpl, const double* px, int ansatz);
inline mps_status launch_circuit_orth64(mps_batch* b, int chi_tpl, bool trunc, const double* px, int ansatz) {
    return trunc ? launch_circuit_orth64_t1(b, chi_tpl, px, ansatz) : launch_circuit_orth64_t0(b, chi_tpl, px, ansatz);
}
// Fill `dst` (allocated by the caller; complex128 entries if f64, else complex64) with
// the one-qubit gate table of a circuit.
mps_status launch_gate_table(mps_batch* b, int ansatz, int L_max, const double* params, int params_n,
                             const double* pixels, bool f64, void* dst);
// Host mirror of the circuit kernels' bond rules for one image: returns the largest
// bond; *svd is set when some step truncates lossily (an SVD split to chi below the
// rank bound 2^c of its cut).
int dry_run_bonds(int n, int L, int chi, int ansatz, bool* svd);
// Smallest compiled bond bucket (4, 8, 16, 32, 64, 128) holding bond mx, or -1.
int chi_bucket(int mx);
// Default cap of the site padding (a batch is laid out again for larger bonds).
constexpr int LD_DEFAULT_CAP = 32;
// Kernel route of one image in mps_apply_circuit: operator product, layer-pipelined,
// sequential in the batch's precision, sequential on a complex128 state (a lossy
// truncation under the mixed precisions).
enum Route { ROUTE_MPO = 0, ROUTE_WAVE = 1, ROUTE_SEQ = 2, ROUTE_CHAIN64 = 3 };
struct ImagePlan {
    int route;
    int bond;     // largest bond of the image's MPS (2^L at every inner cut for ROUTE_MPO)
    bool lossy;   // some step keeps fewer singular values than the rank
};
ImagePlan plan_image(int n, int L, int chi, int ld, int ansatz, int prec, bool layer_pipeline);
// Site padding of an image with n qubits and bond cap chi once a circuit needing `bond` ran.
int site_padding(int n, int chi, int bond);
// Rounds the complex128 sites that an FP64 chain wrote to src64 into b->arena
// (complex64, same offsets) for the images b->run_order[0 .. run_count) (run_order
// NULL: images 0 .. run_count-1).
mps_status launch_round_sites(mps_batch* b, const void* src64);
// Circuits as operator products for b->run_order[0 .. run_count) (ladder_mpo.cu).
mps_status launch_ladder_mpo(mps_batch* b, const double* pixels, int ansatz);
mps_status launch_pauli_fp64(mps_batch* b, void* out, bool diag = false);
// Environments and Pauli cache at bond buckets 64 and 128 (workspace in global memory).
mps_status launch_pauli_large(mps_batch* b, void* out, bool diag, bool f64);
// Environments and Pauli cache of a real state (b->real), complex64 storage, bonds <= 32.
mps_status launch_pauli_real(mps_batch* b, void* out, bool diag);
// Global-memory workspace of at least `bytes` for the kernels of bonds above 32.
mps_status ensure_gws(mps_batch* b, size_t bytes);
mps_status launch_pauli_mixed(mps_batch* b, void* out, bool diag = false);
// Left environments and the per-image sweep Pauli kernel (mixed precisions, bonds up
// to 16, per b->pauli_sweep); *taken = false (and nothing launched) where it does not apply.
mps_status launch_pauli_sweep(mps_batch* b, void* out, bool diag, bool* taken);

}  // namespace mpsano

#define CUDA_TRY(expr)                                                                               \
    do {                                                                                             \
        cudaError_t e_ = (expr);                                                                     \
        if (e_ != cudaSuccess)                                                                       \
            return ::mpsano::fail(e_ == cudaErrorMemoryAllocation ? MPS_ERR_OOM : MPS_ERR_CUDA,      \
                                  "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)
