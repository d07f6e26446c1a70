// Pauli cache without any device allocation: the MPS arena and every other
// piece of working memory live in one fixed-size array in the library's own
// device memory (see mps_pauli_cache_noalloc in include/mpsano.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "batch.h"
#include "common.cuh"
#include "mpsano.h"

using namespace mpsano;

namespace {

constexpr int NA_MAX_IMAGES = 64;
constexpr int NA_MAX_DEVICES = 64;
constexpr size_t NA_ARENA_BYTES = size_t(12) << 20;   // site tensors (complex64)
constexpr size_t NA_RENV_BYTES = size_t(6) << 20;     // right environments
constexpr size_t NA_GATE_BYTES = size_t(512) << 10;   // one-qubit gate table (complex64)
// complex128 state and gate table of a circuit that truncates lossily (the FP64 chain
// of the mixed precision), twice the complex64 sizes
constexpr size_t NA_ARENA64_BYTES = 2 * NA_ARENA_BYTES;
constexpr size_t NA_GATE64_BYTES = 2 * NA_GATE_BYTES;
// per-image workspace of a truncation at bond 32 on a complex128 state (about 270 KB,
// more than a block's shared memory), for up to 64 images
constexpr size_t NA_GWS_BYTES = size_t(18) << 20;

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t OFF_META = 0;
constexpr size_t OFF_UNITS = align256(OFF_META + sizeof(ImageMeta) * NA_MAX_IMAGES);
constexpr size_t OFF_BONDS = align256(OFF_UNITS + sizeof(int32_t) * 2 * NA_MAX_IMAGES * 16);
constexpr size_t OFF_NORMS = align256(OFF_BONDS + sizeof(int32_t) * NA_MAX_IMAGES * 257);
constexpr size_t OFF_DISC = align256(OFF_NORMS + sizeof(double) * NA_MAX_IMAGES);
constexpr size_t OFF_STATUS = align256(OFF_DISC + sizeof(double) * NA_MAX_IMAGES);
constexpr size_t OFF_QUEUE = align256(OFF_STATUS + sizeof(int));
constexpr size_t OFF_ARENA = align256(OFF_QUEUE + sizeof(int));
constexpr size_t OFF_RENV = align256(OFF_ARENA + NA_ARENA_BYTES);
constexpr size_t OFF_GATES = align256(OFF_RENV + NA_RENV_BYTES);
constexpr size_t OFF_ARENA64 = align256(OFF_GATES + NA_GATE_BYTES);
constexpr size_t OFF_GATES64 = align256(OFF_ARENA64 + NA_ARENA64_BYTES);
constexpr size_t OFF_GWS = align256(OFF_GATES64 + NA_GATE64_BYTES);
constexpr size_t NA_TOTAL = align256(OFF_GWS + NA_GWS_BYTES);

}  // namespace

// The scratch array.  Every GPU that loads this library holds it (about 62 MiB)
// until the process exits.  Host code must not use its name as an address: the
// device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_TOTAL];

namespace {

std::mutex g_na_mutex;
void* g_na_ptr[NA_MAX_DEVICES] = {};

// Device address of the scratch array on the current device (looked up once per
// device, with that device current).
mps_status scratch_address(unsigned char** out) {
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NA_MAX_DEVICES) return fail(MPS_ERR_UNSUPPORTED, "device %d beyond %d", dev, NA_MAX_DEVICES);
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_na_ptr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_na_ptr[dev]);
    return MPS_OK;
}

// Writes the per-image records and Pauli work units, clears the per-call state.
__global__ void noalloc_setup_kernel(ImageMeta* meta, int32_t* units, double* discarded, int* status,
                                     int n_images, int p, int chi, int L, int ld) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = p * p;
    if (t < n_images) {
        ImageMeta m;
        m.p = p; m.n = n; m.chi = chi; m.L = L; m.ld = ld;
        m.bond_off = t * (n + 1);
        m.site_off = (int64_t)t * n * 2 * ld * ld;
        m.pixel_off = (int64_t)t * n;
        m.pair_off = (int64_t)t * 2 * p * (p - 1);
        m.pair_off_d = (int64_t)t * (2 * p * (p - 1) + 2 * (p - 1) * (p - 1));
        m.flags = 0;
        m.pad = 0;
        meta[t] = m;
        discarded[t] = 0.0;
    }
    if (t < n_images * p) {
        units[2 * t] = t / p;
        units[2 * t + 1] = t % p;
    }
    if (t == 0) *status = 0;
}

// The device status word of the call (first device-side error, 0 if none) into the
// caller's int.
__global__ void noalloc_status_kernel(const int* __restrict__ status, int32_t* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *out = *status;
}

}  // namespace

extern "C" mps_status mps_pauli_cache_noalloc(int32_t n_images, int32_t p, int32_t chi, int32_t L,
                                              const double* pixels, const double* params, int32_t params_n,
                                              float* out, int32_t* status, void* stream) {
    if (n_images < 1 || n_images > NA_MAX_IMAGES)
        return fail(MPS_ERR_INVALID_ARG, "n_images = %d outside 1..%d for the no-allocation entry point",
                    n_images, NA_MAX_IMAGES);
    if (p < 2 || p > 16) return fail(MPS_ERR_INVALID_ARG, "p = %d outside 2..16", p);
    if (chi < 1 || chi > 32) return fail(MPS_ERR_INVALID_ARG, "chi = %d outside 1..32", chi);
    if (L < 0 || L > 64) return fail(MPS_ERR_INVALID_ARG, "L = %d outside 0..64", L);
    if (!pixels || !out) return fail(MPS_ERR_INVALID_ARG, "pixels and out must be non-NULL");
    const int n = p * p;
    if (L > 0 && (!params || params_n < n))
        return fail(MPS_ERR_INVALID_ARG, "params must be non-NULL with params_n >= %d", n);
    // bond dimensions from the library's one host mirror of the circuit kernels' rules;
    // the kernels check every bond they write against the padding ld and report a
    // violation through the status word
    bool trunc = false;
    const int mx = dry_run_bonds(n, L, chi, MPS_ANSATZ_LADDER, &trunc);
    const int chi_tpl = chi_bucket(mx);
    if (chi_tpl < 0) return fail(MPS_ERR_UNSUPPORTED, "bond dimension %d > 32", mx);
    int ld = 4;
    while (ld < mx) ld <<= 1;
    const size_t arena = (size_t)n_images * n * 2 * ld * ld * sizeof(cx<float>);
    const size_t renv = (size_t)n_images * n * ld * ld * sizeof(cx<float>);
    const size_t gate_bytes = (size_t)(L > 0 ? L : 1) * n * 4 * sizeof(cx<float>);
    if (gate_bytes > NA_GATE_BYTES)
        return fail(MPS_ERR_INVALID_ARG, "L * p^2 = %d gate-table entries exceed the limit of %zu in the "
                    "no-allocation entry point", L * n, NA_GATE_BYTES / (4 * sizeof(cx<float>)));
    if (arena > NA_ARENA_BYTES || renv > NA_RENV_BYTES)
        return fail(MPS_ERR_INVALID_ARG,
                    "%d images of %dx%d at bond %d need %zu B of site storage (limit %zu) and %zu B of "
                    "environments (limit %zu) in the no-allocation entry point",
                    n_images, p, p, ld, arena, NA_ARENA_BYTES, renv, NA_RENV_BYTES);
    unsigned char* base = nullptr;
    mps_status st = scratch_address(&base);
    if (st != MPS_OK) return st;

    mps_batch b;   // describes the static scratch; its host vectors stay empty
    b.B = n_images;
    b.prec = MPS_MIXED;
    b.stream = reinterpret_cast<cudaStream_t>(stream);
    b.ld_max = ld;
    b.n_max = n;
    b.elem = sizeof(cx<float>);
    b.meta_d = reinterpret_cast<ImageMeta*>(base + OFF_META);
    b.units_d = reinterpret_cast<int32_t*>(base + OFF_UNITS);
    b.n_units = n_images * p;
    b.arena = base + OFF_ARENA;
    b.renv = base + OFF_RENV;
    b.renv_stride = (int64_t)n * ld * ld;
    b.norms = base + OFF_NORMS;
    b.bonds_d = reinterpret_cast<int32_t*>(base + OFF_BONDS);
    b.discarded_d = reinterpret_cast<double*>(base + OFF_DISC);
    b.status_d = reinterpret_cast<int*>(base + OFF_STATUS);
    b.gates = base + OFF_GATES;
    b.gates_bytes = NA_GATE_BYTES;
    b.gates_owned = false;
    b.gate_n = n;
    b.queue_d = reinterpret_cast<int*>(base + OFF_QUEUE);
    b.gws = base + OFF_GWS;   // global-memory workspace of the bond-32 complex128 chain
    b.cap_gws = NA_GWS_BYTES;
    b.gws_fixed = true;
    b.order_d = nullptr;   // equal sizes: images in index order
    b.run_order = nullptr;
    b.run_count = n_images;
    b.use_wave = false;
    b.pauli_sweep = MPS_PAULI_COLUMN;   // the column walk: its environments fit the scratch as laid out

    const int threads = 128;
    const int work = std::max(n_images * p, n_images);
    noalloc_setup_kernel<<<(work + threads - 1) / threads, threads, 0, b.stream>>>(
        b.meta_d, b.units_d, b.discarded_d, b.status_d, n_images, p, chi, L, ld);
    CUDA_TRY(cudaGetLastError());
    count_launch();
    if (trunc) {
        // lossy truncation: the circuit runs on a complex128 state (the mixed
        // precision's FP64 chain) in the scratch's FP64 region, then its sites are
        // rounded into the complex64 arena for the environment and Pauli kernels
        b.gates = base + OFF_GATES64;
        b.gates_bytes = NA_GATE64_BYTES;
        b.arena = base + OFF_ARENA64;
        st = launch_gate_table(&b, MPS_ANSATZ_LADDER, L, params, params_n, pixels, true, b.gates);
        if (st != MPS_OK) return st;
        st = launch_circuit_fp64(&b, chi_tpl, true, pixels, MPS_ANSATZ_LADDER);
        if (st != MPS_OK) return st;
        b.arena = base + OFF_ARENA;
        st = launch_round_sites(&b, base + OFF_ARENA64);
        if (st != MPS_OK) return st;
    } else {
        st = launch_gate_table(&b, MPS_ANSATZ_LADDER, L, params, params_n, pixels, false, b.gates);
        if (st != MPS_OK) return st;
        st = launch_circuit_mixed(&b, chi_tpl, false, pixels, MPS_ANSATZ_LADDER);
        if (st != MPS_OK) return st;
    }
    b.chi_tpl = chi_tpl;
    st = launch_pauli_mixed(&b, out);
    if (st != MPS_OK || !status) return st;
    noalloc_status_kernel<<<1, 32, 0, b.stream>>>(b.status_d, status);
    CUDA_TRY(cudaGetLastError());
    count_launch();
    return MPS_OK;
}
