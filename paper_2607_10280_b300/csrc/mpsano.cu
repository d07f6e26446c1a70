// Host side of the C ABI declared in include/mpsano.h: batch handles, metadata,
// launch-shape selection and template dispatch of the kernels.
#include "mpsano.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <climits>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <unordered_map>
#include <string>
#include <vector>

#include "batch.h"
#include "circuit.cuh"
#include "common.cuh"
#include "epilogue.cuh"
#include "gemm_tc.cuh"

using namespace mpsano;

namespace {

thread_local std::string g_err = "no error";
__device__ int g_epilogue_status = 0;   // first failure code of a tensor-core wait
std::atomic<uint64_t> g_launches{0};

}  // namespace

namespace mpsano {

void count_launch() { g_launches.fetch_add(1); }

namespace {
// Y[i] = sum_z P[z][i] (+ bias[i % out_dim]), planes summed in order z = 0, 1, ...
__global__ void sum_planes_kernel(const float* __restrict__ P, int planes, int64_t n, int out_dim,
                                  const float* __restrict__ bias, float* __restrict__ Y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = bias ? bias[i % out_dim] : 0.f;
    for (int z = 0; z < planes; ++z) s += P[(int64_t)z * n + i];
    Y[i] = s;
}
}  // namespace

int linear_tc_splits(int K, int k_split) {
    const int chunks = (K + TC_KC - 1) / TC_KC;
    const int ks = std::max(1, std::min(k_split, chunks));
    const int cps = (chunks + ks - 1) / ks;
    return std::max(1, (chunks + cps - 1) / cps);
}

mps_status launch_linear_tc(const float* X, int64_t xs_r, int64_t xs_k, int rows, int K, const float* W,
                            int64_t ws_o, int64_t ws_k, const float* bias, int out_dim, float* Y,
                            cudaStream_t s, int k_split, float* partial) {
    static int attr_dev = -1;
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (attr_dev != dev) {
        CUDA_TRY(cudaFuncSetAttribute(linear_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)TC_SMEM_BYTES));
        attr_dev = dev;
    }
    int* st = nullptr;
    CUDA_TRY(cudaGetSymbolAddress((void**)&st, g_epilogue_status));
    const int chunks = (K + TC_KC - 1) / TC_KC;
    const int ks = std::max(1, std::min(partial ? k_split : 1, chunks));
    const int cps = (chunks + ks - 1) / ks;          // every plane gets >= 1 chunk
    const int planes = (chunks + cps - 1) / cps;
    dim3 grid((out_dim + TC_N - 1) / TC_N, (unsigned)((rows + TC_M - 1) / TC_M), (unsigned)planes);
    linear_tc_kernel<<<grid, 128, TC_SMEM_BYTES, s>>>(X, xs_r, xs_k, rows, K, W, ws_o, ws_k,
                                                      planes > 1 ? nullptr : bias, out_dim,
                                                      planes > 1 ? partial : Y, std::max(cps, 1), st);
    CUDA_TRY(cudaGetLastError());
    count_launch();
    if (planes > 1) {
        const int64_t n = (int64_t)rows * out_dim;
        sum_planes_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(partial, planes, n, out_dim, bias, Y);
        CUDA_TRY(cudaGetLastError());
        count_launch();
    }
    return MPS_OK;
}

namespace {
cudaEvent_t pooled_event(mps_batch* b) {
    if (!b->event_pool.empty()) {
        cudaEvent_t e = b->event_pool.back();
        b->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}
}  // namespace

void timing_begin(mps_batch* b, int kind) {
    if (!b->timing) return;
    mps_batch::TimedLaunch t{kind, pooled_event(b), pooled_event(b)};
    cudaEventRecord(t.start, b->stream);
    b->timed.push_back(t);
}

mps_status launch_gate_table(mps_batch* b, int ansatz, int L_max, const double* params, int params_n,
                             const double* pixels, bool f64, void* dst) {
    const int rows = ansatz == MPS_ANSATZ_LADDER ? L_max : b->B;
    const int total = rows * b->gate_n;
    if (total <= 0) return MPS_OK;
    const int threads = 128;
    if (f64)
        gate_table_kernel<double><<<(total + threads - 1) / threads, threads, 0, b->stream>>>(
            ansatz, rows, b->gate_n, params, params_n, b->meta_d, pixels, static_cast<cx<double>*>(dst));
    else
        gate_table_kernel<float><<<(total + threads - 1) / threads, threads, 0, b->stream>>>(
            ansatz, rows, b->gate_n, params, params_n, b->meta_d, pixels, static_cast<cx<float>*>(dst));
    CUDA_TRY(cudaGetLastError());
    count_launch();
    return MPS_OK;
}

void timing_end(mps_batch* b) {
    if (!b->timing || b->timed.empty()) return;
    cudaEventRecord(b->timed.back().stop, b->stream);
}

mps_status fail(mps_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}



int smem_optin_limit() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v > 0 ? v : 48 * 1024;
}

// Host mirror of the circuit kernel's bond dimensions (run_pass): returns the largest
// bond; *svd is set when some step truncates lossily (an SVD split to chi below the
// rank bound 2^c of its cut).  Splits that only drop the rank beyond 2^c use the
// pivoted QR, which every circuit kernel has.
int dry_run_bonds(int n, int L, int chi, int ansatz, bool* svd) {
    std::vector<int> bd(n + 1, 1), cn(n + 1, 0);
    int mx = 1;
    bool any = false;
    auto rank_bound = [](int c) { return c >= 30 ? (1 << 30) : (1 << c); };
    auto pass = [&](int first, int stride) {
        bool lossy = false;
        int dl = bd[first];
        for (int k = first; k < n - 1; ++k) {
            if ((k - first) % stride == 0) {
                const int m = 2 * dl, nn = 2 * bd[k + 2];
                const int mn = std::min(m, nn);
                const int rb = rank_bound(cn[k + 1] + 1);
                if (mn > chi && rb > chi) lossy = true;
                dl = std::min(mn, std::min(chi, rb));
            } else {
                dl = std::min(2 * dl, bd[k + 1]);
            }
        }
        if (lossy) {  // centre moves right-to-left (LQ) before the pass
            for (int k = n - 1; k > first; --k) bd[k] = std::min(bd[k], 2 * bd[k + 1]);
        }
        for (int k = first; k < n - 1; ++k) {
            int nb;
            if ((k - first) % stride == 0) {
                const int m = 2 * bd[k], nn = 2 * bd[k + 2];
                const int c = cn[k + 1] + 1;
                const int cap = std::min(chi, rank_bound(c));
                if (std::min(m, nn) > cap && rank_bound(c) > chi) any = true;   // lossy: SVD kernels
                nb = std::min(cap, std::min(m, nn));
                cn[k + 1] = c;
            } else {
                nb = std::min(2 * bd[k], bd[k + 1]);
            }
            bd[k + 1] = nb;
            mx = std::max(mx, nb);
        }
    };
    for (int l = 0; l < L; ++l) {
        if (ansatz == MPS_ANSATZ_LADDER) {
            pass(0, 1);
        } else {
            pass(0, 2);
            if (n > 2) pass(1, 2);
        }
    }
    *svd = any;
    return mx;
}

ImagePlan plan_image(int n, int L, int chi, int ld, int ansatz, int prec, bool layer_pipeline) {
    bool t = false;
    const int bi = dry_run_bonds(n, L, chi, ansatz, &t);
    const bool fast = layer_pipeline && !t && L >= 1 && L <= WAVE_LAYERS;   // nothing truncates
    if (fast && (1 << L) <= std::min(ld, chi) && (1 << L) <= 16) return {ROUTE_MPO, 1 << L, false};
    if (fast && ansatz == MPS_ANSATZ_LADDER) return {ROUTE_WAVE, bi, false};
    if (t && (prec == MPS_MIXED || prec == MPS_MIXED_ORTH64)) return {ROUTE_CHAIN64, bi, true};
    return {ROUTE_SEQ, bi, t};
}

int site_padding(int n, int chi, int bond) {
    int cap = 1;
    while (cap < chi && cap < (1 << std::min(n / 2, 20))) cap <<= 1;
    cap = std::min(std::min(cap, chi), LD_DEFAULT_CAP);
    if (bond > cap && bond <= MPS_BOND_LIMIT) cap = bond;   // laid out again for a larger bond
    int ld = 4;
    while (ld < cap) ld <<= 1;
    return ld;
}

int chi_bucket(int mx) {
    for (int c : {4, 8, 16, 32, 64, 128})
        if (mx <= c) return c;
    return -1;
}

mps_status ensure_gws(mps_batch* b, size_t bytes) {
    if (b->gws && b->cap_gws >= bytes) return MPS_OK;
    if (b->gws_fixed)
        return fail(MPS_ERR_INVALID_ARG, "kernel workspace of %zu B exceeds the fixed scratch of %zu B", bytes,
                    b->cap_gws);
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    cudaFree(b->gws);
    b->gws = nullptr;
    b->cap_gws = 0;
    const cudaError_t e = cudaMalloc(&b->gws, bytes);
    if (e != cudaSuccess) return fail(MPS_ERR_OOM, "kernel workspace of %zu B: %s", bytes, cudaGetErrorString(e));
    b->cap_gws = bytes;
    return MPS_OK;
}

namespace {
// Rounds the complex128 sites of the images order[0 .. count) (order NULL: images
// 0 .. count-1), written by the FP64 chain into src, to complex64 in dst at the same
// offsets, over the bonds the chain wrote.  One CTA per image.
__global__ void round_sites_kernel(const ImageMeta* __restrict__ meta, const int32_t* __restrict__ order, int count,
                                   const int32_t* __restrict__ bonds, const cx<double>* __restrict__ src,
                                   cx<float>* __restrict__ dst) {
    if ((int)blockIdx.x >= count) return;
    const ImageMeta m = meta[order ? order[blockIdx.x] : (int)blockIdx.x];
    const int32_t* bd = bonds + m.bond_off;
    const int ld = m.ld;
    for (int k = 0; k < m.n; ++k) {
        const int Dl = bd[k], Dr = bd[k + 1];
        const size_t off = (size_t)m.site_off + (size_t)k * 2 * ld * ld;
        for (int e = threadIdx.x; e < 2 * Dl * Dr; e += blockDim.x) {
            const int row = e / Dr, r = e - row * Dr;
            const cx<double> v = src[off + (size_t)row * ld + r];
            dst[off + (size_t)row * ld + r] = mk<float>((float)v.re, (float)v.im);
        }
    }
}
}  // namespace

mps_status launch_round_sites(mps_batch* b, const void* src64) {
    if (b->run_count <= 0) return MPS_OK;
    timing_begin(b, KIND_CIRCUIT);
    round_sites_kernel<<<b->run_count, 256, 0, b->stream>>>(b->meta_d, b->run_order, b->run_count, b->bonds_d,
                                                            static_cast<const cx<double>*>(src64),
                                                            static_cast<cx<float>*>(b->arena));
    timing_end(b);
    CUDA_TRY(cudaGetLastError());
    count_launch();
    return MPS_OK;
}

}  // namespace mpsano

namespace {

void free_batch(mps_batch* b) {
    if (!b) return;
    for (auto& t : b->timed) { cudaEventDestroy(t.start); cudaEventDestroy(t.stop); }
    for (auto e : b->event_pool) cudaEventDestroy(e);
    cudaFree(b->meta_d);
    cudaFreeHost(b->meta_pinned);
    cudaFreeHost(b->order_pinned);
    cudaFreeHost(b->units_pinned);
    cudaFree(b->units_d);
    cudaFree(b->arena);
    cudaFree(b->renv);
    cudaFree(b->lenv);
    cudaFree(b->norms);
    cudaFree(b->bonds_d);
    cudaFree(b->discarded_d);
    cudaFree(b->status_d);
    cudaFree(b->queue_d);
    cudaFree(b->order_d);
    cudaFree(b->arena64);
    cudaFree(b->gates64);
    cudaFree(b->gws);
    if (b->gates_owned) cudaFree(b->gates);
    delete b;
}

}  // namespace

extern "C" {

const char* mps_last_error(void) { return g_err.c_str(); }

uint64_t mps_launch_count(void) { return g_launches.load(); }

int64_t mps_pair_count(int32_t p, int32_t pair_set) {
    if (p < 1) return 0;
    int64_t m = 2LL * p * (p - 1);
    if (pair_set == MPS_PAIRS_HVD) m += 2LL * (p - 1) * (p - 1);
    return m;
}

}  // extern "C"

namespace {

// Host-side layout of an image list: per-image records, Pauli work units and sizes.
// Site padding: a power of two >= 4 holding the largest bond the image can reach,
// min(chi, 2^floor(n/2)), by default at most LD_DEFAULT_CAP; ld_min (optional, per
// image) raises it for a circuit that needs a larger bond (up to MPS_BOND_LIMIT).
mps_status layout_images(mps_batch* b, int32_t n_images, const int32_t* p, const int32_t* chi, int32_t chi_all,
                         const int32_t* ld_min = nullptr) {
    if (n_images <= 0) return fail(MPS_ERR_INVALID_ARG, "n_images must be positive, got %d", n_images);
    if (!p) return fail(MPS_ERR_INVALID_ARG, "p is NULL");
    for (int i = 0; i < n_images; ++i) {
        const int ci = chi ? chi[i] : chi_all;
        if (p[i] < 2 || p[i] > 16) return fail(MPS_ERR_INVALID_ARG, "p[%d] = %d outside 2..16", i, p[i]);
        if (ci < 1 || ci > MPS_CHI_LIMIT) return fail(MPS_ERR_INVALID_ARG, "chi[%d] = %d outside 1..%d", i, ci, MPS_CHI_LIMIT);
    }
    if (p != b->p_h.data()) b->p_h.assign(p, p + n_images);
    if (chi) {
        if (chi != b->chi_h.data()) b->chi_h.assign(chi, chi + n_images);
    } else {
        b->chi_h.assign(n_images, chi_all);
    }
    b->B = n_images;
    b->meta_h.assign(n_images, ImageMeta{});
    b->units_h.clear();
    b->ld_max = 1;
    b->n_max = 0;
    int64_t site_off = 0, pix = 0, pair = 0, pair_d = 0, bond = 0;
    for (int i = 0; i < n_images; ++i) {
        const int pi = p[i];
        const int ci = chi ? chi[i] : chi_all;
        const int n = pi * pi;
        // largest bond any circuit can reach: min(chi, 2^floor(n/2)), at most 32 unless
        // a circuit asked for more (ld_min)
        int cap = 1;
        while (cap < ci && cap < (1 << std::min(n / 2, 20))) cap <<= 1;
        cap = std::min(std::min(cap, ci), LD_DEFAULT_CAP);
        if (ld_min) cap = std::max(cap, std::min(ld_min[i], MPS_BOND_LIMIT));
        int ld = 4;
        while (ld < cap) ld <<= 1;
        ImageMeta& m = b->meta_h[i];
        m.p = pi; m.n = n; m.chi = ci; m.L = -1; m.ld = ld;
        m.bond_off = (int32_t)bond;
        m.site_off = site_off;
        m.pixel_off = pix;
        m.pair_off = pair;
        m.pair_off_d = pair_d;
        site_off += (int64_t)n * 2 * ld * ld;
        pix += n;
        pair += mps_pair_count(pi, MPS_PAIRS_HV);
        pair_d += mps_pair_count(pi, MPS_PAIRS_HVD);
        bond += n + 1;
        b->ld_max = std::max(b->ld_max, ld);
        b->n_max = std::max(b->n_max, n);
        for (int c = 0; c < pi; ++c) { b->units_h.push_back(i); b->units_h.push_back(c); }
    }
    b->n_units = (int)(b->units_h.size() / 2);
    b->total_pairs_hv = pair;
    b->total_bonds = bond;
    b->renv_stride = (int64_t)b->n_max * b->ld_max * b->ld_max;  // R_j of any image at any kernel bucket
    b->need_sites = site_off;
    return MPS_OK;
}

template <typename P>
cudaError_t grow(P** ptr, size_t* cap, size_t need, bool pinned = false) {
    if (need <= *cap && *ptr) return cudaSuccess;
    if (pinned) cudaFreeHost(*ptr); else cudaFree(*ptr);
    *ptr = nullptr;
    *cap = 0;
    cudaError_t e = pinned ? cudaMallocHost(reinterpret_cast<void**>(ptr), need)
                           : cudaMalloc(reinterpret_cast<void**>(ptr), need);
    if (e == cudaSuccess) *cap = need;
    return e;
}

// Device buffers at least as large as the current layout needs, then the layout
// uploaded (stream-ordered).
mps_status fit_and_upload(mps_batch* b) {
    const int B = b->B;
#define TRY_GROW(expr)                                                                          \
    do {                                                                                        \
        cudaError_t e_ = (expr);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return fail(e_ == cudaErrorMemoryAllocation ? MPS_ERR_OOM : MPS_ERR_CUDA, "%s: %s", \
                        #expr, cudaGetErrorString(e_));                                         \
    } while (0)
    TRY_GROW(grow(&b->meta_d, &b->cap_meta, sizeof(ImageMeta) * B));
    TRY_GROW(grow(&b->meta_pinned, &b->cap_meta_pinned, sizeof(ImageMeta) * B, true));
    TRY_GROW(grow(&b->units_d, &b->cap_units, sizeof(int32_t) * b->units_h.size()));
    TRY_GROW(grow(reinterpret_cast<unsigned char**>(&b->arena), &b->cap_arena, b->elem * b->need_sites));
    TRY_GROW(grow(reinterpret_cast<unsigned char**>(&b->renv), &b->cap_renv, b->elem * b->renv_stride * B));
    TRY_GROW(grow(reinterpret_cast<unsigned char**>(&b->norms), &b->cap_norms, sizeof(double) * B));
    TRY_GROW(grow(&b->bonds_d, &b->cap_bonds, sizeof(int32_t) * b->total_bonds));
    TRY_GROW(grow(&b->discarded_d, &b->cap_disc, sizeof(double) * B));
    TRY_GROW(grow(&b->status_d, &b->cap_status, sizeof(int)));
    TRY_GROW(grow(&b->queue_d, &b->cap_queue, sizeof(int)));
    TRY_GROW(grow(&b->order_d, &b->cap_order, sizeof(int32_t) * B));
    TRY_GROW(grow(&b->order_pinned, &b->cap_order_pinned, sizeof(int32_t) * B, true));
    TRY_GROW(grow(&b->units_pinned, &b->cap_units_pinned, sizeof(int32_t) * b->units_h.size(), true));
    // work queue: images by descending cost n * ld^3 (largest chains first)
    for (int i = 0; i < B; ++i) b->order_pinned[i] = i;
    std::stable_sort(b->order_pinned, b->order_pinned + B, [&](int a, int c) {
        const ImageMeta& ma = b->meta_h[a];
        const ImageMeta& mc = b->meta_h[c];
        return (int64_t)ma.n * ma.ld * ma.ld * ma.ld > (int64_t)mc.n * mc.ld * mc.ld * mc.ld;
    });
    b->cost_order.assign(b->order_pinned, b->order_pinned + B);
    b->order_h = b->cost_order;
    std::memcpy(b->units_pinned, b->units_h.data(), sizeof(int32_t) * b->units_h.size());
    std::memcpy(b->meta_pinned, b->meta_h.data(), sizeof(ImageMeta) * B);
    TRY_GROW(cudaMemsetAsync(b->status_d, 0, sizeof(int), b->stream));
    TRY_GROW(cudaMemsetAsync(b->discarded_d, 0, sizeof(double) * B, b->stream));
    TRY_GROW(cudaMemcpyAsync(b->order_d, b->order_pinned, sizeof(int32_t) * B, cudaMemcpyHostToDevice, b->stream));
    TRY_GROW(cudaMemcpyAsync(b->units_d, b->units_pinned, sizeof(int32_t) * b->units_h.size(),
                             cudaMemcpyHostToDevice, b->stream));
    TRY_GROW(cudaMemcpyAsync(b->meta_d, b->meta_pinned, sizeof(ImageMeta) * B, cudaMemcpyHostToDevice, b->stream));
#undef TRY_GROW
    b->meta_dirty = false;
    b->layout_ok = true;
    return MPS_OK;
}

// Left environments for every image of the current layout (operator-product images).
mps_status ensure_lenv(mps_batch* b) {
    const size_t need = b->elem * b->renv_stride * b->B;
    if (b->cap_lenv >= need && b->lenv) return MPS_OK;
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    cudaFree(b->lenv);
    b->lenv = nullptr;
    b->cap_lenv = 0;
    const cudaError_t e = cudaMalloc(&b->lenv, need);
    if (e != cudaSuccess) return fail(MPS_ERR_OOM, "left environments: %s", cudaGetErrorString(e));
    b->cap_lenv = need;
    return MPS_OK;
}

// Gate table for `rows` rows (layers of the ladder, images of the paper ansatz) and,
// with chain64, the FP64 chain's complex128 arena and gate table.
mps_status ensure_gates(mps_batch* b, int rows, bool chain64) {
    const size_t gbytes = (size_t)std::max(rows, 1) * b->n_max * 4 * b->elem;
    const size_t g64 = chain64 ? (size_t)std::max(rows, 1) * b->n_max * 4 * sizeof(cx<double>) : 0;
    const size_t a64 = chain64 ? sizeof(cx<double>) * b->need_sites : 0;
    if (gbytes <= b->gates_bytes && g64 <= b->gates64_bytes && a64 <= b->cap_arena64) return MPS_OK;
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    if (gbytes > b->gates_bytes) {
        cudaFree(b->gates);
        b->gates = nullptr;
        b->gates_bytes = 0;
        CUDA_TRY(cudaMalloc(&b->gates, gbytes));
        b->gates_bytes = gbytes;
    }
    if (g64 > b->gates64_bytes) {
        cudaFree(b->gates64);
        b->gates64 = nullptr;
        b->gates64_bytes = 0;
        CUDA_TRY(cudaMalloc(&b->gates64, g64));
        b->gates64_bytes = g64;
    }
    if (a64 > b->cap_arena64) {
        cudaFree(b->arena64);
        b->arena64 = nullptr;
        b->cap_arena64 = 0;
        CUDA_TRY(cudaMalloc(&b->arena64, a64));
        b->cap_arena64 = a64;
    }
    return MPS_OK;
}

}  // namespace

extern "C" {

mps_status mps_create_batch(int32_t n_images, const int32_t* p, const int32_t* chi, int32_t chi_all,
                            int32_t prec, void* stream, mps_batch** out) {
    if (!out) return fail(MPS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (prec != MPS_FP64 && prec != MPS_MIXED && prec != MPS_MIXED_ORTH64 && prec != MPS_MIXED_FAST)
        return fail(MPS_ERR_INVALID_ARG, "unknown precision %d", prec);
    mps_batch* b = new (std::nothrow) mps_batch();
    if (!b) return fail(MPS_ERR_OOM, "host allocation failed");
    b->prec = prec;
    b->stream = reinterpret_cast<cudaStream_t>(stream);
    b->elem = prec == MPS_FP64 ? sizeof(cx<double>) : sizeof(cx<float>);
    mps_status st = layout_images(b, n_images, p, chi, chi_all);
    if (st == MPS_OK) st = fit_and_upload(b);
    if (st == MPS_OK && cudaStreamSynchronize(b->stream) != cudaSuccess)
        st = fail(MPS_ERR_CUDA, "stream synchronisation failed after batch creation");
    if (st != MPS_OK) {
        free_batch(b);
        return st;
    }
    *out = b;
    return MPS_OK;
}

mps_status mps_reshape_batch(mps_batch* b, int32_t n_images, const int32_t* p, const int32_t* chi,
                             int32_t chi_all) {
    if (!b) return fail(MPS_ERR_INVALID_ARG, "batch is NULL");
    // the previous layout's work and its pinned staging must be finished before reuse
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    // layout_images checks every argument before it changes the batch, so refused
    // arguments leave the batch as it was.  Once the host layout has changed, nothing
    // may launch on the batch until the device buffers match it: a reshape that fails
    // in fit_and_upload (out of memory) leaves layout_ok false until one succeeds.
    mps_status st = layout_images(b, n_images, p, chi, chi_all);
    if (st != MPS_OK) return st;
    b->circuit_done = false;
    b->layout_ok = false;
    return fit_and_upload(b);
}

mps_status mps_destroy_batch(mps_batch* b) {
    if (!b) return MPS_OK;
    cudaStreamSynchronize(b->stream);
    free_batch(b);
    return MPS_OK;
}

mps_status mps_plan_image(int32_t p, int32_t L, int32_t chi, int32_t ansatz, int32_t prec, int32_t layer_pipeline,
                          int32_t* out) {
    if (!out) return fail(MPS_ERR_INVALID_ARG, "out is NULL");
    if (p < 2 || p > 16) return fail(MPS_ERR_INVALID_ARG, "p = %d outside 2..16", p);
    if (chi < 1 || chi > MPS_CHI_LIMIT) return fail(MPS_ERR_INVALID_ARG, "chi = %d outside 1..%d", chi, MPS_CHI_LIMIT);
    if (L < 0 || L > 64) return fail(MPS_ERR_INVALID_ARG, "L = %d outside 0..64", L);
    if (ansatz != MPS_ANSATZ_LADDER && ansatz != MPS_ANSATZ_PAPER) return fail(MPS_ERR_INVALID_ARG, "unknown ansatz %d", ansatz);
    if (prec < MPS_FP64 || prec > MPS_MIXED_FAST) return fail(MPS_ERR_INVALID_ARG, "unknown precision %d", prec);
    const int n = p * p;
    bool t = false;
    const int raw = dry_run_bonds(n, L, chi, ansatz, &t);
    const int ld = site_padding(n, chi, raw);
    const ImagePlan pl = plan_image(n, L, chi, ld, ansatz, prec, layer_pipeline != 0);
    out[0] = pl.route;
    out[1] = pl.bond;
    out[2] = pl.lossy ? 1 : 0;
    out[3] = ld;
    if (pl.bond > MPS_BOND_LIMIT) return fail(MPS_ERR_UNSUPPORTED, "bond %d > %d", pl.bond, MPS_BOND_LIMIT);
    return MPS_OK;
}

mps_status mps_reserve(mps_batch* b, int32_t L_max) {
    if (!b) return fail(MPS_ERR_INVALID_ARG, "batch is NULL");
    if (L_max < 0 || L_max > 64) return fail(MPS_ERR_INVALID_ARG, "L_max = %d outside 0..64", L_max);
    if (!b->layout_ok) return fail(MPS_ERR_NOT_READY, "the batch's last reshape failed");
    mps_status st = ensure_lenv(b);
    if (st != MPS_OK) return st;
    const bool chain64 = b->prec == MPS_MIXED || b->prec == MPS_MIXED_ORTH64;
    return ensure_gates(b, std::max(L_max, b->B), chain64);
}

mps_status mps_set_launch_shape(mps_batch* b, int32_t images_per_cta, int32_t circuit_threads,
                                int32_t pauli_threads) {
    if (!b) return fail(MPS_ERR_INVALID_ARG, "batch is NULL");
    // all three checked before any is applied: a refused call changes nothing
    if (circuit_threads != 0 && circuit_threads != 32 && circuit_threads != 64 && circuit_threads != 128)
        return fail(MPS_ERR_INVALID_ARG, "circuit_threads %d (32, 64 or 128)", circuit_threads);
    if (images_per_cta < 0 || images_per_cta > 8) return fail(MPS_ERR_INVALID_ARG, "images_per_cta %d", images_per_cta);
    if (pauli_threads != 0 && pauli_threads != 32 && pauli_threads != 64 && pauli_threads != 128)
        return fail(MPS_ERR_INVALID_ARG, "pauli_threads %d (32, 64 or 128)", pauli_threads);
    if (circuit_threads) b->circuit_threads = circuit_threads;
    if (images_per_cta) b->images_per_cta = images_per_cta;
    if (pauli_threads) b->pauli_warps = pauli_threads / 32;
    return MPS_OK;
}

mps_status mps_set_layer_pipeline(mps_batch* b, int32_t enable) {
    if (!b) return fail(MPS_ERR_INVALID_ARG, "batch is NULL");
    b->layer_pipeline = enable != 0;
    return MPS_OK;
}

mps_status mps_set_real_arithmetic(mps_batch* b, int32_t enable) {
    if (!b) return fail(MPS_ERR_INVALID_ARG, "batch is NULL");
    b->real_allowed = enable != 0;
    return MPS_OK;
}

mps_status mps_set_block_truncation(mps_batch* b, int32_t enable) {
    if (!b) return fail(MPS_ERR_INVALID_ARG, "batch is NULL");
    b->block_truncation = enable != 0;
    return MPS_OK;
}

mps_status mps_set_half_structure(mps_batch* b, int32_t enable) {
    if (!b) return fail(MPS_ERR_INVALID_ARG, "batch is NULL");
    b->half_structure = enable != 0;
    return MPS_OK;
}

mps_status mps_set_pauli_sweep(mps_batch* b, int32_t mode) {
    if (!b) return fail(MPS_ERR_INVALID_ARG, "batch is NULL");
    if (mode != MPS_PAULI_COLUMN && mode != MPS_PAULI_SWEEP && mode != MPS_PAULI_AUTO)
        return fail(MPS_ERR_INVALID_ARG, "Pauli kernel mode %d (0, 1 or 2)", mode);
    b->pauli_sweep = mode;
    return MPS_OK;
}

mps_status mps_apply_circuit(mps_batch* b, const double* pixels, const mps_circuit* circ) {
    if (!b) return fail(MPS_ERR_INVALID_ARG, "batch is NULL");
    if (!pixels) return fail(MPS_ERR_INVALID_ARG, "pixels is NULL");
    if (!circ) return fail(MPS_ERR_INVALID_ARG, "circuit is NULL");
    if (circ->ansatz != MPS_ANSATZ_LADDER && circ->ansatz != MPS_ANSATZ_PAPER)
        return fail(MPS_ERR_INVALID_ARG, "unknown ansatz %d", circ->ansatz);
    if (!b->layout_ok) return fail(MPS_ERR_NOT_READY, "the batch's last reshape failed");
    int L_max = 0;
    for (int i = 0; i < b->B; ++i) {
        const int L = circ->L_per_image ? circ->L_per_image[i] : circ->L;
        if (L < 0 || L > 64) return fail(MPS_ERR_INVALID_ARG, "L[%d] = %d outside 0..64", i, L);
        L_max = std::max(L_max, L);
    }
    if (circ->ansatz == MPS_ANSATZ_LADDER && L_max > 0) {
        if (!circ->params) return fail(MPS_ERR_INVALID_ARG, "ladder ansatz needs params");
        if (circ->params_n < b->n_max)
            return fail(MPS_ERR_INVALID_ARG, "params_n = %d < largest n = %d", circ->params_n, b->n_max);
    }
    // arguments checked: a call that fails from here on leaves no circuit for
    // mps_pauli_cache to read
    b->circuit_done = false;
    // bond dimensions, shared-memory bucket and truncation per image.  Each image's
    // kernel (and so its result) depends on its own circuit only, not on the rest of
    // the batch:
    //  - a circuit (either ansatz) that truncates nowhere, with 1 <= L <= 4 and 2^L within
    //    the image's padding and chi: operator product (ladder_mpo.cu: bond 2^L at every
    //    inner cut, not left-canonical, flagged META_LENV for the Pauli kernel);
    //  - other ladder circuits that truncate nowhere with 1 <= L <= 4: layer-pipelined
    //    kernel;
    //  - a circuit that truncates lossily under MPS_MIXED or MPS_MIXED_ORTH64: the
    //    sequential kernel on a complex128 state (sequential truncation amplifies the
    //    rounding of a complex64 state far beyond 1e-5), rounded to complex64 at the end;
    //  - everything else: the sequential kernel in the batch's own precision.
    // an image whose circuit needs a bond above its site padding (above 32) gets a
    // larger padding: the batch is laid out again (its state is reset by this call anyway)
    // An image's plan depends on its shape alone (sites, layers, cap, padding; the
    // ansatz and precision are the call's), and a batch holds few distinct shapes: each
    // is planned once per call (n < 2^20, L <= 64, chi < 2^20, ld < 2^16).
    auto shape_key = [](int n, int L, int chi, int ld) {
        return (uint64_t)(uint32_t)n | (uint64_t)(uint32_t)L << 20 | (uint64_t)(uint32_t)chi << 28 |
               (uint64_t)(uint32_t)ld << 48;
    };
    std::unordered_map<uint64_t, int> bonds_memo;
    std::unordered_map<uint64_t, ImagePlan> plan_memo;
    {
        std::vector<int32_t> need(b->B, 0);
        bool grow_ld = false;
        for (int i = 0; i < b->B; ++i) {
            const ImageMeta& m = b->meta_h[i];
            const int L = circ->L_per_image ? circ->L_per_image[i] : circ->L;
            const uint64_t key = shape_key(m.n, L, m.chi, 0);
            auto it = bonds_memo.find(key);
            if (it == bonds_memo.end()) {
                bool t = false;
                it = bonds_memo.emplace(key, dry_run_bonds(m.n, L, m.chi, circ->ansatz, &t)).first;
            }
            const int bi = it->second;
            need[i] = std::max(bi, m.ld);
            if (bi > m.ld && bi <= MPS_BOND_LIMIT) grow_ld = true;
        }
        if (grow_ld) {
            CUDA_TRY(cudaStreamSynchronize(b->stream));   // pinned staging may still be in flight
            const std::vector<int32_t> p = b->p_h, chi = b->chi_h;
            b->layout_ok = false;
            mps_status st = layout_images(b, b->B, p.data(), chi.data(), 0, need.data());
            if (st == MPS_OK) st = fit_and_upload(b);
            if (st != MPS_OK) return st;
        }
    }
    int mx = 1, mx_wave = 1, mx_seq = 1, mx_64 = 1;
    bool trunc_seq = false;
    const bool chain64_on = b->prec == MPS_MIXED || b->prec == MPS_MIXED_ORTH64;
    std::vector<char> wave(b->B, 0), mpo(b->B, 0), c64(b->B, 0);
    int n_wave = 0, n_mpo = 0, n_64 = 0;
    (void)chain64_on;
    for (int i = 0; i < b->B; ++i) {
        ImageMeta& m = b->meta_h[i];
        const int L = circ->L_per_image ? circ->L_per_image[i] : circ->L;
        if (m.L != L) { m.L = L; b->meta_dirty = true; }
        const uint64_t key = shape_key(m.n, L, m.chi, m.ld);
        auto it = plan_memo.find(key);
        if (it == plan_memo.end())
            it = plan_memo.emplace(key, plan_image(m.n, L, m.chi, m.ld, circ->ansatz, b->prec, b->layer_pipeline)).first;
        const ImagePlan pl = it->second;
        const bool t = pl.lossy;
        const int bi = pl.bond;
        if (bi > m.ld) return fail(MPS_ERR_UNSUPPORTED, "image %d reaches bond %d > padding %d", i, bi, m.ld);
        mpo[i] = pl.route == ROUTE_MPO;
        const int32_t fl =
            (mpo[i] ? (META_LENV | (circ->ansatz == MPS_ANSATZ_LADDER && b->half_structure ? META_HALF : 0)) : 0) |
            (b->block_truncation ? 0 : META_FULL_EIGH);
        if (m.flags != fl) { m.flags = fl; b->meta_dirty = true; }
        if (mpo[i]) ++n_mpo;
        mx = std::max(mx, bi);
        wave[i] = pl.route == ROUTE_WAVE;
        c64[i] = pl.route == ROUTE_CHAIN64;
        if (wave[i]) {
            ++n_wave;
            mx_wave = std::max(mx_wave, bi);
        } else if (c64[i]) {
            ++n_64;
            mx_64 = std::max(mx_64, bi);
        } else if (!mpo[i]) {
            mx_seq = std::max(mx_seq, bi);
            trunc_seq = trunc_seq || t;
        }
    }
    const int chi_tpl = chi_bucket(mx);
    if (chi_tpl < 0) return fail(MPS_ERR_UNSUPPORTED, "bond dimension %d > %d not supported", mx, MPS_BOND_LIMIT);
    // work order: operator-product images, pipelined images, the rest in the batch's
    // precision, then the FP64 chains, each part by descending cost
    std::vector<int32_t> order;
    order.reserve(b->B);
    for (int32_t i : b->cost_order) if (mpo[i]) order.push_back(i);
    for (int32_t i : b->cost_order) if (wave[i]) order.push_back(i);
    for (int32_t i : b->cost_order) if (!wave[i] && !mpo[i] && !c64[i]) order.push_back(i);
    for (int32_t i : b->cost_order) if (c64[i]) order.push_back(i);
    if (n_mpo > 0) {
        const mps_status se = ensure_lenv(b);
        if (se != MPS_OK) return se;
    }
    b->any_lenv = n_mpo > 0;
    b->all_half = true;
    for (int i = 0; i < b->B; ++i) b->all_half = b->all_half && (b->meta_h[i].flags & META_HALF) != 0;
    if (order != b->order_h) {
        CUDA_TRY(cudaStreamSynchronize(b->stream));  // pinned staging may still be in flight
        std::memcpy(b->order_pinned, order.data(), sizeof(int32_t) * b->B);
        CUDA_TRY(cudaMemcpyAsync(b->order_d, b->order_pinned, sizeof(int32_t) * b->B, cudaMemcpyHostToDevice,
                                 b->stream));
        b->order_h = order;
    }
    // uploaded whenever meta_h differs from the device copy, also when an earlier
    // call changed meta_h and then failed before its upload
    if (b->meta_dirty) {
        CUDA_TRY(cudaStreamSynchronize(b->stream));  // pinned staging may still be in flight
        std::memcpy(b->meta_pinned, b->meta_h.data(), sizeof(ImageMeta) * b->B);
        CUDA_TRY(cudaMemcpyAsync(b->meta_d, b->meta_pinned, sizeof(ImageMeta) * b->B,
                                 cudaMemcpyHostToDevice, b->stream));
        b->meta_dirty = false;
    }
    // one-qubit gate table (FP64 math, rounded to the state type); a second one in FP64
    // for the FP64 chains
    const int rows = circ->ansatz == MPS_ANSATZ_LADDER ? L_max : b->B;
    {
        const mps_status se = ensure_gates(b, rows, n_64 > 0);
        if (se != MPS_OK) return se;
    }
    b->gate_n = b->n_max;
    b->L_max = L_max;
    b->n_chain64 = n_64;
    const double* pr = circ->ansatz == MPS_ANSATZ_LADDER ? circ->params : nullptr;
    mps_status st = launch_gate_table(b, circ->ansatz, L_max, pr, circ->params_n, pixels, b->prec == MPS_FP64,
                                      b->gates);
    if (st != MPS_OK) return st;
    if (n_64 > 0) {
        st = launch_gate_table(b, circ->ansatz, L_max, pr, circ->params_n, pixels, true, b->gates64);
        if (st != MPS_OK) return st;
    }
    auto launch = [&](int bucket, bool trunc) {
        switch (b->prec) {
            case MPS_FP64: return launch_circuit_fp64(b, bucket, trunc, pixels, circ->ansatz);
            case MPS_MIXED:
            case MPS_MIXED_FAST: return launch_circuit_mixed(b, bucket, trunc, pixels, circ->ansatz);
            default: return launch_circuit_orth64(b, bucket, trunc, pixels, circ->ansatz);
        }
    };
    if (n_mpo > 0) {
        b->use_wave = false;
        b->run_order = b->order_d;
        b->run_count = n_mpo;
        st = launch_ladder_mpo(b, pixels, circ->ansatz);
        if (st != MPS_OK) return st;
    }
    if (n_wave > 0) {
        b->use_wave = true;
        b->run_order = b->order_d + n_mpo;
        b->run_count = n_wave;
        st = launch(chi_bucket(mx_wave), false);
        if (st != MPS_OK) return st;
    }
    const int n_seq = b->B - n_mpo - n_wave - n_64;
    if (n_seq > 0) {
        b->use_wave = false;
        b->run_order = b->order_d + n_mpo + n_wave;
        b->run_count = n_seq;
        st = launch(chi_bucket(mx_seq), trunc_seq);
        if (st != MPS_OK) return st;
    }
    if (n_64 > 0) {
        // the FP64 chain runs on the complex128 arena and gate table, then its sites are
        // rounded into the batch's complex64 arena
        b->use_wave = false;
        b->run_order = b->order_d + (b->B - n_64);
        b->run_count = n_64;
        void* arena = b->arena;
        void* gates = b->gates;
        b->arena = b->arena64;
        b->gates = b->gates64;
        st = launch_circuit_fp64(b, chi_bucket(mx_64), true, pixels, circ->ansatz);
        b->arena = arena;
        b->gates = gates;
        if (st != MPS_OK) return st;
        st = launch_round_sites(b, b->arena64);
        if (st != MPS_OK) return st;
    }
    b->chi_tpl = chi_tpl;
    // H, R_Y(2 pi x - pi) and CNOT are real: the paper ansatz's state is real in every
    // amplitude (every kernel keeps its imaginary parts exactly zero)
    b->real = b->real_allowed && circ->ansatz == MPS_ANSATZ_PAPER && b->prec != MPS_FP64;
    b->circuit_done = true;
    return MPS_OK;
}

mps_status mps_pauli_cache(mps_batch* b, int32_t pair_set, void* out, int64_t* pair_offsets) {
    if (!b) return fail(MPS_ERR_INVALID_ARG, "batch is NULL");
    if (!out) return fail(MPS_ERR_INVALID_ARG, "out is NULL");
    if (pair_set != MPS_PAIRS_HV && pair_set != MPS_PAIRS_HVD)
        return fail(MPS_ERR_INVALID_ARG, "unknown pair set %d", pair_set);
    if (!b->circuit_done) return fail(MPS_ERR_NOT_READY, "no circuit has run on this batch");
    if (pair_offsets) {
        pair_offsets[0] = 0;
        for (int i = 0; i < b->B; ++i) pair_offsets[i + 1] = pair_offsets[i] + mps_pair_count(b->meta_h[i].p, pair_set);
    }
    const bool diag = pair_set == MPS_PAIRS_HVD;
    if (b->prec == MPS_FP64) return launch_pauli_fp64(b, out, diag);
    return launch_pauli_mixed(b, out, diag);
}

mps_status ano_features(const void* pauli, int32_t pauli_f64, int64_t n_images, int32_t m, const float* abd,
                        const float* W, const float* bias, int32_t out_dim, float* features, float* out,
                        void* stream) {
    if (!pauli || !abd || !features) return fail(MPS_ERR_INVALID_ARG, "pauli, abd and features must be non-NULL");
    if (n_images <= 0 || m <= 0) return fail(MPS_ERR_INVALID_ARG, "n_images and m must be positive");
    if (n_images > INT32_MAX) return fail(MPS_ERR_INVALID_ARG, "n_images %lld above 2^31 - 1", (long long)n_images);
    if (W && (!out || out_dim <= 0)) return fail(MPS_ERR_INVALID_ARG, "linear layer needs out and out_dim > 0");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int64_t tot = n_images * (int64_t)m;
    const int threads = 256;
    const int64_t blocks = (tot + threads - 1) / threads;
    if (pauli_f64)
        ano_kernel<double><<<(unsigned)blocks, threads, 0, s>>>(static_cast<const double*>(pauli), n_images, m, abd, features);
    else
        ano_kernel<float><<<(unsigned)blocks, threads, 0, s>>>(static_cast<const float*>(pauli), n_images, m, abd, features);
    CUDA_TRY(cudaGetLastError());
    count_launch();
    if (W) {
        const char* force = getenv("MPSANO_LINEAR");
        if (force && strcmp(force, "fp32") == 0) {
            // plain FP32 CUDA-core GEMM (kept for comparison)
            dim3 grid((out_dim + 15) / 16, (unsigned)((n_images + 15) / 16));
            linear_fp32_kernel<<<grid, 256, 0, s>>>(features, n_images, m, W, bias, out_dim, out);
        } else {
            return launch_linear_tc(features, m, 1, (int)n_images, m, W, m, 1, bias, out_dim, out, s);
        }
        CUDA_TRY(cudaGetLastError());
        count_launch();
    }
    return MPS_OK;
}

mps_status ano_status(void) {
    CUDA_TRY(cudaDeviceSynchronize());
    int st = 0, zero = 0;
    CUDA_TRY(cudaMemcpyFromSymbol(&st, g_epilogue_status, sizeof(int)));
    if (st != 0) {
        CUDA_TRY(cudaMemcpyToSymbol(g_epilogue_status, &zero, sizeof(int)));
        return fail(MPS_ERR_TIMEOUT, "a tensor-core wait of the linear layer gave up (code %d)", st);
    }
    return MPS_OK;
}

mps_status mps_sync(mps_batch* b) {
    if (!b) return fail(MPS_ERR_INVALID_ARG, "batch is NULL");
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    int st = 0;
    CUDA_TRY(cudaMemcpy(&st, b->status_d, sizeof(int), cudaMemcpyDeviceToHost));
    if (st != DEV_OK) {
        cudaMemset(b->status_d, 0, sizeof(int));
        return fail(MPS_ERR_DEVICE, "device check failed with code %d (%s)", st,
                    st == DEV_BOND_OVERFLOW ? "bond overflow" : st == DEV_BAD_SHAPE ? "bad shape" : "other");
    }
    return MPS_OK;
}

mps_status mps_bond_dims(mps_batch* b, int32_t* out) {
    if (!b || !out) return fail(MPS_ERR_INVALID_ARG, "batch and out must be non-NULL");
    if (!b->layout_ok) return fail(MPS_ERR_NOT_READY, "the batch's last reshape failed");
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    CUDA_TRY(cudaMemcpy(out, b->bonds_d, sizeof(int32_t) * b->total_bonds, cudaMemcpyDeviceToHost));
    return MPS_OK;
}

mps_status mps_set_timing(mps_batch* b, int32_t enable) {
    if (!b) return fail(MPS_ERR_INVALID_ARG, "batch is NULL");
    b->timing = enable != 0;
    return MPS_OK;
}

mps_status mps_kernel_times(mps_batch* b, double* ms, int64_t* launches) {
    if (!b || !ms || !launches) return fail(MPS_ERR_INVALID_ARG, "batch, ms and launches must be non-NULL");
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    for (int k = 0; k < KIND_COUNT; ++k) { ms[k] = 0.0; launches[k] = 0; }
    for (auto& t : b->timed) {
        float e = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&e, t.start, t.stop));
        ms[t.kind] += e;
        launches[t.kind] += 1;
        b->event_pool.push_back(t.start);
        b->event_pool.push_back(t.stop);
    }
    b->timed.clear();
    return MPS_OK;
}

mps_status mps_discarded_weight(mps_batch* b, double* out) {
    if (!b || !out) return fail(MPS_ERR_INVALID_ARG, "batch and out must be non-NULL");
    if (!b->layout_ok) return fail(MPS_ERR_NOT_READY, "the batch's last reshape failed");
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    CUDA_TRY(cudaMemcpy(out, b->discarded_d, sizeof(double) * b->B, cudaMemcpyDeviceToHost));
    return MPS_OK;
}

}  // extern "C"
