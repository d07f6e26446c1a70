// Linear reconstruction layer y = W q + b (Eq. 6) on the tcgen05 tensor cores.
//
// Y[r][o] = sum_k X(r, k) W(o, k) + bias[o], FP32 in and out (optionally split over
// K: plane z of Y gets the sum over K chunks [z cps, (z+1) cps)), with X(r, k) at
// X[r * xs_r + k * xs_k] and W(o, k) at W[o * ws_o + k * ws_k] (so transposed
// operands of the backward pass need no copy).  TF32 alone has an
// 11-bit significand, so each operand is split as x = x_hi + x_lo with
// x_hi = tf32(x), x_lo = tf32(x - x_hi), and three products x_hi w_hi + x_hi w_lo +
// x_lo w_hi accumulate in FP32 (relative error near 2^-22 per term).
//
// One CTA of 128 threads computes a 128 x 128 tile of Y: D (128 lanes x 128 FP32
// columns) lives in tensor memory; A (rows of X) and B (rows of W) are staged in
// shared memory K-major without swizzling, in 8-row x 16-byte core matrices:
//   element (row, k) of a 128 x 32 panel at ((row/8)*8 + k/4)*128 + (row%8)*16 + (k%4)*4
// so core matrices adjacent in K are 128 B apart (leading byte offset) and 8-row
// groups are 1024 B apart (stride byte offset).  Thread 0 issues the MMAs
// (kind::tf32, M = 128, N = 128, K = 8 each) and commits them to an mbarrier that
// every thread waits on (bounded) before the panel is overwritten.
#pragma once
#include <stdint.h>

#include "common.cuh"

namespace mpsano {

constexpr int TC_M = 128, TC_N = 128, TC_KC = 32;               // tile and K chunk
constexpr int TC_PANEL = TC_M * TC_KC * 4;                       // bytes per operand panel
constexpr uint32_t TC_LBO = 128, TC_SBO = 1024;
constexpr long TC_WAIT_LIMIT = 1L << 22;                         // mbarrier polls before giving up
constexpr int DEV_TC_TIMEOUT = 16;                               // status code of a failed wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor of tcgen05 (no swizzle).
__device__ __forceinline__ uint64_t tc_smem_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((TC_LBO >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((TC_SBO >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version
    return d;
}

// Instruction descriptor: D = F32, A = B = TF32, both K-major, N = 128, M = 128.
constexpr uint32_t TC_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_N >> 3) << 17) |
                              ((uint32_t)(TC_M >> 4) << 24);

__device__ __forceinline__ uint32_t tf32_round(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ int tc_panel_offset(int row, int k) {
    return ((row >> 3) * (TC_KC / 4) + (k >> 2)) * 128 + (row & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ bool tc_mbar_wait(uint32_t mbar, uint32_t parity) {
    for (long i = 0; i < TC_WAIT_LIMIT; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__global__ void __launch_bounds__(128) linear_tc_kernel(const float* __restrict__ X, int64_t xs_r, int64_t xs_k,
                                                        int rows, int K, const float* __restrict__ W,
                                                        int64_t ws_o, int64_t ws_k,
                                                        const float* __restrict__ bias, int out_dim,
                                                        float* __restrict__ Y, int chunks_per_split, int* status) {
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    unsigned char* a_hi = tc_smem;
    unsigned char* a_lo = a_hi + TC_PANEL;
    unsigned char* b_hi = a_lo + TC_PANEL;
    unsigned char* b_lo = b_hi + TC_PANEL;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(b_lo + TC_PANEL);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int r0 = blockIdx.y * TC_M, o0 = blockIdx.x * TC_N;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TC_N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;

    // split K: CTA z of the grid's z dimension takes K chunks [z cps, (z+1) cps) and
    // writes its partial sums to plane z of Y (rows x out_dim each)
    const int chunks = (K + TC_KC - 1) / TC_KC;
    const int ch0 = blockIdx.z * chunks_per_split;
    const int ch1 = ch0 + chunks_per_split < chunks ? ch0 + chunks_per_split : chunks;
    Y += (size_t)blockIdx.z * rows * out_dim;
    bool ok = true;
    int failed_parity = 0;
    for (int ch = ch0; ch < ch1 && ok; ++ch) {
        const int lc = ch - ch0;   // local chunk: mbarrier phase and accumulate flag
        // stage the hi/lo panels of this K chunk (zero outside the matrices); consecutive
        // threads walk the operand's unit-stride index so the loads coalesce
        const bool x_kfast = xs_k == 1, w_kfast = ws_k == 1;
        // unrolled so that several global loads are in flight per thread (the staging
        // is latency-bound: 32 loads per thread and operand per chunk; by 32 the index
        // arithmetic takes 255 registers, by 16 it takes 60)
#pragma unroll 16
        for (int e = tid; e < TC_M * TC_KC; e += 128) {
            const int row = x_kfast ? e / TC_KC : e % TC_M, k = x_kfast ? e % TC_KC : e / TC_M;
            const int kk = ch * TC_KC + k;
            const int off = tc_panel_offset(row, k);
            float xa = 0.f;
            if (r0 + row < rows && kk < K) xa = X[(int64_t)(r0 + row) * xs_r + (int64_t)kk * xs_k];
            const uint32_t xh = tf32_round(xa);
            *reinterpret_cast<uint32_t*>(a_hi + off) = xh;
            *reinterpret_cast<uint32_t*>(a_lo + off) = tf32_round(xa - __uint_as_float(xh));
        }
#pragma unroll 16
        for (int e = tid; e < TC_N * TC_KC; e += 128) {
            const int row = w_kfast ? e / TC_KC : e % TC_N, k = w_kfast ? e % TC_KC : e / TC_N;
            const int kk = ch * TC_KC + k;
            const int off = tc_panel_offset(row, k);
            float wb = 0.f;
            if (o0 + row < out_dim && kk < K) wb = W[(int64_t)(o0 + row) * ws_o + (int64_t)kk * ws_k];
            const uint32_t wh = tf32_round(wb);
            *reinterpret_cast<uint32_t*>(b_hi + off) = wh;
            *reinterpret_cast<uint32_t*>(b_lo + off) = tf32_round(wb - __uint_as_float(wh));
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            for (int ks = 0; ks < TC_KC / 8; ++ks) {
                const uint32_t koff = ks * 2 * TC_LBO;   // 8 TF32 = two core matrices along K
                const uint64_t dah = tc_smem_desc(smem_u32(a_hi) + koff), dal = tc_smem_desc(smem_u32(a_lo) + koff);
                const uint64_t dbh = tc_smem_desc(smem_u32(b_hi) + koff), dbl = tc_smem_desc(smem_u32(b_lo) + koff);
                const uint32_t acc0 = (lc > 0 || ks > 0) ? 1u : 0u;
                // D (+)= A_lo B_hi, then + A_hi B_lo, then + A_hi B_hi
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
                    "l"(dal), "l"(dbh), "r"(TC_IDESC), "r"(acc0));
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
                    "l"(dah), "l"(dbl), "r"(TC_IDESC), "r"(1u));
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
                    "l"(dah), "l"(dbh), "r"(TC_IDESC), "r"(1u));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(mbar)));
        }
        // every thread waits for the MMAs of this chunk before the panels are reused;
        // the outcome is made uniform over the CTA (the epilogue is warp-collective)
        ok = __syncthreads_and(tc_mbar_wait(smem_u32(mbar), (uint32_t)(lc & 1)) ? 1 : 0) != 0;
        failed_parity = lc & 1;
        asm volatile("tcgen05.fence::after_thread_sync;");
    }
    if (!ok) {
        // record the failure, give the MMAs in flight one more bounded wait, then free TMEM
        if (tid == 0) raise_status(status, DEV_TC_TIMEOUT);
        tc_mbar_wait(smem_u32(mbar), (uint32_t)failed_parity);
    } else {
        // epilogue: warp w reads TMEM lanes 32w..32w+31 (rows), 8 columns at a time
        const int row = r0 + 32 * warp + lane;
        for (int c0 = 0; c0 < TC_N; c0 += 8) {
            uint32_t v[8];
            const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            if (row < rows) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int o = o0 + c0 + j;
                    if (o < out_dim) Y[(size_t)row * out_dim + o] = __uint_as_float(v[j]) + (bias ? bias[o] : 0.f);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_N));
    }
}

constexpr size_t TC_SMEM_BYTES = 4 * TC_PANEL + 64;

}  // namespace mpsano
