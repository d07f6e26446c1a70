// ANO epilogue (Sec. II.A, II.C): Hermitian observables from (A, B, D), Pauli
// coefficients c_{q,alpha} = Tr(H_q P_alpha) / 4 (Eq. 4), features
// q_q = sum_alpha c_{q,alpha} <P_alpha> (Eq. 5).
#pragma once
#include "common.cuh"

namespace mpsano {

// Row x of a one-qubit Pauli has one nonzero entry, at column pauli_col(a, x),
// with value pauli_val(a, x) (I, X, Y, Z = 0..3).
__device__ __forceinline__ int pauli_col(int a, int x) { return (a == 1 || a == 2) ? 1 - x : x; }
__device__ __forceinline__ cx<float> pauli_val(int a, int x) {
    if (a == 2) return mk<float>(0.f, x == 0 ? -1.f : 1.f);
    if (a == 3) return mk<float>(x == 0 ? 1.f : -1.f, 0.f);
    return mk<float>(1.f, 0.f);
}

// H_q[k][l] from the 16 parameters: D on the diagonal, A + iB above it for the
// upper pairs (0,1),(0,2),(0,3),(1,2),(1,3),(2,3), conjugates below.
__device__ __forceinline__ cx<float> herm_entry(const float* abd, int k, int l) {
    if (k == l) return mk<float>(abd[12 + k], 0.f);
    const int lo = k < l ? k : l, hi = k < l ? l : k;
    const int u = lo == 0 ? hi - 1 : (lo == 1 ? hi + 1 : 5);
    return mk<float>(abd[u], k < l ? abd[6 + u] : -abd[6 + u]);
}

// c_alpha = Tr(H P_alpha) / 4 = sum_row H[col(row)][row] val(row) / 4
__device__ __forceinline__ float pauli_coeff(const float* abd, int alpha) {
    const int a = alpha >> 2, b = alpha & 3;
    cx<float> acc = czero<float>();
    for (int row = 0; row < 4; ++row) {
        const int x = row >> 1, y = row & 1;
        const int col = 2 * pauli_col(a, x) + pauli_col(b, y);
        cmac(acc, herm_entry(abd, col, row), pauli_val(a, x) * pauli_val(b, y));
    }
    return 0.25f * acc.re;
}

// One thread per (image, pair).
template <typename TP>
__global__ void ano_kernel(const TP* __restrict__ pauli, int64_t n_images, int m,
                           const float* __restrict__ abd, float* __restrict__ features) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_images * m) return;
    const int q = (int)(t % m);
    const float* pq = abd + (size_t)q * 16;
    const TP* P = pauli + (size_t)t * 16;
    float acc = 0.f;
#pragma unroll
    for (int alpha = 0; alpha < 16; ++alpha) acc = fmaf(pauli_coeff(pq, alpha), (float)P[alpha], acc);
    features[t] = acc;
}

// Plain FP32 y = W q + b on CUDA cores, used when tensor-core tiles do not apply.
// 16 x 16 output tile per block, K staged through shared memory.
static __global__ void linear_fp32_kernel(const float* __restrict__ X, int64_t rows, int K,
                                   const float* __restrict__ W, const float* __restrict__ bias,
                                   int out_dim, float* __restrict__ Y) {
    __shared__ float xs[16][17], ws[16][17];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t r = (int64_t)blockIdx.y * 16 + ty;
    const int o = blockIdx.x * 16 + tx;
    float acc = 0.f;
    for (int k0 = 0; k0 < K; k0 += 16) {
        const int64_t rr = (int64_t)blockIdx.y * 16 + ty;
        xs[ty][tx] = (rr < rows && k0 + tx < K) ? X[rr * K + k0 + tx] : 0.f;
        const int oo = blockIdx.x * 16 + ty;
        ws[ty][tx] = (oo < out_dim && k0 + tx < K) ? W[(size_t)oo * K + k0 + tx] : 0.f;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) acc = fmaf(xs[ty][k], ws[tx][k], acc);
        __syncthreads();
    }
    if (r < rows && o < out_dim) Y[r * out_dim + o] = acc + (bias ? bias[o] : 0.f);
}

}  // namespace mpsano
