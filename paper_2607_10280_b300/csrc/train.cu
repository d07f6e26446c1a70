// Training on cached Pauli expectations (Sec. II.C-D): one full-batch step of the
// MSE term of Eq. 7 through the ANO features (Eq. 4-5) and the linear layer
// (Eq. 6), with two Adam optimizers, one for (A, B, D) and one for (W, b).
//
// Forward:  f[i][q] = sum_alpha c[q][alpha] P[i][q][alpha],  c[q] = M abd[q]
//           y_hat[i] = W f[i] + b
// Backward: g_y = 2 lambda / (B O) (y_hat - y)
//           g_W = g_y^T f,  g_b = sum_i g_y[i],  g_f = g_y W
//           g_c[q][alpha] = sum_i g_f[i][q] P[i][q][alpha],  g_abd[q] = M^T g_c[q]
// The three GEMMs run on the tcgen05 kernel of the linear layer (strided operands,
// 3-term TF32 split); reductions over the batch accumulate in FP64 in a fixed
// order, so a step is bit-reproducible.
#include "mpsano.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "batch.h"
#include "common.cuh"
#include "epilogue.cuh"

using namespace mpsano;

namespace {

constexpr int LOSS_BLOCKS = 296;   // 2 x 148 SMs, fixed so the reduction order is fixed
constexpr int RED_THREADS = 256;

// g_y = scale (y_hat - y) in place; per-block sums of (y_hat - y)^2 in FP64.
__global__ void __launch_bounds__(RED_THREADS) mse_grad_kernel(float* __restrict__ yhat, const float* __restrict__ y,
                                                              int64_t total, float scale,
                                                              double* __restrict__ partial) {
    __shared__ double red[RED_THREADS / 32];
    double acc = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const float r = yhat[t] - y[t];
        acc += (double)r * (double)r;
        yhat[t] = scale * r;
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < RED_THREADS / 32; ++w) s += red[w];
        partial[blockIdx.x] = s;
    }
}

// one warp: lane l sums partials l, l + 32, ...; the lane sums combine in a fixed
// butterfly order
__global__ void loss_final_kernel(const double* __restrict__ partial, int n, double factor, double* __restrict__ loss) {
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += 32) s += partial[i];
    s = warp_sum(s);
    if (threadIdx.x == 0) *loss = factor * s;
}

// g_b[o] = sum_i g_y[i][o]: block of 32 x 8 threads per 32 outputs, 8 row slices
// summed in FP64 and combined in a fixed order.
__global__ void __launch_bounds__(256) bias_grad_kernel(const float* __restrict__ gy, int64_t B, int O,
                                                        float* __restrict__ gb) {
    __shared__ double part[8][33];
    const int c = threadIdx.x & 31, slice = threadIdx.x >> 5;
    const int o = blockIdx.x * 32 + c;
    double s = 0.0;
    if (o < O)
        for (int64_t i = slice; i < B; i += 8) s += gy[i * O + o];
    part[slice][c] = s;
    __syncthreads();
    if (slice == 0 && o < O) {
        double t = 0.0;
        for (int k = 0; k < 8; ++k) t += part[k][c];
        gb[o] = (float)t;
    }
}

// One block per pair q: g_c[q][alpha] = sum_i g_f[i][q] P[i][q][alpha] (16 partial
// sums per alpha, combined in a fixed order), then g_abd[q][k] = sum_alpha M[alpha][k]
// g_c[q][alpha] with M[alpha][k] = c_alpha(e_k) from the closed form of Eq. 4.
template <typename TP>
__global__ void __launch_bounds__(RED_THREADS) coeff_grad_kernel(const TP* __restrict__ pauli,
                                                                const float* __restrict__ gf, int64_t B, int m,
                                                                float* __restrict__ gabd) {
    __shared__ double part[16][17];
    __shared__ float gc[16];
    const int q = blockIdx.x;
    const int alpha = threadIdx.x & 15, slice = threadIdx.x >> 4;
    double s = 0.0;
    for (int64_t i = slice; i < B; i += 16)
        s += (double)gf[i * m + q] * (double)pauli[(i * m + q) * 16 + alpha];
    part[slice][alpha] = s;
    __syncthreads();
    if (threadIdx.x < 16) {
        double t = 0.0;
        for (int p = 0; p < 16; ++p) t += part[p][threadIdx.x];
        gc[threadIdx.x] = (float)t;
    }
    __syncthreads();
    if (threadIdx.x < 16) {
        const int k = threadIdx.x;
        float e[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) e[j] = j == k ? 1.f : 0.f;
        float acc = 0.f;
        for (int a = 0; a < 16; ++a) acc = fmaf(pauli_coeff(e, a), gc[a], acc);
        gabd[(size_t)q * 16 + k] = acc;
    }
}

// Adam (Kingma and Ba, Algorithm 1) over three parameter segments that share one
// gradient array and one moment array: [0, n0) abd, [n0, n1) W, [n1, n2) b.
__global__ void adam_kernel(float* __restrict__ abd, float* __restrict__ W, float* __restrict__ b,
                            const float* __restrict__ g, float* __restrict__ mom1, float* __restrict__ mom2,
                            int64_t n0, int64_t n1, int64_t n2, float lr_abd, float lr_lin, float beta1,
                            float beta2, float eps, float c1, float c2) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n2) return;
    float* theta;
    float lr;
    if (t < n0) { theta = abd + t; lr = lr_abd; }
    else if (t < n1) { theta = W + (t - n0); lr = lr_lin; }
    else { theta = b + (t - n1); lr = lr_lin; }
    const float gt = g[t];
    const float m = beta1 * mom1[t] + (1.f - beta1) * gt;
    const float v = beta2 * mom2[t] + (1.f - beta2) * gt * gt;
    mom1[t] = m;
    mom2[t] = v;
    *theta -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

constexpr int GEMM_SPLIT = 16;     // K splits of the two backward GEMMs (K = out_dim, n_images)

struct TrainLayout {
    int64_t feats, gy, gf, grads, partial, planes, total;   // float offsets
    int64_t n_abd, n_w, n_b;
};

TrainLayout train_layout(int64_t B, int m, int O) {
    TrainLayout t;
    t.n_abd = (int64_t)m * 16;
    t.n_w = (int64_t)O * m;
    t.n_b = O;
    t.feats = 0;
    t.gy = t.feats + B * m;
    t.gf = t.gy + B * O;
    t.grads = t.gf + B * m;
    t.partial = (t.grads + t.n_abd + t.n_w + t.n_b + 1) & ~int64_t(1);   // 8-byte aligned doubles
    t.planes = t.partial + 2 * LOSS_BLOCKS;                               // split-K partial tiles
    t.total = t.planes + GEMM_SPLIT * std::max(B * m, (int64_t)O * m);
    return t;
}

}  // namespace

extern "C" {

int64_t ano_train_workspace_floats(int64_t n_images, int32_t m, int32_t out_dim) {
    if (n_images <= 0 || m <= 0 || out_dim <= 0) return -1;
    return train_layout(n_images, m, out_dim).total;
}

mps_status ano_train_step(const void* pauli, int32_t pauli_f64, int64_t n_images, int32_t m, float* abd, float* W,
                          float* bias, int32_t out_dim, const float* targets, float* adam_moments, int32_t step,
                          const ano_adam* hp, float* workspace, double* loss, void* stream) {
    if (!pauli || !abd || !W || !bias || !targets || !adam_moments || !hp || !workspace || !loss)
        return fail(MPS_ERR_INVALID_ARG, "ano_train_step: a required pointer is NULL");
    if (n_images <= 0 || m <= 0 || out_dim <= 0)
        return fail(MPS_ERR_INVALID_ARG, "n_images, m and out_dim must be positive");
    if (n_images > (1 << 30)) return fail(MPS_ERR_INVALID_ARG, "n_images %lld too large", (long long)n_images);
    if (step < 1) return fail(MPS_ERR_INVALID_ARG, "step %d (Adam steps count from 1)", step);
    if (!(hp->beta1 >= 0.f && hp->beta1 < 1.f && hp->beta2 >= 0.f && hp->beta2 < 1.f && hp->eps > 0.f))
        return fail(MPS_ERR_INVALID_ARG, "Adam needs 0 <= beta1, beta2 < 1 and eps > 0");
    if ((reinterpret_cast<uintptr_t>(workspace) & 7) != 0)
        return fail(MPS_ERR_INVALID_ARG, "workspace must be 8-byte aligned");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const TrainLayout t = train_layout(n_images, m, out_dim);
    float* feats = workspace + t.feats;
    float* gy = workspace + t.gy;
    float* gf = workspace + t.gf;
    float* g_abd = workspace + t.grads;
    float* g_w = g_abd + t.n_abd;
    float* g_b = g_w + t.n_w;
    double* partial = reinterpret_cast<double*>(workspace + t.partial);
    const int B = (int)n_images, O = out_dim;

    // forward: features and y_hat (into the g_y buffer)
    mps_status st = ano_features(pauli, pauli_f64, n_images, m, abd, W, bias, out_dim, feats, gy, stream);
    if (st != MPS_OK) return st;
    // loss and g_y
    const int64_t total = (int64_t)B * O;
    const double factor = (double)hp->mse_weight / (double)total;
    mse_grad_kernel<<<LOSS_BLOCKS, RED_THREADS, 0, s>>>(gy, targets, total, (float)(2.0 * factor), partial);
    CUDA_TRY(cudaGetLastError());
    count_launch();
    loss_final_kernel<<<1, 32, 0, s>>>(partial, LOSS_BLOCKS, factor, loss);
    CUDA_TRY(cudaGetLastError());
    count_launch();
    // g_f[i][q] = sum_o g_y[i][o] W[o][q]      (X = g_y, "W"(q, o) = W[o][q])
    st = launch_linear_tc(gy, O, 1, B, O, W, 1, m, nullptr, m, gf, s, GEMM_SPLIT, workspace + t.planes);
    if (st != MPS_OK) return st;
    // g_W[o][q] = sum_i g_y[i][o] f[i][q]       (X(o, i) = g_y[i][o], "W"(q, i) = f[i][q])
    st = launch_linear_tc(gy, 1, O, O, B, feats, 1, m, nullptr, m, g_w, s, GEMM_SPLIT, workspace + t.planes);
    if (st != MPS_OK) return st;
    bias_grad_kernel<<<(O + 31) / 32, 256, 0, s>>>(gy, n_images, O, g_b);
    CUDA_TRY(cudaGetLastError());
    count_launch();
    if (pauli_f64)
        coeff_grad_kernel<double><<<m, RED_THREADS, 0, s>>>(static_cast<const double*>(pauli), gf, n_images, m, g_abd);
    else
        coeff_grad_kernel<float><<<m, RED_THREADS, 0, s>>>(static_cast<const float*>(pauli), gf, n_images, m, g_abd);
    CUDA_TRY(cudaGetLastError());
    count_launch();
    // both Adam optimizers in one launch
    const int64_t n2 = t.n_abd + t.n_w + t.n_b;
    const double c1 = 1.0 - std::pow((double)hp->beta1, step), c2 = 1.0 - std::pow((double)hp->beta2, step);
    adam_kernel<<<(unsigned)((n2 + 255) / 256), 256, 0, s>>>(abd, W, bias, g_abd, adam_moments, adam_moments + n2,
                                                             t.n_abd, t.n_abd + t.n_w, n2, hp->lr_abd, hp->lr_linear,
                                                             hp->beta1, hp->beta2, hp->eps, (float)c1, (float)c2);
    CUDA_TRY(cudaGetLastError());
    count_launch();
    return MPS_OK;
}

}  // extern "C"
