// Device-side helpers shared by the MPS kernels: a minimal complex type, warp
// reductions and the per-image metadata record.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mpsano {

template <typename T>
struct __align__(2 * sizeof(T)) cx {
    T re, im;
};

template <typename T> __device__ __forceinline__ cx<T> mk(T r, T i) { cx<T> z; z.re = r; z.im = i; return z; }
template <typename T> __device__ __forceinline__ cx<T> czero() { return mk<T>(T(0), T(0)); }
template <typename T> __device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return mk<T>(a.re + b.re, a.im + b.im); }
template <typename T> __device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return mk<T>(a.re - b.re, a.im - b.im); }
template <typename T> __device__ __forceinline__ cx<T> operator-(cx<T> a) { return mk<T>(-a.re, -a.im); }
// Products that the compiler may not fuse into a neighbouring add: with every
// multiply of the complex helpers either an explicit fma or one of these, each
// kernel instantiation computes the same bits from the same inputs.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
template <typename T> __device__ __forceinline__ cx<T> operator*(cx<T> a, cx<T> b) {
    return mk<T>(fma(a.re, b.re, -mul_rn(a.im, b.im)), fma(a.re, b.im, mul_rn(a.im, b.re)));
}
template <typename T> __device__ __forceinline__ cx<T> operator*(T s, cx<T> a) {
    return mk<T>(mul_rn(s, a.re), mul_rn(s, a.im));
}
template <typename T> __device__ __forceinline__ cx<T> conj(cx<T> a) { return mk<T>(a.re, -a.im); }
template <typename T> __device__ __forceinline__ T norm2(cx<T> a) { return fma(a.re, a.re, mul_rn(a.im, a.im)); }
// acc += a * b
template <typename T> __device__ __forceinline__ void cmac(cx<T>& acc, cx<T> a, cx<T> b) {
    acc.re = fma(a.re, b.re, acc.re); acc.re = fma(-a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im); acc.im = fma(a.im, b.re, acc.im);
}
// acc += conj(a) * b
template <typename T> __device__ __forceinline__ void cmac_cj(cx<T>& acc, cx<T> a, cx<T> b) {
    acc.re = fma(a.re, b.re, acc.re); acc.re = fma(a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im); acc.im = fma(-a.im, b.re, acc.im);
}
// acc -= a * b
template <typename T> __device__ __forceinline__ void cmsub(cx<T>& acc, cx<T> a, cx<T> b) {
    acc.re = fma(-a.re, b.re, acc.re); acc.re = fma(a.im, b.im, acc.re);
    acc.im = fma(-a.re, b.im, acc.im); acc.im = fma(-a.im, b.re, acc.im);
}
// u0 * a0 + u1 * a1 as one fma chain
template <typename T> __device__ __forceinline__ cx<T> cdot2(cx<T> u0, cx<T> a0, cx<T> u1, cx<T> a1) {
    cx<T> acc = mk<T>(mul_rn(u0.re, a0.re), mul_rn(u0.re, a0.im));
    acc.re = fma(-u0.im, a0.im, acc.re); acc.im = fma(u0.im, a0.re, acc.im);
    cmac(acc, u1, a1);
    return acc;
}
template <typename To, typename Ti> __device__ __forceinline__ cx<To> cvt(cx<Ti> a) {
    return mk<To>(To(a.re), To(a.im));
}

// The encoding R_Y(pi x)|0> = (cos(pi x / 2), sin(pi x / 2)) (Sec. II.B) in the state's
// own precision: sincospi of x / 2 in FP32 for a complex64 state (the pixel rounds to
// float, so the amplitudes carry ~1e-7, the rounding level of that state), in FP64
// for a complex128 one.
__device__ __forceinline__ void encode_amplitudes(double x, float* s, float* c) { sincospif((float)(0.5 * x), s, c); }
__device__ __forceinline__ void encode_amplitudes(double x, double* s, double* c) { sincospi(0.5 * x, s, c); }

// Element types of the contraction kernels: complex (cx<T>) or, for a state that is
// real in every amplitude (the paper ansatz: H, R_Y and CNOT are real), the scalar
// itself.  For a real element the complex helpers reduce to plain fma.
template <typename E> struct elem_traits;
template <typename T> struct elem_traits<cx<T>> {
    using scalar = T;
    static constexpr bool real = false;
};
template <> struct elem_traits<float> {
    using scalar = float;
    static constexpr bool real = true;
};
template <> struct elem_traits<double> {
    using scalar = double;
    static constexpr bool real = true;
};
template <typename E> __device__ __forceinline__ E ezero() {
    if constexpr (elem_traits<E>::real) return E(0);
    else return czero<typename elem_traits<E>::scalar>();
}
template <typename E> __device__ __forceinline__ E eone() {
    using T = typename elem_traits<E>::scalar;
    if constexpr (elem_traits<E>::real) return E(1);
    else return mk<T>(T(1), T(0));
}
// the element of a complex value stored in global memory (its real part for a real element)
template <typename E, typename T> __device__ __forceinline__ E to_elem(cx<T> v) {
    if constexpr (elem_traits<E>::real) return E(v.re);
    else return v;
}
template <typename E> __device__ __forceinline__ typename elem_traits<E>::scalar ereal(E v) {
    if constexpr (elem_traits<E>::real) return v;
    else return v.re;
}
__device__ __forceinline__ float conj(float a) { return a; }
__device__ __forceinline__ double conj(double a) { return a; }
__device__ __forceinline__ void cmac(float& acc, float a, float b) { acc = fmaf(a, b, acc); }
__device__ __forceinline__ void cmac(double& acc, double a, double b) { acc = fma(a, b, acc); }
__device__ __forceinline__ void cmac_cj(float& acc, float a, float b) { acc = fmaf(a, b, acc); }
__device__ __forceinline__ void cmac_cj(double& acc, double a, double b) { acc = fma(a, b, acc); }

template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Per-image record, built on the host, read by every kernel.
struct ImageMeta {
    int32_t p;          // image side
    int32_t n;          // qubits = p*p
    int32_t chi;        // bond cap
    int32_t L;          // layers of the last circuit
    int32_t ld;         // site-tensor padding: a site is [ld][2][ld], element (l,s,r) at (2l+s)*ld+r
    int32_t bond_off;   // offset of this image's bond array (n+1 entries)
    int64_t site_off;   // offset (in complex elements) of site 0 in the arena
    int64_t pixel_off;  // offset of the image's pixels in the packed pixel array
    int64_t pair_off;   // offset (in pairs) of the image's Pauli-cache block, horizontal + vertical
    int64_t pair_off_d; // the same with both diagonal pair sets
    int32_t flags;      // META_LENV: the MPS is not left-canonical (see ladder_mpo.cu)
    int32_t pad;
};

// ImageMeta::flags: the Pauli kernel contracts the left environments L_i (written by
// lenv_kernel) instead of taking them as the identity.
constexpr int32_t META_LENV = 1;
// ImageMeta::flags: every site but the last is half-structured (A[2l+s][r] = 0 unless
// r / (D_right / 2) == s: a ladder circuit built as an operator product), so the
// contractions over a site's right index run over half of it (see times_site_t).
constexpr int32_t META_HALF = 2;
// ImageMeta::flags: FP64 truncations always run the full FP64 eigen-decomposition, never
// the block solve that only decouples the kept from the dropped directions (both give
// the same truncated state to rounding; the flag exists to check exactly that).
constexpr int32_t META_FULL_EIGH = 4;

// Device status word: first error wins.
enum : int { DEV_OK = 0, DEV_BOND_OVERFLOW = 1, DEV_SMEM_OVERFLOW = 2, DEV_BAD_SHAPE = 3 };

__device__ __forceinline__ void raise_status(int* status, int code) {
    if (status) atomicCAS(status, DEV_OK, code);
}

}  // namespace mpsano
