// Pauli-cache kernels (Sec. II.C, Eq. 5).
//
// The circuit kernel leaves every MPS left-canonical with the centre at site n-1,
// so the environment of sites 0..i-1 is the identity.  Two kernels remain:
//
//   renv_kernel   one warp per image: right environments R_j (contraction of sites
//                 j+1..n-1 with their conjugates, bra index first) for j = n-1..0,
//                 R_{j-1} = sum_s conj(A_j^s) R_j A_j^{sT}, and <psi|psi> = R_{-1}.
//
//   pauli_kernel  one warp per (image, grid column c).  The warp walks column c
//                 from the bottom row up.  At a column site j it
//                   - closes the vertical pair (j, j+p) with the three closing
//                     matrices C_b carried up from site j+p,
//                   - builds the closings of site j as a right site,
//                       C_b^{(j)} = sum_{s,s'} P_b[s][s'] conj(A_j^s) R_j A_j^{s'T},
//                   - closes the horizontal pair (j-1, j) with them,
//                   - carries them through sites j-1, ..., j-p+1 with
//                       C <- sum_s conj(A^s) C A^{sT}.
//                 A left site i contributes E_a[r][r'] = sum_{l,s,s'} conj(A[l,s,r])
//                 P_a[s][s'] A[l,s',r'] and <P_a (x) P_b> = <E_a, C_b> / <psi|psi>,
//                 <P_a> = <E_a, R_i> / <psi|psi> (elementwise product summed).
//
// D x D matrices live in per-warp shared memory with row stride CS = CHI + 1.
#pragma once
#include "common.cuh"

namespace mpsano {

template <typename T, int CHI>
struct PauliLayout {
    static constexpr int CS = CHI + 1;
    static constexpr int MAT = CHI * CS;
    // A (2 MAT), R, Z (2 MAT), C (3 MAT), E
    static constexpr int NMAT = 9;
    static constexpr size_t bytes = sizeof(cx<T>) * NMAT * MAT;
};

// Z_s[r][l'] = sum_{r'} M[r][r'] A[l', s, r'] for s = 0, 1  (M is Dr x Dr, Z is Dr x Dl)
template <typename T, int CS>
__device__ __forceinline__ void prod_MAt(const cx<T>* M, const cx<T>* A, cx<T>* Z0, cx<T>* Z1,
                                         int Dl, int Dr, int lane) {
    const int tot = 2 * Dl * Dr;
    for (int o = lane; o < tot; o += 32) {
        const int r = o % Dr;
        const int rest = o / Dr;
        const int lp = rest % Dl, s = rest / Dl;
        const cx<T>* m = M + r * CS;
        const cx<T>* a = A + (2 * lp + s) * CS;
        cx<T> acc = czero<T>();
#pragma unroll 4
        for (int rp = 0; rp < Dr; ++rp) cmac(acc, m[rp], a[rp]);
        (s ? Z1 : Z0)[r * CS + lp] = acc;
    }
}

// out[l][l'] = sum_r conj(A[l, sa, r]) Za[r][l'] (+ conj(A[l, sb, r]) Zb[r][l'] if Zb)
template <typename T, int CS>
__device__ __forceinline__ void prod_AhZ(const cx<T>* A, int sa, const cx<T>* Za, int sb, const cx<T>* Zb,
                                         cx<T>* out, int Dl, int Dr, int lane) {
    for (int o = lane; o < Dl * Dl; o += 32) {
        const int l = o / Dl, lp = o % Dl;
        cx<T> acc = czero<T>();
        const cx<T>* aa = A + (2 * l + sa) * CS;
#pragma unroll 4
        for (int r = 0; r < Dr; ++r) cmac_cj(acc, aa[r], Za[r * CS + lp]);
        if (Zb) {
            const cx<T>* ab = A + (2 * l + sb) * CS;
#pragma unroll 4
            for (int r = 0; r < Dr; ++r) cmac_cj(acc, ab[r], Zb[r * CS + lp]);
        }
        out[l * CS + lp] = acc;
    }
}

template <typename T, int CS>
__device__ __forceinline__ void load_site_p(cx<T>* dst, const cx<T>* src, int ld, int Dl, int Dr, int lane) {
    for (int o = lane; o < 2 * Dl * Dr; o += 32) {
        const int row = o / Dr, r = o % Dr;
        dst[row * CS + r] = src[row * ld + r];
    }
}

template <typename T, int CS>
__device__ __forceinline__ void load_mat(cx<T>* dst, const cx<T>* src, int ld, int D, int lane) {
    for (int o = lane; o < D * D; o += 32) dst[(o / D) * CS + (o % D)] = src[(o / D) * ld + (o % D)];
}

// sum_{r,r'} X[r][r'] Y[r][r'] (real part), full-warp result
template <typename T, int CS>
__device__ __forceinline__ T dot_re(const cx<T>* X, const cx<T>* Y, int D, int lane) {
    T acc = T(0);
    for (int o = lane; o < D * D; o += 32) {
        const int i = (o / D) * CS + (o % D);
        acc = fma(X[i].re, Y[i].re, acc);
        acc = fma(-X[i].im, Y[i].im, acc);
    }
    return warp_sum(acc);
}

// E_a (a = 1..3: X, Y, Z) of a left site A (Dl x 2 x Dr) with identity left
// environment: E_a = sum_{s,s'} P_a[s][s'] F_{ss'}, F_{ss'}[r][r'] = sum_l conj(A[l,s,r]) A[l,s',r'].
template <typename T, int CS>
__device__ __forceinline__ void left_pauli_env(const cx<T>* A, int a, cx<T>* E, int Dl, int Dr, int lane) {
    for (int o = lane; o < Dr * Dr; o += 32) {
        const int r = o / Dr, rp = o % Dr;
        cx<T> v = czero<T>();
        if (a == 3) {  // Z: F00 - F11
            cx<T> f0 = czero<T>(), f1 = czero<T>();
            for (int l = 0; l < Dl; ++l) {
                cmac_cj(f0, A[(2 * l) * CS + r], A[(2 * l) * CS + rp]);
                cmac_cj(f1, A[(2 * l + 1) * CS + r], A[(2 * l + 1) * CS + rp]);
            }
            v = f0 - f1;
        } else {
            cx<T> f01 = czero<T>(), f10 = czero<T>();
            for (int l = 0; l < Dl; ++l) {
                cmac_cj(f01, A[(2 * l) * CS + r], A[(2 * l + 1) * CS + rp]);
                cmac_cj(f10, A[(2 * l + 1) * CS + r], A[(2 * l) * CS + rp]);
            }
            if (a == 1) v = f01 + f10;                       // X
            else v = mk<T>(f01.im - f10.im, f10.re - f01.re);  // Y: -i f01 + i f10
        }
        E[r * CS + rp] = v;
    }
}

// Closings of a right site: from G_{ss'} = conj(A^s) R A^{s'T}:
//   C_X = G01 + G10, C_Y = -i G01 + i G10, C_Z = G00 - G11, R_new = G00 + G11.
// Z0, Z1 hold R A^{sT}.  G10 = G01^H because R is Hermitian.
template <typename T, int CS>
__device__ __forceinline__ void right_closings(const cx<T>* A, const cx<T>* Z0, const cx<T>* Z1,
                                               cx<T>* CX, cx<T>* CY, cx<T>* CZ, cx<T>* Rnew,
                                               int Dl, int Dr, int lane) {
    // G00 -> CZ, G11 -> CX, G01 -> CY (scratch), then combine in place
    prod_AhZ<T, CS>(A, 0, Z0, 0, nullptr, CZ, Dl, Dr, lane);
    prod_AhZ<T, CS>(A, 1, Z1, 0, nullptr, CX, Dl, Dr, lane);
    prod_AhZ<T, CS>(A, 0, Z1, 0, nullptr, CY, Dl, Dr, lane);
    __syncwarp();
    // element-wise combine; G10[l][l'] = conj(G01[l'][l]) needs the transpose, so
    // read everything first into registers per (l, l') pair with l <= l'
    for (int o = lane; o < Dl * Dl; o += 32) {
        const int l = o / Dl, lp = o % Dl;
        if (lp < l) continue;
        const cx<T> g00a = CZ[l * CS + lp], g00b = CZ[lp * CS + l];
        const cx<T> g11a = CX[l * CS + lp], g11b = CX[lp * CS + l];
        const cx<T> g01a = CY[l * CS + lp], g01b = CY[lp * CS + l];
        const cx<T> g10a = conj(g01b), g10b = conj(g01a);   // G10[l][l'], G10[l'][l]
        if (Rnew) { Rnew[l * CS + lp] = g00a + g11a; Rnew[lp * CS + l] = g00b + g11b; }
        CZ[l * CS + lp] = g00a - g11a; CZ[lp * CS + l] = g00b - g11b;
        CX[l * CS + lp] = g01a + g10a; CX[lp * CS + l] = g01b + g10b;
        const cx<T> da = g10a - g01a, db = g10b - g01b;       // -i G01 + i G10 = i (G10 - G01)
        CY[l * CS + lp] = mk<T>(-da.im, da.re); CY[lp * CS + l] = mk<T>(-db.im, db.re);
    }
    __syncwarp();
}

template <typename T, int CHI>
__global__ void __launch_bounds__(512) renv_kernel(const ImageMeta* __restrict__ meta, int n_images,
                                                   const cx<T>* __restrict__ arena,
                                                   const int32_t* __restrict__ bonds,
                                                   cx<T>* __restrict__ renv, int64_t renv_stride,
                                                   T* __restrict__ norm_out) {
    using Lay = PauliLayout<T, CHI>;
    constexpr int CS = Lay::CS, MAT = Lay::MAT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int img = blockIdx.x * (blockDim.x >> 5) + warp;
    if (img >= n_images) return;
    cx<T>* base = reinterpret_cast<cx<T>*>(smem_raw + (size_t)warp * Lay::bytes);
    cx<T>* A = base;
    cx<T>* R = base + 2 * MAT;
    cx<T>* Z0 = base + 3 * MAT;
    cx<T>* Z1 = base + 4 * MAT;
    const ImageMeta mt = meta[img];
    const int n = mt.n, ld = mt.ld;
    const int32_t* bd = bonds + mt.bond_off;
    const cx<T>* sites = arena + mt.site_off;
    cx<T>* rg = renv + (size_t)img * renv_stride;
    if (lane == 0) R[0] = mk<T>(T(1), T(0));
    __syncwarp();
    for (int j = n - 1; j >= 0; --j) {
        const int Dl = bd[j], Dr = bd[j + 1];
        // store R_j
        cx<T>* dst = rg + (size_t)j * CHI * CHI;
        for (int o = lane; o < Dr * Dr; o += 32) dst[(o / Dr) * CHI + (o % Dr)] = R[(o / Dr) * CS + (o % Dr)];
        load_site_p<T, CS>(A, sites + (size_t)j * 2 * ld * ld, ld, Dl, Dr, lane);
        __syncwarp();
        prod_MAt<T, CS>(R, A, Z0, Z1, Dl, Dr, lane);
        __syncwarp();
        prod_AhZ<T, CS>(A, 0, Z0, 1, Z1, R, Dl, Dr, lane);
        __syncwarp();
    }
    if (lane == 0) norm_out[img] = R[0].re;
}

template <typename T, int CHI>
__global__ void __launch_bounds__(512) pauli_kernel(const ImageMeta* __restrict__ meta, int n_units,
                                                    const int32_t* __restrict__ unit_image,
                                                    const cx<T>* __restrict__ arena,
                                                    const int32_t* __restrict__ bonds,
                                                    const cx<T>* __restrict__ renv, int64_t renv_stride,
                                                    const T* __restrict__ norms, T* __restrict__ out) {
    using Lay = PauliLayout<T, CHI>;
    constexpr int CS = Lay::CS, MAT = Lay::MAT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int unit = blockIdx.x * (blockDim.x >> 5) + warp;
    if (unit >= n_units) return;
    const int img = unit_image[2 * unit], c = unit_image[2 * unit + 1];
    cx<T>* base = reinterpret_cast<cx<T>*>(smem_raw + (size_t)warp * Lay::bytes);
    cx<T>* A = base;               // 2 MAT
    cx<T>* R = base + 2 * MAT;
    cx<T>* Z0 = base + 3 * MAT;
    cx<T>* Z1 = base + 4 * MAT;
    cx<T>* C = base + 5 * MAT;     // 3 MAT: C_X, C_Y, C_Z
    cx<T>* E = base + 8 * MAT;
    const ImageMeta mt = meta[img];
    const int p = mt.p, ld = mt.ld;
    const int32_t* bd = bonds + mt.bond_off;
    const cx<T>* sites = arena + mt.site_off;
    const cx<T>* rg = renv + (size_t)img * renv_stride;
    const T inv_norm = T(1) / norms[img];
    T* outp = out + (size_t)mt.pair_off * 16;
    const int nh = p * (p - 1);  // horizontal pairs come first

    T single_up[3] = {T(0), T(0), T(0)};   // <P_b> of the site that created the carried C
    for (int row = p - 1; row >= 0; --row) {
        const int j = row * p + c;
        const int Dl = bd[j], Dr = bd[j + 1];
        load_site_p<T, CS>(A, sites + (size_t)j * 2 * ld * ld, ld, Dl, Dr, lane);
        load_mat<T, CS>(R, rg + (size_t)j * CHI * CHI, CHI, Dr, lane);
        __syncwarp();
        // site j as the left site: single-site terms and the vertical pair (j, j+p)
        T single_j[3], vert[9];
        for (int a = 1; a <= 3; ++a) {
            left_pauli_env<T, CS>(A, a, E, Dl, Dr, lane);
            __syncwarp();
            single_j[a - 1] = dot_re<T, CS>(E, R, Dr, lane) * inv_norm;
            if (row < p - 1)
                for (int b = 0; b < 3; ++b) vert[(a - 1) * 3 + b] = dot_re<T, CS>(E, C + b * MAT, Dr, lane) * inv_norm;
            __syncwarp();
        }
        if (row < p - 1) {
            T* o = outp + (size_t)(nh + j) * 16;
            for (int e = lane; e < 16; e += 32) {
                const int a = e >> 2, b = e & 3;
                T v;
                if (a == 0 && b == 0) v = T(1);
                else if (b == 0) v = single_j[a - 1];
                else if (a == 0) v = single_up[b - 1];
                else v = vert[(a - 1) * 3 + (b - 1)];
                o[e] = v;
            }
        }
        // closings of site j as a right site (R_{j-1} is not needed here)
        prod_MAt<T, CS>(R, A, Z0, Z1, Dl, Dr, lane);
        __syncwarp();
        right_closings<T, CS>(A, Z0, Z1, C, C + MAT, C + 2 * MAT, nullptr, Dl, Dr, lane);
        for (int b = 0; b < 3; ++b) single_up[b] = single_j[b];
        if (c == 0 && row == 0) break;
        // next site to the left: horizontal pair (j-1, j) and the first carry step
        const int k0 = j - 1;
        const int Dl0 = bd[k0];   // bond between k0-1 and k0; Dr of k0 is Dl
        load_site_p<T, CS>(A, sites + (size_t)k0 * 2 * ld * ld, ld, Dl0, Dl, lane);
        __syncwarp();
        if (c > 0) {
            load_mat<T, CS>(R, rg + (size_t)k0 * CHI * CHI, CHI, Dl, lane);
            __syncwarp();
            T single_k[3], hor[9];
            for (int a = 1; a <= 3; ++a) {
                left_pauli_env<T, CS>(A, a, E, Dl0, Dl, lane);
                __syncwarp();
                single_k[a - 1] = dot_re<T, CS>(E, R, Dl, lane) * inv_norm;
                for (int b = 0; b < 3; ++b) hor[(a - 1) * 3 + b] = dot_re<T, CS>(E, C + b * MAT, Dl, lane) * inv_norm;
                __syncwarp();
            }
            T* o = outp + (size_t)(row * (p - 1) + (c - 1)) * 16;
            for (int e = lane; e < 16; e += 32) {
                const int a = e >> 2, b = e & 3;
                T v;
                if (a == 0 && b == 0) v = T(1);
                else if (b == 0) v = single_k[a - 1];
                else if (a == 0) v = single_j[b - 1];
                else v = hor[(a - 1) * 3 + (b - 1)];
                o[e] = v;
            }
        }
        if (row == 0) break;
        // carry C_X, C_Y, C_Z through sites j-1 .. j-p+1
        for (int k = k0; k > j - p; --k) {
            const int Dlk = bd[k], Drk = bd[k + 1];
            if (k != k0) {
                load_site_p<T, CS>(A, sites + (size_t)k * 2 * ld * ld, ld, Dlk, Drk, lane);
                __syncwarp();
            }
            for (int b = 0; b < 3; ++b) {
                cx<T>* Cb = C + b * MAT;
                prod_MAt<T, CS>(Cb, A, Z0, Z1, Dlk, Drk, lane);
                __syncwarp();
                prod_AhZ<T, CS>(A, 0, Z0, 1, Z1, Cb, Dlk, Drk, lane);
                __syncwarp();
            }
        }
    }
}

}  // namespace mpsano
