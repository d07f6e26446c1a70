// Pauli-cache kernels (Sec. II.C, Eq. 5).
//
// The circuit kernels leave every MPS left-canonical with the centre at site n-1,
// so the environment of sites 0..i-1 is the identity; the operator-product ladder
// path (ladder_mpo.cu) does not, and its images (META_LENV) bring left environments
// L_i, contracted into E_a (left_blocks_env).  Two kernels remain:
//
//   renv_kernel   one warp per image: right environments R_j (contraction of sites
//                 j+1..n-1 with their conjugates, bra index first) for j = n-1..0,
//                 R_{j-1} = sum_s conj(A_j^s) R_j A_j^{sT}, and <psi|psi> = R_{-1}.
//
//   pauli_kernel  one warp per (image, grid column c).  The warp walks column c
//                 from the bottom row up.  At a column site j it
//                   - closes the vertical pair (j, j+p) with the closing
//                     matrices C_b carried up from site j+p,
//                   - builds the closings of site j as a right site,
//                       C_b^{(j)} = sum_{s,s'} P_b[s][s'] conj(A_j^s) R_j A_j^{s'T},
//                   - closes the horizontal pair (j-1, j) with them,
//                   - carries them through sites j-1, ..., j-p+1 with
//                       C <- sum_s conj(A^s) C A^{sT}.
//                 A left site i contributes E_a[r][r'] = sum_{l,s,s'} conj(A[l,s,r])
//                 P_a[s][s'] A[l,s',r'] and <P_a (x) P_b> = <E_a, C_b> / <psi|psi>,
//                 <P_a> = <E_a, R_i> / <psi|psi> (elementwise product summed).
//                 The closings are Hermitian and the transfer is complex-linear
//                 and keeps Hermiticity, so C_X and C_Y travel as the single
//                 matrix M = C_X + i C_Y (= 2 G01: X + iY is twice the raising
//                 operator), split back at a closing as C_X = (M + M^H)/2,
//                 C_Y = (M - M^H)/(2i): two carried matrices instead of three.
//
// Every contraction is a small complex GEMM done by a team of UW warps (one
// (image, column) unit per CTA) with a register tile of TM x TN outputs per thread;
// threads take interleaved rows (tm + MT*i) and columns (tn + NT*j) so that the shared-memory reads of a k-step hit distinct banks or
// broadcast.  D x D matrices use row stride CS = CHI + 1; the GEMM scratch S has
// 3*CHI rows of stride ZS = 2*CHI + 1.
#pragma once
#include <type_traits>

#include "common.cuh"
#include "linalg.cuh"

namespace mpsano {

// Smallest right bond at which a half-structured site's split contractions (one
// product per physical index, see times_site_t) beat the dense ones: below it the
// two products of depth D/2 cost more in launch overhead than they save.
constexpr int HALF_SPLIT_MIN = 8;

// HALF: every image of the launch is half-structured (META_HALF), whose contractions
// never need more than 2 CHI rows of S (the dense left blocks of a site with a right
// bond above CHI/2 would; the Pauli kernel checks it), so S shrinks by a third.
template <typename E, int CHI, bool HALF = false>
struct PauliLayout {
    using T = typename elem_traits<E>::scalar;
    static constexpr int CS = CHI + 1;
    static constexpr int MAT = CHI * CS;
    static constexpr int ZS = 2 * CHI + 1;
    static constexpr int SROWS = HALF ? 2 * CHI : 3 * CHI;
    // A (2 MAT), R (1 MAT), C (2 MAT: M = C_X + i C_Y, C_Z), S (SROWS rows x ZS);
    // with diagonal pairs also Cd (2 MAT, the carried closings one site further)
    static constexpr int ELEMS = 5 * MAT + SROWS * ZS;
    static constexpr size_t bytes = sizeof(E) * ELEMS;
    __host__ __device__ static constexpr size_t elems(bool diag) { return ELEMS + (diag ? 2 * MAT : 0); }
    // environment kernel: two site buffers, R, and CHI scratch rows (one transfer;
    // the left-environment chain needs 3 MAT + CHI rows)
    static constexpr size_t env_bytes = sizeof(E) * (5 * MAT + CHI * ZS);
    // plus the cross-warp reduction buffer of a UW-warp team
    __host__ __device__ static constexpr size_t team_bytes(int uw, bool diag = false) {
        return sizeof(E) * elems(diag) + sizeof(T) * 12 * uw;
    }
};

// Register-tile shape for an M x N output (compile-time bounds) computed by NTHR
// threads: MT x NT threads, TM x TN complex accumulators per thread, at most 48
// (float) or 24 (double), or CAPX when given.
template <typename E, int M_HINT, int N_HINT, int NTHR = 32, int CAPX = 0>
struct Tile {
    using T = typename elem_traits<E>::scalar;
    static constexpr int MT = (NTHR == 32) ? ((M_HINT >= 2 * N_HINT) ? 8 : 4)
                                           : ((M_HINT >= 2 * N_HINT) ? 16 : (M_HINT * 2 > N_HINT ? 8 : 4));
    static constexpr int NT = NTHR / MT;
    // register tile cap; products of bonds above 32 (hints above 64) take small tiles
    static constexpr int CAP = CAPX > 0 ? CAPX
                               : (M_HINT > 64 || N_HINT > 64) ? (sizeof(T) == 4 ? 16 : 8) : (sizeof(T) == 4 ? 48 : 24);
    static constexpr int TM0 = (M_HINT + MT - 1) / MT;
    static constexpr int TM = TM0 < 1 ? 1 : (TM0 > CAP ? CAP : TM0);
    static constexpr int TN0 = (N_HINT + NT - 1) / NT;
    static constexpr int TN1 = TN0 < 1 ? 1 : TN0;
    static constexpr int TN = TM * TN1 <= CAP ? TN1 : (CAP / TM < 1 ? 1 : CAP / TM);
};

// out[m][n] = sum_{seg < NSEG} sum_{k < K} opA(Ab[ao(m) + seg*as_seg + k*as])
//                                          * Bb[bo(n) + seg*bs_seg + k*bs]
// (NEG1: segment 1 enters with a minus sign; only with CONJA)
// for m < M, n < N, delivered through store(m, so(n), value); the column offsets
// ao, bo and so are evaluated once per tile row / column.
// KU: unroll factor of the k loop (1 keeps the Pauli kernel's code small enough for
// the instruction cache; the environment kernel, one warp per image, prefers 2).
template <typename E, int MT, int NT, int TM, int TN, int NSEG, bool CONJA, int KU, bool NEG1 = false, class AO,
          class BO, class SO, class ST>
__device__ __forceinline__ void team_gemm(const E* Ab, AO ao, int as, int as_seg,
                                          const E* Bb, BO bo, int bs, int bs_seg,
                                          int M, int N, int K, SO so, ST store, int lane) {
    const int tm = lane / NT, tn = lane % NT;
    for (int m0 = 0; m0 < M; m0 += MT * TM) {
        for (int n0 = 0; n0 < N; n0 += NT * TN) {
            int aoff[TM], boff[TN], soff[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) {
                const int m = m0 + tm + MT * i;
                aoff[i] = ao(m < M ? m : M - 1);
            }
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                const int n = n0 + tn + NT * j;
                boff[j] = bo(n < N ? n : N - 1);
                soff[j] = so(n < N ? n : N - 1);
            }
            E acc[TM][TN];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = ezero<E>();
#pragma unroll
            for (int seg = 0; seg < NSEG; ++seg) {
                const E* As = Ab + seg * as_seg;
                const E* Bs = Bb + seg * bs_seg;
#pragma unroll KU
                for (int k = 0; k < K; ++k) {
                    E a[TM], b[TN];
#pragma unroll
                    for (int i = 0; i < TM; ++i) a[i] = As[aoff[i] + k * as];
#pragma unroll
                    for (int j = 0; j < TN; ++j) b[j] = Bs[boff[j] + k * bs];
#pragma unroll
                    for (int i = 0; i < TM; ++i)
#pragma unroll
                        for (int j = 0; j < TN; ++j) {
                            if (NEG1 && seg == 1) cmac_cj(acc[i][j], -a[i], b[j]);   // segment 1 subtracted
                            else if (CONJA) cmac_cj(acc[i][j], a[i], b[j]);
                            else cmac(acc[i][j], a[i], b[j]);
                        }
                }
            }
#pragma unroll
            for (int i = 0; i < TM; ++i) {
                const int m = m0 + tm + MT * i;
#pragma unroll
                for (int j = 0; j < TN; ++j) {
                    const int n = n0 + tn + NT * j;
                    if (m < M && n < N) store(m, soff[j], acc[i][j]);
                }
            }
        }
    }
}

// S[b*Dr + r][n] = sum_k C_b[r][k] A[n][k]: NB source matrices (Dr x Dr, stride MAT)
// times the transposed site rows n = 2l + s < 2 Dl.
__device__ __forceinline__ void team_sync() { __syncthreads(); }

// half: the site is "half-structured": A[2l+s][r] = 0 unless r lies in half s of the
// right bond (s h <= r < (s+1) h, h = Dr/2), as every site but the last of a ladder
// circuit built as an operator product (the last layer's parity bit is the top bit of
// the right bond and equals the output bit).  The contractions over r then run over
// that half only; the skipped terms are exact zeros, which leave an fma chain
// unchanged, so the result is the same bit for bit at half the work.
template <typename E, int CHI, int NB, int NTHR, int KU = 1>
__device__ __forceinline__ void times_site_t(const E* C, const E* A, E* S, int Dl, int Dr, int lane,
                                             bool half = false) {
    using Lay = PauliLayout<E, CHI>;
    constexpr int CS = Lay::CS, MAT = Lay::MAT, ZS = Lay::ZS;
    if (half) {
        const int h = Dr >> 1;
        using Tl = Tile<E, NB * CHI, CHI, NTHR>;
        for (int s = 0; s < 2; ++s)   // the columns 2l'+s of one physical index
            team_gemm<E, Tl::MT, Tl::NT, Tl::TM, Tl::TN, 1, false, KU>(
                C, [Dr, s, h](int m) { return (m / Dr) * MAT + (m % Dr) * CS + s * h; }, 1, 0,
                A, [s, h](int l) { return (2 * l + s) * CS + s * h; }, 1, 0, NB * Dr, Dl, h,
                [s](int l) { return 2 * l + s; }, [S](int m, int sn, E v) { S[m * ZS + sn] = v; }, lane);
        return;
    }
    using Tl = Tile<E, NB * CHI, 2 * CHI, NTHR>;
    team_gemm<E, Tl::MT, Tl::NT, Tl::TM, Tl::TN, 1, false, KU>(
        C, [Dr](int m) { return (m / Dr) * MAT + (m % Dr) * CS; }, 1, 0,
        A, [](int n) { return n * CS; }, 1, 0, NB * Dr, 2 * Dl, Dr,
        [](int n) { return n; }, [S](int m, int sn, E v) { S[m * ZS + sn] = v; }, lane);
}

// Transfer of NB matrices through a site A (Dl x 2 x Dr), in place:
//   C_b <- sum_s conj(A^s) C_b A^{sT}     (C_b: Dr x Dr in, Dl x Dl out)
// with S[b*Dr + r][2l'+s] = (C_b A^{sT})[r][l'] as the intermediate.
// diag_out: only the two diagonal blocks of the result are needed (its next use is a
// transfer through a half-structured site, which reads nothing else), so the second
// product forms those blocks alone; the rest of C_b is left as it was.
template <typename E, int CHI, int NB, int NTHR, int KU = 1>
__device__ __forceinline__ void transfer(E* C, const E* A, E* S, int Dl, int Dr, int lane,
                                         bool half = false, bool diag_out = false) {
    using Lay = PauliLayout<E, CHI>;
    constexpr int CS = Lay::CS, MAT = Lay::MAT, ZS = Lay::ZS;
    if (half) {
        // A^s touches half s of the right bond only, so the transfer reads only the two
        // diagonal blocks of C_b: S[b Dr + s h + i][2l'+s] = sum_{k<h} C_b[s h + i][s h + k]
        // A[2l'+s][s h + k], i < h (the rows the second product reads)
        const int h = Dr >> 1;
        using Tl = Tile<E, NB * CHI / 2, CHI, NTHR>;
        for (int s = 0; s < 2; ++s)
            team_gemm<E, Tl::MT, Tl::NT, Tl::TM, Tl::TN, 1, false, KU>(
                C, [s, h](int m) { const int b = m / h, i = m - b * h; return b * MAT + (s * h + i) * CS + s * h; }, 1, 0,
                A, [s, h](int l) { return (2 * l + s) * CS + s * h; }, 1, 0, NB * h, Dl, h,
                [s](int l) { return 2 * l + s; },
                [S, s, h, Dr](int m, int sn, E v) {
                    const int b = m / h, i = m - b * h;
                    S[(b * Dr + s * h + i) * ZS + sn] = v;
                }, lane);
    } else {
        times_site_t<E, CHI, NB, NTHR, KU>(C, A, S, Dl, Dr, lane);
    }
    team_sync();
    // segment s: r over half s of the right bond when the site is half-structured
    const int K = half ? Dr >> 1 : Dr;
    const int h = half ? Dr >> 1 : 0;
    if (diag_out) {
        const int g = Dl >> 1;
        using Tl = Tile<E, CHI / 2, NB * CHI / 2, NTHR>;
        for (int q = 0; q < 2; ++q)   // rows and columns l, l' in half q of the left bond
            team_gemm<E, Tl::MT, Tl::NT, Tl::TM, Tl::TN, 2, true, KU>(
                A, [q, g](int i) { return 2 * (q * g + i) * CS; }, 1, CS + h,
                S, [Dr, q, g](int nn) { const int b = nn / g, i = nn - b * g; return b * Dr * ZS + 2 * (q * g + i); },
                ZS, 1 + h * ZS, g, NB * g, K,
                [q, g](int nn) { const int b = nn / g, i = nn - b * g; return b * MAT + q * g + i; },
                [C, q, g](int i, int sn, E v) { C[(q * g + i) * CS + sn] = v; }, lane);
    } else {
        using Tl = Tile<E, CHI, NB * CHI, NTHR>;
        team_gemm<E, Tl::MT, Tl::NT, Tl::TM, Tl::TN, 2, true, KU>(
            A, [](int l) { return 2 * l * CS; }, 1, CS + h,
            S, [Dl, Dr](int n) { return (n / Dl) * Dr * ZS + 2 * (n % Dl); }, ZS, 1 + h * ZS, Dl, NB * Dl, K,
            [Dl](int n) { return (n / Dl) * MAT + (n % Dl); },
            [C](int l, int sn, E v) { C[l * CS + sn] = v; }, lane);
    }
    team_sync();
}

// F[m][n] = sum_l conj(A[2l+s_m][r_m]) A[2l+s_n][r_n], m = s_m*Dr + r_m, n = s_n*Dr + r_n:
// the four physical blocks F_{ss'} of a left site, into S rows CHI .. CHI + 2 Dr.
// half (a half-structured site, see times_site_t): F_ss'[r][r'] vanishes unless r is
// in half s and r' in half s', so one Dr x Dr matrix F'[r][r'] = F_{s(r) s(r')}[r][r']
// (s(r) = r >= Dr/2) holds every nonzero value, at a quarter of the work.
template <typename E, int CHI, int NTHR>
__device__ __forceinline__ void left_blocks(const E* A, E* S, int Dl, int Dr, int lane, bool half = false) {
    using Lay = PauliLayout<E, CHI>;
    constexpr int CS = Lay::CS, ZS = Lay::ZS;
    E* F = S + CHI * ZS;
    if (half) {
        const int h = Dr >> 1;
        auto off = [h](int r) { return (r >= h ? CS : 0) + r; };
        using Tl = Tile<E, CHI, CHI, NTHR>;
        team_gemm<E, Tl::MT, Tl::NT, Tl::TM, Tl::TN, 1, true, 1>(
            A, off, 2 * CS, 0, A, off, 2 * CS, 0, Dr, Dr, Dl,
            [](int n) { return n; }, [F](int m, int sn, E v) { F[m * ZS + sn] = v; }, lane);
        return;
    }
    using Tl = Tile<E, 2 * CHI, 2 * CHI, NTHR>;
    auto off = [Dr](int m) { return (m / Dr) * CS + (m % Dr); };
    team_gemm<E, Tl::MT, Tl::NT, Tl::TM, Tl::TN, 1, true, 1>(
        A, off, 2 * CS, 0, A, off, 2 * CS, 0, 2 * Dr, 2 * Dr, Dl,
        [](int n) { return n; }, [F](int m, int sn, E v) { F[m * ZS + sn] = v; }, lane);
}

// The same blocks with a left environment L (Dl x Dl, row stride LS: CHI as stored in
// global memory, or a shared-memory copy; NULL: the identity, left_blocks):
// F[m][n] = sum_{l,l'} conj(A[2l+s_m][r_m]) L[l][l'] A[2l'+s_n][r_n], through
// T[l][s Dr + r] = sum_l' L[l][l'] A[2l'+s][r] in S rows 0 .. Dl.
template <typename E, int CHI, int NTHR, int LS = CHI>
__device__ __forceinline__ void left_blocks_env(const E* A, const E* Lg, E* S, int Dl, int Dr,
                                                int lane, bool half = false) {
    if (!Lg) {
        left_blocks<E, CHI, NTHR>(A, S, Dl, Dr, lane, half);
        return;
    }
    using Lay = PauliLayout<E, CHI>;
    constexpr int CS = Lay::CS, ZS = Lay::ZS;
    if (half) {   // compact F' as in left_blocks, through T'[l][r'] = sum_l' L[l][l'] A[2l'+s(r')][r']
        const int h = Dr >> 1;
        auto off = [h](int r) { return (r >= h ? CS : 0) + r; };
        {
            using Tl = Tile<E, CHI, CHI, NTHR>;
            team_gemm<E, Tl::MT, Tl::NT, Tl::TM, Tl::TN, 1, false, 1>(
                Lg, [](int l) { return l * LS; }, 1, 0, A, off, 2 * CS, 0, Dl, Dr, Dl,
                [](int nn) { return nn; }, [S](int l, int sn, E v) { S[l * ZS + sn] = v; }, lane);
        }
        team_sync();
        E* F = S + CHI * ZS;
        using Tl = Tile<E, CHI, CHI, NTHR>;
        team_gemm<E, Tl::MT, Tl::NT, Tl::TM, Tl::TN, 1, true, 1>(
            A, off, 2 * CS, 0, S, [](int nn) { return nn; }, ZS, 0, Dr, Dr, Dl,
            [](int nn) { return nn; }, [F](int m, int sn, E v) { F[m * ZS + sn] = v; }, lane);
        return;
    }
    {
        using Tl = Tile<E, CHI, 2 * CHI, NTHR>;
        team_gemm<E, Tl::MT, Tl::NT, Tl::TM, Tl::TN, 1, false, 1>(
            Lg, [](int l) { return l * LS; }, 1, 0, A, [Dr](int nn) { return (nn / Dr) * CS + (nn % Dr); }, 2 * CS, 0,
            Dl, 2 * Dr, Dl, [](int nn) { return nn; }, [S](int l, int sn, E v) { S[l * ZS + sn] = v; }, lane);
    }
    team_sync();
    E* F = S + CHI * ZS;
    using Tl = Tile<E, 2 * CHI, 2 * CHI, NTHR>;
    team_gemm<E, Tl::MT, Tl::NT, Tl::TM, Tl::TN, 1, true, 1>(
        A, [Dr](int m) { return (m / Dr) * CS + (m % Dr); }, 2 * CS, 0, S, [](int nn) { return nn; }, ZS, 0,
        2 * Dr, 2 * Dr, Dl, [](int nn) { return nn; }, [F](int m, int sn, E v) { F[m * ZS + sn] = v; }, lane);
}

// <E_a, Y> for a = X, Y, Z (from the blocks F_{ss'} at F, row stride ZS) and Y in
// {C_X, C_Y, C_Z, R}: out[4(a-1) + y], with C_X, C_Y unpacked from M = C[0] and
// C_Z = C[MAT].  C may be null (then only the R column is formed).  One warp (lane < 32)
// forms every sum in a fixed order, so the bits of the result depend on neither the team
// size nor on which warp runs it; every lane receives the sums.
template <typename E, int CHI>
__device__ __forceinline__ void left_dots_warp(const E* F, int ZS, const E* C, const E* R, int D,
                                               typename elem_traits<E>::scalar* out, int lane,
                                               bool half = false) {
    using T = typename elem_traits<E>::scalar;
    using Lay = PauliLayout<E, CHI>;
    constexpr int CS = Lay::CS, MAT = Lay::MAT;
    const int h = D >> 1;
    T acc[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) acc[i] = T(0);
    team_for_2d<32, 4>(D, D, lane, [&](int r, int rp) {
      if constexpr (elem_traits<E>::real) {
        // a real state (no half-structured sites): E_X, E_Z, C_X, C_Z and R are real,
        // E_Y = i (F10 - F01) and C_Y = -i (M - M^T) / 2 imaginary, so the entries with
        // one Y vanish and <E_Y, C_Y> = sum (F10 - F01) (M - M^T) / 2
        const E f00 = F[r * ZS + rp], f01 = F[r * ZS + D + rp];
        const E f10 = F[(D + r) * ZS + rp], f11 = F[(D + r) * ZS + D + rp];
        const E ex = f01 + f10, ey = f10 - f01, ez = f00 - f11;
        const E rr = R[r * CS + rp];
        acc[3] = fma(ex, rr, acc[3]);
        acc[11] = fma(ez, rr, acc[11]);
        if (C) {
            const E m1 = C[r * CS + rp], m2 = C[rp * CS + r];
            const E yx = T(0.5) * (m1 + m2), yy = T(0.5) * (m1 - m2), yz = C[MAT + r * CS + rp];
            acc[0] = fma(ex, yx, acc[0]);
            acc[2] = fma(ex, yz, acc[2]);
            acc[5] = fma(ey, yy, acc[5]);
            acc[8] = fma(ez, yx, acc[8]);
            acc[10] = fma(ez, yz, acc[10]);
        }
      } else {
        E e[3];
        if (half) {
            // compact F' (left_blocks): the one nonzero block at (r, r') is F_{s s'}
            // with s = r >= h, s' = r' >= h; the same values as the full form
            const E f = F[r * ZS + rp], z = ezero<E>();
            const int s0 = r >= h, s1 = rp >= h;
            e[0] = s0 != s1 ? f : z;                                                   // X
            e[1] = s0 == s1 ? z : (s0 ? mk<T>(-f.im, f.re) : mk<T>(f.im, -f.re));      // Y
            e[2] = s0 != s1 ? z : (s0 ? mk<T>(-f.re, -f.im) : f);                      // Z
        } else {
            const E f00 = F[r * ZS + rp], f01 = F[r * ZS + D + rp];
            const E f10 = F[(D + r) * ZS + rp], f11 = F[(D + r) * ZS + D + rp];
            e[0] = f01 + f10;                                     // X
            e[1] = mk<T>(f01.im - f10.im, f10.re - f01.re);       // Y: i (F10 - F01)
            e[2] = f00 - f11;                                     // Z
        }
        E y[4];
        y[3] = R[r * CS + rp];
        if (C) {
            const E m1 = C[r * CS + rp], m2 = conj(C[rp * CS + r]);
            const E u = m1 + m2, v = m1 - m2;
            y[0] = mk<T>(T(0.5) * u.re, T(0.5) * u.im);       // (M + M^H) / 2
            y[1] = mk<T>(T(0.5) * v.im, T(-0.5) * v.re);      // (M - M^H) / (2i)
            y[2] = C[MAT + r * CS + rp];
        }
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b)
                if (C || b == 3) acc[4 * a + b] = fma(-e[a].im, y[b].im, fma(e[a].re, y[b].re, acc[4 * a + b]));
      }
    });
#pragma unroll
    for (int i = 0; i < 12; ++i) out[i] = warp_sum(acc[i]);
}

// left_dots_warp run by warp 0 of a team, the sums handed to the other warps through red.
template <typename E, int CHI, int NTHR>
__device__ __forceinline__ void left_dots(const E* S, const E* C, const E* R, int D,
                                          typename elem_traits<E>::scalar* out,
                                          typename elem_traits<E>::scalar* red, int lane, bool half = false) {
    if (lane < 32) {
        left_dots_warp<E, CHI>(S + CHI * PauliLayout<E, CHI>::ZS, PauliLayout<E, CHI>::ZS, C, R, D, out, lane, half);
        if (NTHR > 32 && lane == 0)
#pragma unroll
            for (int i = 0; i < 12; ++i) red[i] = out[i];
    }
    if (NTHR > 32) {
        team_sync();
        if (lane >= 32)
#pragma unroll
            for (int i = 0; i < 12; ++i) out[i] = red[i];
        team_sync();
    }
}

// Closings of a right site A (Dl x 2 x Dr) with right environment R:
//   G[2l+s][2l'+s'] = sum_r conj(A[2l+s][r]) (R A^{s'T})[r][l'],
//   C_X = G01 + G10, C_Y = i (G10 - G01), C_Z = G00 - G11  (Dl x Dl each); into C go
//   M = C_X + i C_Y = 2 G01 and C_Z, each formed directly from S = R A^T (G itself is
//   never stored): M from the even rows of A and the odd columns of S, C_Z as one
//   two-segment product, the odd segment subtracted.
template <typename E, int CHI, int NTHR>
__device__ __forceinline__ void right_closings(const E* A, const E* R, E* C, E* S,
                                               int Dl, int Dr, int lane, bool half = false) {
    using Lay = PauliLayout<E, CHI>;
    constexpr int CS = Lay::CS, MAT = Lay::MAT, ZS = Lay::ZS;
    times_site_t<E, CHI, 1, NTHR>(R, A, S, Dl, Dr, lane, half);   // S[r][n] = (R A^T)[r][n]
    team_sync();
    // rows 2l+s contract r over half s only when the site is half-structured
    const int K = half ? Dr >> 1 : Dr;
    const int h = half ? Dr >> 1 : 0;
    using Tl = Tile<E, CHI, CHI, NTHR>;
    team_gemm<E, Tl::MT, Tl::NT, Tl::TM, Tl::TN, 1, true, 1>(
        A, [](int l) { return 2 * l * CS; }, 1, 0, S, [](int n) { return 2 * n + 1; }, ZS, 0, Dl, Dl, K,
        [](int n) { return n; }, [C](int l, int sn, E v) { C[l * CS + sn] = v + v; }, lane);
    team_gemm<E, Tl::MT, Tl::NT, Tl::TM, Tl::TN, 2, true, 1, true>(
        A, [](int l) { return 2 * l * CS; }, 1, CS + h, S, [](int n) { return 2 * n; }, ZS, 1 + h * ZS, Dl, Dl, K,
        [](int n) { return n; }, [C](int l, int sn, E v) { C[MAT + l * CS + sn] = v; }, lane);
    team_sync();
}

template <typename E, int CS, int NTHR = 32>
__device__ __forceinline__ void load_site_p(E* dst, const cx<typename elem_traits<E>::scalar>* src, int ld, int Dl,
                                            int Dr, int lane) {
    team_for_2d<NTHR, 4>(2 * Dl, Dr, lane, [&](int row, int r) { dst[row * CS + r] = to_elem<E>(src[row * ld + r]); });
}

template <typename E, int CS, int NTHR = 32>
__device__ __forceinline__ void load_mat(E* dst, const E* src, int ld, int D, int lane) {
    team_for_2d<NTHR, 4>(D, D, lane, [&](int r, int c) { dst[r * CS + c] = src[r * ld + c]; });
}

// Asynchronous global -> shared copy of one complex element (cp.async, 8 or 16 B).
template <typename T>
__device__ __forceinline__ void cp_async_elem(cx<T>* dst, const cx<T>* src) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
    if constexpr (sizeof(cx<T>) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
// The real part alone (4 or 8 B) into a real element.
template <typename T>
__device__ __forceinline__ void cp_async_re(T* dst, const cx<T>* src) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(&src->re) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(&src->re) : "memory");
}
// An element of E from global memory of the same type (4, 8 or 16 B).
template <typename E>
__device__ __forceinline__ void cp_async_same(E* dst, const E* src) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
    if constexpr (sizeof(E) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
    else if constexpr (sizeof(E) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Left environments of one image (a warp): L_0 = 1 and L_{k+1}[r][r'] =
// sum_{l,l',s} conj(A_k[l][s][r]) L_k[l][l'] A_k[l'][s][r'], stored like the right
// environments (L_k, D_k x D_k, at k * CHI * CHI of the image's block).  At a
// half-structured site the product formed on the way is the compact left block
// F'_k[r][r'] = sum_{l,l'} conj(A_k[l][s(r)][r]) L_k[l][l'] A_k[l'][s(r')][r'] of the
// Pauli kernels (left_blocks_env), of which L_{k+1} keeps the diagonal blocks; with fg
// it is stored too (at k * CHI * CHI of fg).  ASYNC: site k+1 arrives by cp.async in a
// second buffer while site k is contracted (shared-memory workspace only).  A team of
// NTHR threads (lane = its thread index) runs the chain.
template <typename E, int CHI, bool ASYNC = false, int NTHR = 32>
__device__ __forceinline__ void lenv_image(const ImageMeta& mt,
                                           const cx<typename elem_traits<E>::scalar>* __restrict__ arena,
                                           const int32_t* __restrict__ bonds, E* lg, E* fg, E* base,
                                           int lane) {
    using Lay = PauliLayout<E, CHI>;
    constexpr int CS = Lay::CS, MAT = Lay::MAT, ZS = Lay::ZS;
    E* const A0 = base;                      // 2 MAT each (the second within env_bytes)
    E* const A1 = base + 3 * MAT + CHI * ZS;
    E* Lm = base + 2 * MAT;  // MAT
    E* S = base + 3 * MAT;   // CHI rows of ZS
    const int n = mt.n, ld = mt.ld;
    const int32_t* bd = bonds + mt.bond_off;
    const cx<typename elem_traits<E>::scalar>* sites = arena + mt.site_off;
    const bool half_img = (mt.flags & META_HALF) != 0;
    // site k is half-structured: row 2l+s of A_k is zero outside column half s
    auto half_site = [=](int k) { return half_img && k < n - 1 && bd[k + 1] >= 2; };
    auto prefetch = [=](int k, E* dstA) {
        const auto* src = sites + (size_t)k * 2 * ld * ld;
        team_for_2d<NTHR, 4>(2 * bd[k], bd[k + 1], lane, [=](int r, int c) {
            if constexpr (elem_traits<E>::real) cp_async_re(dstA + r * CS + c, src + r * ld + c);
            else cp_async_same(dstA + r * CS + c, src + r * ld + c);
        });
        cp_async_commit();
    };
    if (lane == 0) Lm[0] = eone<E>();
    if (ASYNC && n > 0) prefetch(0, A0);
    tsync<NTHR>();
    for (int k = 0; k < n; ++k) {
        const int Dl = bd[k], Dr = bd[k + 1];
        E* dst = lg + (size_t)k * CHI * CHI;
        E* A = (ASYNC && (k & 1)) ? A1 : A0;
        // L_k (with fg, a half-structured site keeps F'_k instead, which is what is read there)
        if (!(fg && half_site(k)))
            team_for_2d<NTHR, 4>(Dl, Dl, lane, [&](int r, int c) { dst[r * CHI + c] = Lm[r * CS + c]; });
        if constexpr (ASYNC) {
            // site k has landed for every thread, and the buffer of site k-1 (read before
            // the last barrier) takes site k+1
            cp_async_wait_all();
            tsync<NTHR>();
            if (k + 1 < n) prefetch(k + 1, (k & 1) ? A0 : A1);
        } else {
            load_site_p<E, CS, NTHR>(A, sites + (size_t)k * 2 * ld * ld, ld, Dl, Dr, lane);
            tsync<NTHR>();
        }
        if (half_site(k)) {
            // half-structured site: L A is needed only at (s, r) with r in half s
            // (T'[l][r] = sum_l' L[l][l'] A[2l'+s(r)][r]), and L_{k+1} is block diagonal
            // over the two halves (zero between them, as the full form gives)
            const int h = Dr >> 1;
            auto off = [h](int r) { return (r >= h ? CS : 0) + r; };
            if (k >= 1 && Dl >= 2) {
                // the previous site was half-structured too, so L_k is block diagonal over
                // the halves of its bond: row l of T' sums over the l' of its own half only
                // (the zero block adds nothing); one half of the team per half of the rows
                constexpr int HT = NTHR >= 64 ? NTHR / 2 : NTHR;
                using Tl = Tile<E, CHI / 2, CHI, HT>;
                const int g = Dl >> 1;
                for (int q = NTHR >= 64 ? lane / HT : 0; q < 2; q += NTHR >= 64 ? 2 : 1) {
                    const int q0 = q ? g : 0, Mq = q ? Dl - g : g;
                    team_gemm<E, Tl::MT, Tl::NT, Tl::TM, Tl::TN, 1, false, 1>(
                        Lm, [q0](int l) { return (q0 + l) * CS + q0; }, 1, 0, A,
                        [off, q0](int r) { return off(r) + q0 * 2 * CS; }, 2 * CS, 0, Mq, Dr, Mq,
                        [](int nn) { return nn; }, [S, q0](int l, int sn, E v) { S[(q0 + l) * ZS + sn] = v; },
                        lane & (HT - 1));
                }
            } else {
                using Tl = Tile<E, CHI, CHI, NTHR>;
                team_gemm<E, Tl::MT, Tl::NT, Tl::TM, Tl::TN, 1, false, 1>(
                    Lm, [](int l) { return l * CS; }, 1, 0, A, off, 2 * CS, 0, Dl, Dr, Dl,
                    [](int nn) { return nn; }, [S](int l, int sn, E v) { S[l * ZS + sn] = v; }, lane);
            }
            tsync<NTHR>();
            {
                using Tl = Tile<E, CHI, CHI, NTHR>;
                E* fk = fg ? fg + (size_t)k * CHI * CHI : nullptr;
                team_gemm<E, Tl::MT, Tl::NT, Tl::TM, Tl::TN, 1, true, 1>(
                    A, off, 2 * CS, 0, S, [](int nn) { return nn; }, ZS, 0, Dr, Dr, Dl, [](int nn) { return nn; },
                    [Lm, h, fk](int r, int sn, E v) {
                        Lm[r * CS + sn] = (r >= h) == (sn >= h) ? v : ezero<E>();
                        if (fk) fk[r * CHI + sn] = v;
                    }, lane);
            }
            tsync<NTHR>();
            continue;
        }
        // S[l][s Dr + r] = sum_l' L[l][l'] A[2l'+s][r]
        {
            using Tl = Tile<E, CHI, 2 * CHI, NTHR>;
            team_gemm<E, Tl::MT, Tl::NT, Tl::TM, Tl::TN, 1, false, 1>(
                Lm, [](int l) { return l * CS; }, 1, 0, A, [Dr](int nn) { return (nn / Dr) * CS + (nn % Dr); }, 2 * CS, 0,
                Dl, 2 * Dr, Dl, [](int nn) { return nn; }, [S](int l, int sn, E v) { S[l * ZS + sn] = v; }, lane);
        }
        tsync<NTHR>();
        // L'[r][r'] = sum_{l,s} conj(A[2l+s][r]) S[l][s Dr + r']
        {
            using Tl = Tile<E, CHI, CHI, NTHR>;
            team_gemm<E, Tl::MT, Tl::NT, Tl::TM, Tl::TN, 2, true, 1>(
                A, [](int r) { return r; }, 2 * CS, CS, S, [](int nn) { return nn; }, ZS, Dr, Dr, Dr, Dl,
                [](int nn) { return nn; }, [Lm](int r, int sn, E v) { Lm[r * CS + sn] = v; }, lane);
        }
        tsync<NTHR>();
    }
}

// CTA i < n_images (after first_block is added): the right environments of image i;
// with lenv, CTA n_images + i:
// the left environments of image i when it is flagged META_LENV (the two chains are
// independent and latency-bound, so one launch runs them side by side), and with
// fblk the compact left blocks of its half-structured sites (lenv_image).
// GMEM (bonds above 32): the workspace is a slice of global memory, env_bytes per CTA.
// REAL: a real state (every amplitude real): real elements, environments stored as
// reals in the same buffers.
template <typename T, int CHI, bool GMEM = false, bool REAL = false>
__global__ void __launch_bounds__(32) renv_kernel(const ImageMeta* __restrict__ meta, int n_images,
                                                   const cx<T>* __restrict__ arena,
                                                   const int32_t* __restrict__ bonds,
                                                   cx<T>* __restrict__ renv_c, int64_t renv_stride,
                                                   cx<T>* __restrict__ lenv_c,
                                                   T* __restrict__ norm_out, unsigned char* __restrict__ gws,
                                                   int first_block, cx<T>* __restrict__ fblk_c) {
    using E = std::conditional_t<REAL, T, cx<T>>;
    using Lay = PauliLayout<E, CHI>;
    constexpr int CS = Lay::CS, MAT = Lay::MAT;
    E* renv = reinterpret_cast<E*>(renv_c);
    E* lenv = reinterpret_cast<E*>(lenv_c);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* raw = GMEM ? gws + (size_t)blockIdx.x * Lay::env_bytes : smem_raw;
    // one warp per image and one image per CTA (block-wide syncs are warp syncs);
    // first_block = n_images: the left environments alone
    const int lane = threadIdx.x;
    const int bid = blockIdx.x + first_block;
    if (bid >= n_images) {
        const int li = bid - n_images;
        if (!lenv || li >= n_images) return;
        const ImageMeta ml = meta[li];
        E* fg = fblk_c ? reinterpret_cast<E*>(fblk_c) + (size_t)li * renv_stride : nullptr;
        if (ml.flags & META_LENV)
            lenv_image<E, CHI, !GMEM>(ml, arena, bonds, lenv + (size_t)li * renv_stride, fg,
                                      reinterpret_cast<E*>(raw), lane);
        return;
    }
    const int img = bid;
    E* base = reinterpret_cast<E*>(raw);
    const bool half_img = (meta[img].flags & META_HALF) != 0;
    E* Abuf[2] = {base, base + 3 * MAT};   // site j in one, site j-1 arriving in the other
    E* R = base + 2 * MAT;
    E* S = base + 5 * MAT;                 // CHI rows of ZS (env_bytes)
    const ImageMeta mt = meta[img];
    const int n = mt.n, ld = mt.ld;
    const int32_t* bd = bonds + mt.bond_off;
    const cx<T>* sites = arena + mt.site_off;
    E* rg = renv + (size_t)img * renv_stride;
    // site j -> dstA with cp.async, so that its load overlaps the transfer through site j+1
    // (plain loads into a global workspace, or converting to real elements)
    auto prefetch = [&](int j, E* dstA) {
        const int Dl = bd[j], Dr = bd[j + 1];
        const cx<T>* src = sites + (size_t)j * 2 * ld * ld;
        if constexpr (GMEM || REAL) {
            team_for_2d<32, 4>(2 * Dl, Dr, lane, [&](int row, int r) { dstA[row * CS + r] = to_elem<E>(src[row * ld + r]); });
        } else {
            team_for_2d<32, 4>(2 * Dl, Dr, lane, [&](int row, int r) { cp_async_elem(dstA + row * CS + r, src + row * ld + r); });
            cp_async_commit();
        }
    };
    if (lane == 0) R[0] = eone<E>();
    if (n > 0) prefetch(n - 1, Abuf[0]);
    int cb = 0;
    for (int j = n - 1; j >= 0; --j) {
        const int Dl = bd[j], Dr = bd[j + 1];
        E* dst = rg + (size_t)j * CHI * CHI;
        team_for_2d<32, 4>(Dr, Dr, lane, [&](int r, int c) { dst[r * CHI + c] = R[r * CS + c]; });
        if constexpr (!(GMEM || REAL)) cp_async_wait_all();
        __syncwarp();
        if (j > 0) prefetch(j - 1, Abuf[cb ^ 1]);
        transfer<E, CHI, 1, 32, 2>(R, Abuf[cb], S, Dl, Dr, lane, half_img && j < n - 1 && Dr >= HALF_SPLIT_MIN);
        cb ^= 1;
    }
    if (lane == 0) norm_out[img] = ereal(R[0]);
}

// One (image, column) unit of the Pauli kernel, worked on by the CTA's UW warps with
// its workspace at smem_raw.
template <typename T, int CHI, int UW, bool DIAG, bool REAL, bool HALF = false>
__device__ __forceinline__ void pauli_unit(int unit, unsigned char* smem_raw, const ImageMeta* __restrict__ meta,
                                           const int32_t* __restrict__ unit_image,
                                           const cx<T>* __restrict__ arena, const int32_t* __restrict__ bonds,
                                           const cx<T>* __restrict__ renv_c, int64_t renv_stride,
                                           const cx<T>* __restrict__ lenv_c, const T* __restrict__ norms,
                                           T* __restrict__ out, int* status) {
    using E = std::conditional_t<REAL, T, cx<T>>;
    using Lay = PauliLayout<E, CHI, HALF>;
    const E* renv = reinterpret_cast<const E*>(renv_c);
    const E* lenv = reinterpret_cast<const E*>(lenv_c);
    constexpr int CS = Lay::CS, MAT = Lay::MAT;
    constexpr int NTHR = 32 * UW;
    constexpr bool diag = DIAG;   // both diagonal pair sets as well (a separate instantiation)
    const int lane = threadIdx.x;
    const int img = unit_image[2 * unit], c = unit_image[2 * unit + 1];
    E* base = reinterpret_cast<E*>(smem_raw);
    T* red = reinterpret_cast<T*>(base + Lay::ELEMS + (diag ? 2 * MAT : 0));
    E* A = base;               // 2 MAT
    E* R = base + 2 * MAT;
    E* C = base + 3 * MAT;     // 2 MAT: M = C_X + i C_Y, C_Z
    E* S = base + 5 * MAT;     // GEMM scratch
    E* Cd = base + Lay::ELEMS; // 2 MAT (diagonal pairs only)
    const ImageMeta mt = meta[img];
    const int p = mt.p, ld = mt.ld;
    const int32_t* bd = bonds + mt.bond_off;
    const cx<T>* sites = arena + mt.site_off;
    const E* rg = renv + (size_t)img * renv_stride;
    // left environments (images whose MPS is not left-canonical), same layout as renv
    const E* lgb = (lenv && (mt.flags & META_LENV)) ? lenv + (size_t)img * renv_stride : nullptr;
    auto lenv_of = [lgb](int i) -> const E* { return lgb ? lgb + (size_t)i * CHI * CHI : nullptr; };
    // half-structured sites (META_HALF): every site but the last.  half_at: the compact
    // left blocks (one product either way); half_tr: the contractions that split into
    // one product per physical index, from bond HALF_SPLIT_MIN on
    const bool half_img = (mt.flags & META_HALF) != 0;
    if constexpr (HALF) {
        // the reduced scratch holds only half-structured images (the host launches this
        // variant when every image is one)
        if (!half_img) {
            if (threadIdx.x == 0) raise_status(status, DEV_BAD_SHAPE);
            return;
        }
    }
    auto half_at = [half_img, &mt, bd](int i) { return half_img && i < mt.n - 1 && bd[i + 1] >= 2; };
    auto half_tr = [half_img, &mt, bd](int i) { return half_img && i < mt.n - 1 && bd[i + 1] >= HALF_SPLIT_MIN; };
    const T inv_norm = T(1) / norms[img];
    T* outp = out + (size_t)(diag ? mt.pair_off_d : mt.pair_off) * 16;
    const int nh = p * (p - 1);                  // horizontal pairs come first, then vertical,
    const int base_dd = 2 * p * (p - 1);         // then (r,c)-(r+1,c+1),
    const int base_da = base_dd + (p - 1) * (p - 1);   // then (r,c+1)-(r+1,c)
    auto write_pair = [&](int q, const T* sa, const T* sb, const T* dv) {
        // sa: <P_a> of the lower-index site, sb: <P_b> of the other, dv: the 9 two-body sums
        if (lane < 16) {
            const int a = lane >> 2, b = lane & 3;
            T v;
            if (a == 0 && b == 0) v = T(1);
            else if (b == 0) v = sa[a - 1];
            else if (a == 0) v = sb[b - 1];
            else v = dv[4 * (a - 1) + (b - 1)] * inv_norm;
            outp[(size_t)q * 16 + lane] = v;
        }
    };

    T single_up[3] = {T(0), T(0), T(0)};   // <P_b> of the site that created the carried C
    T d[12], dd[12];
    for (int row = p - 1; row >= 0; --row) {
        const int j = row * p + c;
        const int Dl = bd[j], Dr = bd[j + 1];
        load_site_p<E, CS, NTHR>(A, sites + (size_t)j * 2 * ld * ld, ld, Dl, Dr, lane);
        load_mat<E, CS, NTHR>(R, rg + (size_t)j * CHI * CHI, CHI, Dr, lane);
        team_sync();
        // site j as the left site: single-site terms and the vertical pair (j, j+p)
        left_blocks_env<E, CHI, NTHR>(A, lenv_of(j), S, Dl, Dr, lane, half_at(j));
        team_sync();
        left_dots<E, CHI, NTHR>(S, row < p - 1 ? C : nullptr, R, Dr, d, red, lane, half_at(j));
        T single_j[3];
        for (int a = 0; a < 3; ++a) single_j[a] = d[4 * a + 3] * inv_norm;
        if (row < p - 1) write_pair(nh + j, single_j, single_up, d);
        team_sync();
        // diagonal (row, c-1)-(row+1, c): the closings carried from j+p, one site further
        const bool has_dd = diag && row < p - 1 && c >= 1;
        if (has_dd) {
            for (int o = lane; o < 2 * MAT; o += NTHR) Cd[o] = C[o];
            team_sync();
            transfer<E, CHI, 2, NTHR>(Cd, A, S, Dl, Dr, lane, half_tr(j));
        }
        // closings of site j as a right site
        right_closings<E, CHI, NTHR>(A, R, C, S, Dl, Dr, lane, half_tr(j));
        T single_prev[3];
        for (int b = 0; b < 3; ++b) { single_prev[b] = single_up[b]; single_up[b] = single_j[b]; }
        if (c == 0 && row == 0) break;
        // next site to the left: horizontal pair (j-1, j) and the first carry step
        const int k0 = j - 1;
        const int Dl0 = bd[k0];   // left bond of site k0; its right bond is Dl
        load_site_p<E, CS, NTHR>(A, sites + (size_t)k0 * 2 * ld * ld, ld, Dl0, Dl, lane);
        team_sync();
        if (c > 0) {
            load_mat<E, CS, NTHR>(R, rg + (size_t)k0 * CHI * CHI, CHI, Dl, lane);
            team_sync();
            left_blocks_env<E, CHI, NTHR>(A, lenv_of(k0), S, Dl0, Dl, lane, half_at(k0));
            team_sync();
            left_dots<E, CHI, NTHR>(S, C, R, Dl, d, red, lane, half_at(k0));
            T single_k[3];
            for (int a = 0; a < 3; ++a) single_k[a] = d[4 * a + 3] * inv_norm;
            write_pair(row * (p - 1) + (c - 1), single_k, single_j, d);
            if (has_dd) {
                left_dots<E, CHI, NTHR>(S, Cd, R, Dl, dd, red, lane, half_at(k0));
                write_pair(base_dd + row * (p - 1) + (c - 1), single_k, single_prev, dd);
            }
            team_sync();
        }
        if (row == 0) break;
        // carry M and C_Z through sites j-1 .. j-p+1
        for (int k = k0; k > j - p; --k) {
            const int Dlk = bd[k], Drk = bd[k + 1];
            if (k != k0) {
                load_site_p<E, CS, NTHR>(A, sites + (size_t)k * 2 * ld * ld, ld, Dlk, Drk, lane);
                team_sync();
            }
            if (diag && k == j - p + 1 && c <= p - 2) {
                // anti-diagonal (row-1, c+1)-(row, c): site k is the left site
                load_mat<E, CS, NTHR>(R, rg + (size_t)k * CHI * CHI, CHI, Drk, lane);
                team_sync();
                left_blocks_env<E, CHI, NTHR>(A, lenv_of(k), S, Dlk, Drk, lane, half_at(k));
                team_sync();
                left_dots<E, CHI, NTHR>(S, C, R, Drk, dd, red, lane, half_at(k));
                T single_k[3];
                for (int a = 0; a < 3; ++a) single_k[a] = dd[4 * a + 3] * inv_norm;
                write_pair(base_da + (row - 1) * (p - 1) + c, single_k, single_j, dd);
                team_sync();
            }
            // the last transfer brings the closings to site j - p, where they close in full;
            // before it, their next use is the transfer through site k - 1 (H+V pairs)
            const bool dout = !diag && k > j - p + 1 && half_tr(k - 1);
            transfer<E, CHI, 2, NTHR>(C, A, S, Dlk, Drk, lane, half_tr(k), dout);
        }
    }
}


// One (image, column) unit per CTA (GMEM: bonds above 32, workspace in global memory,
// Lay::team_bytes per CTA, the CTAs stepping through the units).
// Resident CTAs per SM the compiler is asked to fit for the half-structured variant
// (64-thread teams): 10 fit its 19.4 KB of shared memory and 96 registers per thread.
#ifndef PAULI_HALF_MIN_BLOCKS
#define PAULI_HALF_MIN_BLOCKS 10
#endif
template <typename T, int CHI, int UW, bool DIAG, bool GMEM = false, bool REAL = false, bool HALF = false>
__global__ void __launch_bounds__(32 * UW, (UW == 4 ? 4 : (UW == 2 && CHI <= 16) ? (HALF ? PAULI_HALF_MIN_BLOCKS : 9) : 8) / (sizeof(T) == 8 ? 2 : 1)) pauli_kernel(const ImageMeta* __restrict__ meta, int n_units,
                                                    const int32_t* __restrict__ unit_image,
                                                    const cx<T>* __restrict__ arena,
                                                    const int32_t* __restrict__ bonds,
                                                    const cx<T>* __restrict__ renv, int64_t renv_stride,
                                                    const cx<T>* __restrict__ lenv,
                                                    const T* __restrict__ norms, T* __restrict__ out,
                                                    unsigned char* __restrict__ gws, int* status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if constexpr (GMEM) {
        constexpr size_t ws = (PauliLayout<std::conditional_t<REAL, T, cx<T>>, CHI>::team_bytes(UW, DIAG) + 255) &
                              ~size_t(255);
        unsigned char* raw = gws + (size_t)blockIdx.x * ws;
        for (int unit = blockIdx.x; unit < n_units; unit += gridDim.x) {
            pauli_unit<T, CHI, UW, DIAG, REAL>(unit, raw, meta, unit_image, arena, bonds, renv, renv_stride, lenv,
                                               norms, out, status);
            __syncthreads();
        }
    } else {
        if ((int)blockIdx.x >= n_units) return;
        pauli_unit<T, CHI, UW, DIAG, REAL, HALF>(blockIdx.x, smem_raw, meta, unit_image, arena, bonds, renv,
                                                 renv_stride, lenv, norms, out, status);
    }
}

}  // namespace mpsano
