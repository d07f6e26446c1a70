// Small dense linear algebra on shared memory for a team of NTHR threads (one
// warp, or the whole CTA when NTHR > 32): Householder QR, the explicit Q factor,
// and a cyclic Jacobi eigensolver for Hermitian matrices (run by warp 0).
// Matrices are column-major: element (r, c) at A[c * ld + r].
#pragma once
#include "common.cuh"

namespace mpsano {

template <int NTHR>
__device__ __forceinline__ void tsync() {
    if (NTHR == 32) __syncwarp();
    else __syncthreads();
}

// Sum of v over the team; every thread gets the result.  red: NTHR/32 doubles.
template <int NTHR, typename T>
__device__ __forceinline__ T team_sum(T v, double* red, int tid) {
    v = warp_sum(v);
    if (NTHR == 32) return v;
    if ((tid & 31) == 0) red[tid >> 5] = (double)v;
    __syncthreads();
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < NTHR / 32; ++w) s += red[w];
    __syncthreads();
    return (T)s;
}

// Calls f(row, col) for every row < R and col < C, spreading the pairs over the
// NTHR threads without integer division: columns are padded to a power of two cp,
// thread -> (col = tid % cp, first row = tid / cp).
// UNROLL: unroll factor of the row loop.  The circuit kernels keep 1 (their many
// short loops otherwise overflow the instruction cache); load loops that wait on
// global memory use 4.
template <int NTHR, int UNROLL = 1, class F>
__device__ __forceinline__ void team_for_2d(int R, int C, int tid, F f) {
    if (C <= 0 || R <= 0) return;
    const int cp = C <= 1 ? 1 : 1 << (32 - __clz(C - 1));
    if (cp >= NTHR) {
        for (int row = 0; row < R; ++row)
            for (int col = tid; col < C; col += NTHR) f(row, col);
    } else {
        const int shift = __ffs(cp) - 1;
        const int col = tid & (cp - 1);
        const int rstep = NTHR >> shift;
        if (col < C) {
#pragma unroll UNROLL
            for (int row = tid >> shift; row < R; row += rstep) f(row, col);
        }
    }
}

// Calls f(i, j) for every 0 <= i <= j < K (the upper triangle of a K x K matrix),
// K (K + 1) / 2 calls spread evenly over the NTHR threads: t = j (j + 1) / 2 + i.
// (team_for_2d over K x K with the lower half skipped leaves about half of every
// warp's lanes idle, and an FP64 instruction costs its issue slots on the FP64 pipe
// whether or not its lanes are active.)
template <int NTHR, class F>
__device__ __forceinline__ void team_for_upper(int K, int tid, F f) {
    const int total = K * (K + 1) / 2;
    for (int t = tid; t < total; t += NTHR) {
        int j = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
        while (j * (j + 1) / 2 > t) --j;
        while ((j + 1) * (j + 2) / 2 <= t) ++j;
        f(t - j * (j + 1) / 2, j);
    }
}

// Largest power of two G <= 32 with G * nc <= NTHR (at least 1): threads per column
// when nc columns are processed by the team.
template <int NTHR>
__device__ __forceinline__ int threads_per_col(int nc) {
    int G = 32;
    while (G > 1 && G * nc > NTHR) G >>= 1;
    return G;
}

// A(j:M, j+1:N) <- (I - t v v^H) A(j:M, j+1:N), v = [1; A(j+1:M, j)] stored in column j.
// Rows are split over G threads per column; partial dot products are combined with
// xor-shuffles inside each aligned group of G lanes.
template <int NTHR, typename T>
__device__ __forceinline__ void apply_reflector(cx<T>* A, int ld, int M, int N, int j, cx<T> t, int tid) {
    const int nc = N - j - 1;
    if (nc <= 0) return;
    const cx<T>* v = A + j * ld;
    const int G = threads_per_col<NTHR>(nc);
    const int cg = tid / G, g = tid % G;
    const int per_pass = NTHR / G;
    for (int c0 = 0; c0 < nc; c0 += per_pass) {
        const int cc = c0 + cg;
        const bool active = cc < nc;
        cx<T>* a = A + (j + 1 + (active ? cc : 0)) * ld;
        cx<T> w = czero<T>();
        if (active) {
            // four independent partial sums keep the FMA chains short
            cx<T> w1 = czero<T>(), w2 = czero<T>(), w3 = czero<T>();
            if (g == 0) w = a[j];
            int r = j + 1 + g;
            for (; r + 3 * G < M; r += 4 * G) {
                cmac_cj(w, v[r], a[r]);
                cmac_cj(w1, v[r + G], a[r + G]);
                cmac_cj(w2, v[r + 2 * G], a[r + 2 * G]);
                cmac_cj(w3, v[r + 3 * G], a[r + 3 * G]);
            }
            for (; r < M; r += G) cmac_cj(w, v[r], a[r]);
            w = (w + w1) + (w2 + w3);
        }
        for (int o = G >> 1; o > 0; o >>= 1) {
            w.re += __shfl_xor_sync(0xffffffffu, w.re, o);
            w.im += __shfl_xor_sync(0xffffffffu, w.im, o);
        }
        if (active) {
            w = t * w;
            if (g == 0) a[j] = a[j] - w;
#pragma unroll 1
            for (int r = j + 1 + g; r < M; r += G) cmsub(a[r], v[r], w);
        }
    }
}

// Householder step j of a QR: reflector for column j (rows j..M-1), applied to
// columns j+1..N-1 (LAPACK geqr2 convention, H_j = I - tau_j v_j v_j^H, R[j][j]
// real).  The reflector tail replaces A(j+1:M, j); tau[j] gets the scalar.
template <int NTHR, typename T>
__device__ __forceinline__ void householder_step(cx<T>* A, int ld, int M, int N, int j, cx<T>* tau, double* red,
                                                 int tid) {
    cx<T>* col = A + j * ld;
    T s = T(0);
    for (int r = j + 1 + tid; r < M; r += NTHR) s += norm2(col[r]);
    s = team_sum<NTHR>(s, red, tid);
    const cx<T> alpha = col[j];
    const bool trivial = (s == T(0)) && (alpha.im == T(0));
    cx<T> t = czero<T>();
    T beta = alpha.re;
    cx<T> scale = mk<T>(T(1), T(0));
    if (!trivial) {
        const T nrm = sqrt(norm2(alpha) + s);
        beta = alpha.re >= T(0) ? -nrm : nrm;
        t = mk<T>((beta - alpha.re) / beta, -alpha.im / beta);
        const cx<T> d = mk<T>(alpha.re - beta, alpha.im);
        const T dd = norm2(d);
        scale = mk<T>(d.re / dd, -d.im / dd);
    }
    tsync<NTHR>();
    if (!trivial) {
        for (int r = j + 1 + tid; r < M; r += NTHR) col[r] = col[r] * scale;
    }
    if (tid == 0) {
        col[j] = mk<T>(beta, T(0));
        tau[j] = t;
    }
    tsync<NTHR>();
    if (!trivial) apply_reflector<NTHR>(A, ld, M, N, j, conj(t), tid);
    tsync<NTHR>();
}

// Householder QR of the M x N matrix A (K = min(M, N) reflectors,
// A = H_0 ... H_{K-1} R).  On return the upper trapezoid holds R (real diagonal),
// the strict lower part the reflector tails, tau[0..K) the scalars.  red: NTHR/32
// doubles of scratch.
template <int NTHR, typename T>
__device__ void team_qr(cx<T>* A, int ld, int M, int N, cx<T>* tau, double* red, int tid) {
    const int K = M < N ? M : N;
    for (int j = 0; j < K; ++j) householder_step<NTHR>(A, ld, M, N, j, tau, red, tid);
}

// Householder QR with column pivoting (Businger-Golub), stopped after `steps`
// reflectors: A P = Q R with the largest remaining column moved to position j
// before step j (ties: the lowest index).  perm[c] is the original index of
// column c; cnorm: N scratch values.  For a matrix of rank <= steps the rows of R
// below `steps` are rounding noise, so Q(:, 0:steps) and R(0:steps, :) P^T
// reproduce A to the working precision (rank-revealing split).
template <int NTHR, typename T>
__device__ void team_qrcp(cx<T>* A, int ld, int M, int N, int steps, cx<T>* tau, int* perm, T* cnorm,
                          double* red, int tid) {
    for (int c = tid; c < N; c += NTHR) perm[c] = c;
    tsync<NTHR>();
    for (int j = 0; j < steps; ++j) {
        for (int c = j + tid; c < N; c += NTHR) {
            const cx<T>* a = A + c * ld;
            T s = T(0);
            for (int r = j; r < M; ++r) s += norm2(a[r]);
            cnorm[c] = s;
        }
        tsync<NTHR>();
        int p = j;
        T best = cnorm[j];
        for (int c = j + 1; c < N; ++c)
            if (cnorm[c] > best) { best = cnorm[c]; p = c; }
        if (p != j) {
            cx<T>* a = A + j * ld;
            cx<T>* b = A + p * ld;
            for (int r = tid; r < M; r += NTHR) {
                const cx<T> x = a[r];
                a[r] = b[r];
                b[r] = x;
            }
            if (tid == 0) {
                const int x = perm[j];
                perm[j] = perm[p];
                perm[p] = x;
            }
        }
        tsync<NTHR>();
        householder_step<NTHR>(A, ld, M, N, j, tau, red, tid);
    }
}

// Overwrite the reflectors left by team_qr with the explicit M x K factor Q
// (LAPACK ung2r): Q = H_0 ... H_{K-1} [I_K; 0].
template <int NTHR, typename T>
__device__ void team_form_q(cx<T>* A, int ld, int M, int K, const cx<T>* tau, int tid) {
    for (int i = K - 1; i >= 0; --i) {
        const cx<T> t = tau[i];
        if (t.re != T(0) || t.im != T(0)) apply_reflector<NTHR>(A, ld, M, K, i, t, tid);
        tsync<NTHR>();
        cx<T>* v = A + i * ld;
        for (int r = tid; r < M; r += NTHR) {
            cx<T> val;
            if (r < i) val = czero<T>();
            else if (r == i) val = mk<T>(T(1) - t.re, -t.im);
            else val = czero<T>() - t * v[r];
            v[r] = val;
        }
        tsync<NTHR>();
    }
}

// c a - f b for real c and complex f, as one fma chain per component.
template <typename T>
__device__ __forceinline__ cx<T> rot_minus(T c, cx<T> a, cx<T> f, cx<T> b) {
    const T tr = fma(f.re, b.re, -mul_rn(f.im, b.im)), ti = fma(f.re, b.im, mul_rn(f.im, b.re));
    return mk<T>(fma(c, a.re, -tr), fma(c, a.im, -ti));
}
// s a + g b for real s and complex g.
template <typename T>
__device__ __forceinline__ cx<T> rot_plus(T s, cx<T> a, cx<T> g, cx<T> b) {
    const T tr = fma(g.re, b.re, -mul_rn(g.im, b.im)), ti = fma(g.re, b.im, mul_rn(g.im, b.re));
    return mk<T>(fma(s, a.re, tr), fma(s, a.im, ti));
}

// One round of a parallel Jacobi method on the K x K Hermitian matrix G (column-major,
// ld) with the accumulated basis V: the calling thread belongs to the group of LP
// threads (sub = its index there) that owns the pair (p, q), p < q (p < 0: no pair),
// and every pair of the round is disjoint from the others.  The rotation
// J = [[c, conj(z)], [-z, c]] (c real, c^2 + |z|^2 = 1) zeroes G[p][q] = g:
// z = c (t / |g|) conj(g), t the tangent of the rotation angle,
// t / |g| = 2 sgn(d) / (|d| + sqrt(d^2 + 4 |g|^2)), d = G[q][q] - G[p][p].  For
// |g| < 5e-4 |d| (every rotation of a warm-started solve) the series
// t / |g| = w (1 - q + 2 q^2), c = 1 - t^2 / 2 + 3 t^4 / 8 (w = 1 / d,
// q = |g|^2 w^2 < 2.5e-7; the truncation errors are below 1e-19) need one division and
// no square root.  |g| itself is never formed: the rotate-or-not test compares
// |g|^2 with abs_tol2 and eps2 |G_pp G_qq|.  Returns whether this pair rotated.
template <int NTHR, typename T>
__device__ __forceinline__ bool jacobi_round(cx<T>* G, cx<T>* V, int ld, int K, int p, int q, int sub, int LP,
                                             T eps2, T abs_tol2) {
    T c = T(1);
    cx<T> z = czero<T>();
    bool rot = false;
    if (p >= 0) {
        const T a = G[p * ld + p].re, b = G[q * ld + q].re;
        const cx<T> g = G[q * ld + p];  // G[p][q]
        const T gg = norm2(g);
        if (gg > abs_tol2 && gg > eps2 * fabs(a * b)) {
            rot = true;
            const T d = b - a;
            T tg, t2;
            if (T(4) * gg < T(1e-6) * d * d) {
                const T w = T(1) / d, qq = gg * w * w;
                tg = w * fma(qq, fma(T(2), qq, T(-1)), T(1));
                t2 = gg * tg * tg;
                c = fma(t2, fma(T(0.375), t2, T(-0.5)), T(1));
            } else {
                tg = (d >= T(0) ? T(2) : T(-2)) / (fabs(d) + sqrt(fma(d, d, T(4) * gg)));
                t2 = gg * tg * tg;
                if constexpr (sizeof(T) == 8) c = rsqrt(T(1) + t2);
                else c = T(1) / sqrt(T(1) + t2);
            }
            const T f = c * tg;
            z = mk<T>(f * g.re, -f * g.im);
        }
    }
    tsync<NTHR>();
    // columns of G and V: G <- G J, V <- V J
    if (rot) {
        const cx<T> zc = conj(z);
        for (int r = sub; r < K; r += LP) {
            const cx<T> gp = G[p * ld + r], gq = G[q * ld + r];
            G[p * ld + r] = rot_minus(c, gp, z, gq);
            G[q * ld + r] = rot_plus(c, gq, zc, gp);
            const cx<T> vp = V[p * ld + r], vq = V[q * ld + r];
            V[p * ld + r] = rot_minus(c, vp, z, vq);
            V[q * ld + r] = rot_plus(c, vq, zc, vp);
        }
    }
    tsync<NTHR>();
    // rows of G: G <- J^H G, J^H = [[c, -conj(z)], [z, c]]
    if (rot) {
        const cx<T> zc = conj(z);
        for (int col = sub; col < K; col += LP) {
            const cx<T> gp = G[col * ld + p], gq = G[col * ld + q];
            G[col * ld + p] = rot_minus(c, gp, zc, gq);
            G[col * ld + q] = rot_plus(c, gq, z, gp);
        }
    }
    tsync<NTHR>();
    if (rot && sub == 0) {  // the 2x2 block is diagonal in exact arithmetic
        G[q * ld + p] = czero<T>();
        G[p * ld + q] = czero<T>();
        G[p * ld + p].im = T(0);
        G[q * ld + q].im = T(0);
    }
    tsync<NTHR>();
    return rot;
}

// Rotation thresholds of the Jacobi solvers: rotate while |G_pq| exceeds the rounding
// level of the pair's diagonal (eps) or of the trace (abs_tol); returned squared.
template <int NTHR, typename T>
__device__ __forceinline__ void jacobi_thresholds(const cx<T>* G, int ld, int K, int tid, double* red, T* eps2,
                                                  T* abs_tol2) {
    T tr = T(0);
    for (int r = tid; r < K; r += NTHR) tr += fabs(G[r * ld + r].re);
    tr = team_sum<NTHR>(tr, red, tid);
    const T eps = sizeof(T) == 4 ? T(3e-7) : T(1e-15);
    const T abs_tol = (sizeof(T) == 4 ? T(3e-8) : T(1e-17)) * (tr > T(0) ? tr : T(1));
    *eps2 = eps * eps;
    *abs_tol2 = abs_tol * abs_tol;
}

template <int NTHR>
__device__ __forceinline__ bool team_any(bool v) {
    if constexpr (NTHR == 32) return __any_sync(0xffffffffu, v);
    else return __syncthreads_or(v) != 0;
}

// Cyclic parallel (round-robin) Jacobi eigensolver for the K x K Hermitian matrix G
// (column-major, ld), K <= 2 NTHR, run by a team of NTHR threads in the arithmetic of
// T.  On return diag(G) holds the eigenvalues and the columns of V (K x K, ld) the
// eigenvectors: G_in = V diag(lambda) V^H.  A round rotates K/2 disjoint index pairs;
// each pair is owned by a group of LP threads (a power of two) that split the rows
// (column phase) and the columns (row phase) of the update.  With v_given the columns
// of V already hold an orthonormal starting basis (G being the matrix in that basis)
// and the rotations accumulate onto it.  red: NTHR/32 doubles.  Returns the sweeps.
template <int NTHR, typename T>
__device__ int team_jacobi_eigh(cx<T>* G, cx<T>* V, int ld, int K, int tid, int max_sweeps, double* red,
                                bool v_given = false) {
    if (!v_given)
        for (int c = 0; c < K; ++c)
            for (int r = tid; r < K; r += NTHR) V[c * ld + r] = mk<T>(r == c ? T(1) : T(0), T(0));
    T eps2, abs_tol2;
    jacobi_thresholds<NTHR, T>(G, ld, K, tid, red, &eps2, &abs_tol2);
    const int Kp = (K + 1) & ~1;          // even number of slots; slot K (if K odd) is a dummy
    const int npairs = Kp / 2;
    int LP = 1;                           // threads per pair
    while (LP * 2 * npairs <= NTHR) LP *= 2;
    const int pair = tid / LP, sub = tid % LP;
    int sweep = 0;
    tsync<NTHR>();
    for (; sweep < max_sweeps; ++sweep) {
        bool rotated = false;
        for (int round = 0; round < Kp - 1; ++round) {
            // round-robin pairing: slot 0 fixed, slots 1..Kp-1 rotate
            int p = -1, q = -1;
            if (pair < npairs) {
                const int a = pair, b = Kp - 1 - pair;
                auto pos = [&](int s) { return s == 0 ? 0 : 1 + (s - 1 + round) % (Kp - 1); };
                p = pos(a);
                q = pos(b);
                if (p > q) { int tmp = p; p = q; q = tmp; }
                if (q >= K) p = -1;  // pair with the dummy slot
            }
            rotated |= jacobi_round<NTHR, T>(G, V, ld, K, p, q, sub, LP, eps2, abs_tol2);
        }
        if (!team_any<NTHR>(rotated)) break;
    }
    return sweep;
}

// Block version for a truncation: the indices ord[0 .. keep) (kept) and
// ord[keep .. K) (discarded) split G, and only pairs with one index in each part are
// rotated, until G has no entry between the two parts above the rounding level.  The
// kept columns of V then span the invariant subspace of the kept part's eigenvalues,
// and the discarded part's diagonal sums to its eigenvalues, which is all a truncation
// uses (the basis inside the kept subspace is a gauge of the new bond).  Round r pairs
// index i of the smaller part with index (i + r) mod (size of the larger part) of the
// other, so every cross pair appears once per sweep: keep (K - keep) rotations in
// max(keep, K - keep) rounds, against K (K - 1) / 2 in K - 1 rounds for the full solve.
// The split must not separate a cluster of eigenvalues (the caller checks the gap).
template <int NTHR, typename T>
__device__ int team_jacobi_cross(cx<T>* G, cx<T>* V, int ld, int K, const int* ord, int keep, int tid,
                                 int max_sweeps, double* red) {
    T eps2, abs_tol2;
    jacobi_thresholds<NTHR, T>(G, ld, K, tid, red, &eps2, &abs_tol2);
    const int nd = K - keep;
    const int small = keep < nd ? keep : nd, large = keep < nd ? nd : keep;
    int LP = 1;
    while (LP * 2 * small <= NTHR) LP *= 2;
    const int pair = tid / LP, sub = tid % LP;
    int sweep = 0;
    tsync<NTHR>();
    for (; sweep < max_sweeps; ++sweep) {
        bool rotated = false;
        for (int round = 0; round < large; ++round) {
            int p = -1, q = -1;
            if (pair < small) {
                int j = pair + round;
                if (j >= large) j -= large;
                const int x = keep <= nd ? ord[pair] : ord[j];
                const int y = keep <= nd ? ord[keep + j] : ord[keep + pair];
                p = x < y ? x : y;
                q = x < y ? y : x;
            }
            rotated |= jacobi_round<NTHR, T>(G, V, ld, K, p, q, sub, LP, eps2, abs_tol2);
        }
        if (!team_any<NTHR>(rotated)) break;
    }
    return sweep;
}

}  // namespace mpsano
