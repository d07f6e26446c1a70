// Warp-level small dense linear algebra on shared memory: Householder QR,
// explicit Q, and a cyclic Jacobi eigensolver for Hermitian matrices.
// Matrices are column-major: element (r, c) at A[c * ld + r].
#pragma once
#include "common.cuh"

namespace mpsano {

// Largest power of two G <= 32 with G * nc <= 32 (at least 1): lanes per column
// when nc columns are processed by one warp.
__device__ __forceinline__ int lanes_per_col(int nc) {
    int G = 32;
    while (G > 1 && G * nc > 32) G >>= 1;
    return G;
}

// A(j:M, j+1:N) <- (I - t v v^H) A(j:M, j+1:N), v = [1; A(j+1:M, j)] stored in column j.
// Rows are split over G lanes per column; partial dot products are combined with
// xor-shuffles inside each aligned lane group.
template <typename T>
__device__ __forceinline__ void apply_reflector(cx<T>* A, int ld, int M, int N, int j, cx<T> t, int lane) {
    const int nc = N - j - 1;
    if (nc <= 0) return;
    const cx<T>* v = A + j * ld;
    const int G = lanes_per_col(nc);
    const int cg = lane / G, g = lane % G;
    const int per_pass = 32 / G;
    for (int c0 = 0; c0 < nc; c0 += per_pass) {
        const int cc = c0 + cg;
        const bool active = cc < nc;
        cx<T>* a = A + (j + 1 + (active ? cc : 0)) * ld;
        cx<T> w = czero<T>();
        if (active) {
            if (g == 0) w = a[j];
            for (int r = j + 1 + g; r < M; r += G) cmac_cj(w, v[r], a[r]);
        }
        for (int o = G >> 1; o > 0; o >>= 1) {
            w.re += __shfl_xor_sync(0xffffffffu, w.re, o);
            w.im += __shfl_xor_sync(0xffffffffu, w.im, o);
        }
        if (active) {
            w = t * w;
            if (g == 0) a[j] = a[j] - w;
            for (int r = j + 1 + g; r < M; r += G) a[r] = a[r] - v[r] * w;
        }
    }
}

// Householder QR of the M x N matrix A (LAPACK geqr2 convention, K = min(M, N)
// reflectors H_j = I - tau_j v_j v_j^H, A = H_0 ... H_{K-1} R).  On return the
// upper trapezoid holds R (real diagonal), the strict lower part the reflector
// tails, tau[0..K) the scalars.
template <typename T>
__device__ void warp_qr(cx<T>* A, int ld, int M, int N, cx<T>* tau, int lane) {
    const int K = M < N ? M : N;
    for (int j = 0; j < K; ++j) {
        cx<T>* col = A + j * ld;
        T s = T(0);
        for (int r = j + 1 + lane; r < M; r += 32) s += norm2(col[r]);
        s = warp_sum(s);
        const cx<T> alpha = col[j];
        const bool trivial = (s == T(0)) && (alpha.im == T(0));
        cx<T> t = czero<T>();
        T beta = alpha.re;
        cx<T> scale = mk<T>(T(1), T(0));
        if (!trivial) {
            const T nrm = sqrt(alpha.re * alpha.re + alpha.im * alpha.im + s);
            beta = alpha.re >= T(0) ? -nrm : nrm;
            t = mk<T>((beta - alpha.re) / beta, -alpha.im / beta);
            const cx<T> d = mk<T>(alpha.re - beta, alpha.im);
            const T dd = norm2(d);
            scale = mk<T>(d.re / dd, -d.im / dd);
        }
        __syncwarp();
        if (!trivial) {
            for (int r = j + 1 + lane; r < M; r += 32) col[r] = col[r] * scale;
        }
        if (lane == 0) {
            col[j] = mk<T>(beta, T(0));
            tau[j] = t;
        }
        __syncwarp();
        if (!trivial) apply_reflector(A, ld, M, N, j, conj(t), lane);
        __syncwarp();
    }
}

// Overwrite the reflectors left by warp_qr with the explicit M x K factor Q
// (LAPACK ung2r): Q = H_0 ... H_{K-1} [I_K; 0].
template <typename T>
__device__ void warp_form_q(cx<T>* A, int ld, int M, int K, const cx<T>* tau, int lane) {
    for (int i = K - 1; i >= 0; --i) {
        const cx<T> t = tau[i];
        if (t.re != T(0) || t.im != T(0)) apply_reflector(A, ld, M, K, i, t, lane);
        __syncwarp();
        cx<T>* v = A + i * ld;
        for (int r = lane; r < M; r += 32) {
            cx<T> val;
            if (r < i) val = czero<T>();
            else if (r == i) val = mk<T>(T(1) - t.re, -t.im);
            else val = czero<T>() - t * v[r];
            v[r] = val;
        }
        __syncwarp();
    }
}

// Cyclic parallel (round-robin) Jacobi eigensolver for the K x K Hermitian matrix G
// (column-major, ld), K <= 64.  On return diag(G) holds the eigenvalues and the
// columns of V (K x K, ld) the eigenvectors: G_in = V diag(lambda) V^H.  Each lane
// owns one disjoint index pair per round; a round applies all rotations to the
// columns of G and V, then to the rows of G.  Returns the sweeps used.
static __device__ int warp_jacobi_eigh(cx<double>* G, cx<double>* V, int ld, int K, int lane, int max_sweeps) {
    for (int c = 0; c < K; ++c)
        for (int r = lane; r < K; r += 32) V[c * ld + r] = mk<double>(r == c ? 1.0 : 0.0, 0.0);
    // scale for the absolute threshold
    double tr = 0.0;
    for (int r = lane; r < K; r += 32) tr += fabs(G[r * ld + r].re);
    tr = warp_sum(tr);
    const double abs_tol = 1e-17 * (tr > 0.0 ? tr : 1.0);
    const int Kp = (K + 1) & ~1;          // even number of slots; slot K (if K odd) is a dummy
    const int npairs = Kp / 2;
    int sweep = 0;
    __syncwarp();
    for (; sweep < max_sweeps; ++sweep) {
        int rotated = 0;
        for (int round = 0; round < Kp - 1; ++round) {
            // round-robin pairing: slot 0 fixed, slots 1..Kp-1 rotate
            int p = -1, q = -1;
            if (lane < npairs) {
                int a = lane, b = Kp - 1 - lane;
                auto pos = [&](int s) { return s == 0 ? 0 : 1 + (s - 1 + round) % (Kp - 1); };
                p = pos(a);
                q = pos(b);
                if (p > q) { int tmp = p; p = q; q = tmp; }
                if (q >= K) p = -1;  // pair with the dummy slot
            }
            double c = 1.0, s = 0.0;
            cx<double> e = mk<double>(1.0, 0.0);  // e^{-i phi}
            bool rot = false;
            if (p >= 0) {
                const double a = G[p * ld + p].re, b = G[q * ld + q].re;
                const cx<double> g = G[q * ld + p];  // G[p][q]
                const double ag = sqrt(norm2(g));
                if (ag > abs_tol && ag * ag > 1e-30 * fabs(a * b)) {
                    rot = true;
                    e = mk<double>(g.re / ag, -g.im / ag);
                    const double tau = (b - a) / (2.0 * ag);
                    const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                    c = 1.0 / sqrt(1.0 + t * t);
                    s = t * c;
                }
            }
            rotated |= rot;
            __syncwarp();
            // columns of G and V: G <- G J, V <- V J,
            // J(p,p) = c, J(p,q) = s, J(q,p) = -s e, J(q,q) = c e, e = e^{-i phi}
            if (rot) {
                for (int r = 0; r < K; ++r) {
                    const cx<double> gp = G[p * ld + r], gq = G[q * ld + r];
                    G[p * ld + r] = c * gp - s * (e * gq);
                    G[q * ld + r] = s * gp + c * (e * gq);
                    const cx<double> vp = V[p * ld + r], vq = V[q * ld + r];
                    V[p * ld + r] = c * vp - s * (e * vq);
                    V[q * ld + r] = s * vp + c * (e * vq);
                }
            }
            __syncwarp();
            // rows of G: G <- J^H G
            if (rot) {
                const cx<double> ec = conj(e);
                for (int col = 0; col < K; ++col) {
                    const cx<double> gp = G[col * ld + p], gq = G[col * ld + q];
                    G[col * ld + p] = c * gp - s * (ec * gq);
                    G[col * ld + q] = s * gp + c * (ec * gq);
                }
            }
            __syncwarp();
            if (rot) {  // the 2x2 block is diagonal in exact arithmetic
                G[q * ld + p] = czero<double>();
                G[p * ld + q] = czero<double>();
                G[p * ld + p].im = 0.0;
                G[q * ld + q].im = 0.0;
            }
            __syncwarp();
        }
        if (!__any_sync(0xffffffffu, rotated)) break;
    }
    return sweep;
}

}  // namespace mpsano
