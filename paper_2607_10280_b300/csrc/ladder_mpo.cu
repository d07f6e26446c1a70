// Circuits as operator products (Sec. II.B, Eq. 3), and the left environments they
// then need.
//
// The CNOT ladder CNOT(0->1), CNOT(1->2), ..., CNOT(n-2->n-1) applied in that order
// maps the basis state |x_0 x_1 ... x_{n-1}> to |p_0 p_1 ... p_{n-1}> with the prefix
// parities p_k = x_0 xor ... xor x_k.  As a matrix product operator its bond carries
// the running parity (dimension 2): site k reads the incoming parity a and its input
// bit x, and emits output bit and outgoing parity b = a xor x.  Applied to an MPS it
// doubles every bond and only copies entries:
//     A'[(l, a)][b][(r, b)] = A[l][a xor b][r],   zero for an output bit other than b,
// with a = 0 at site 0 (no incoming parity) and the outgoing parity equal to the output
// bit at site n-1 (A'[(l, a)][s][r] = A[l][a xor s][r]).  A layer is its one-qubit gates
// followed by this operator, so L layers on the encoded product state give an exact
// MPS with bond 2^L at every inner cut, site by site and without any factorisation:
// ladder_mpo_kernel builds each site tensor independently.  No step truncates, so this
// path is for circuits with 2^L <= chi; the state is exact up to rounding.
//
// The paper's brick-wall layer (CNOTs on the even bonds, then on the odd bonds) has
// the same form: a CNOT is sum_c |c><c| (x) X^c, i.e. the projector P_c on the control
// and X^c on the target joined by a bond index c, and every bond carries one CNOT per
// layer.  Site k gets P_b from the CNOT on its right bond and X^a from the one on its
// left bond, in the order the layer applies them: left first (P_b X^a: the whole
// ladder, and the odd sites of the brick-wall), giving A[l][a xor b][r] at output bit
// b, or right first (X^a P_b: the even sites of the brick-wall), giving A[l][b][r] at
// output bit a xor b.
//
// The result is not left-canonical (a layer's operator keeps left orthonormality only
// where the incoming parity is summed, not at site 0), so the Pauli kernel contracts
// the left environments L_k = sum_s A_{k-1}^{s dagger} L_{k-1} A_{k-1}^s (L_0 = 1)
// that renv_kernel writes beside the right ones (lenv_image), for the images marked
// META_LENV.
#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "batch.h"
#include "circuit.cuh"

namespace mpsano {
namespace {

constexpr int MPO_MAXB = 16;                       // largest bond 2^L of this path (L <= 4)
constexpr int MPO_BUF = MPO_MAXB * 2 * MPO_MAXB;   // one site tensor, compact [Dl][2][Dr]
constexpr int MPO_WARPS = 4;

// One CTA per image of order[0 .. n_images), its warps taking the sites in turn.
template <typename T>
__global__ void __launch_bounds__(32 * MPO_WARPS) ladder_mpo_kernel(
    const ImageMeta* __restrict__ meta, int n_images, const int32_t* __restrict__ order,
    const double* __restrict__ pixels, const cx<T>* __restrict__ gates, int gn, int ansatz,
    cx<T>* __restrict__ arena, int32_t* __restrict__ bonds_out, double* __restrict__ discarded_out,
    int* status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T>* buf = reinterpret_cast<cx<T>*>(smem_raw);   // per warp: two site tensors
    const int slot = blockIdx.x;
    if (slot >= n_images) return;
    const int img = order ? order[slot] : slot;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const ImageMeta mt = meta[img];
    const int n = mt.n, ld = mt.ld, L = mt.L;
    if ((1 << L) > MPO_MAXB || (1 << L) > ld) {   // never expected: the host routes by these bounds
        if (threadIdx.x == 0) raise_status(status, DEV_BOND_OVERFLOW);
        return;
    }
    const double* px = pixels + mt.pixel_off;
    cx<T>* sites = arena + mt.site_off;
    for (int k = warp; k < n; k += MPO_WARPS) {
        cx<T>* cur = buf + (size_t)warp * 2 * MPO_BUF;
        cx<T>* nxt = cur + MPO_BUF;
        // ladder: the encoding R_Y(pi x) on |0>; paper: |0> (it encodes in every layer)
        if (lane == 0) {
            T sn = T(0), cs = T(1);
            if (ansatz == 0) encode_amplitudes(px[k], &sn, &cs);
            cur[0] = mk<T>(cs, T(0));
            cur[1] = mk<T>(sn, T(0));
        }
        // the CNOT on the right bond acts before the one on the left bond (brick-wall,
        // even site): X^a P_b; otherwise P_b X^a
        const bool right_first = ansatz != 0 && (k & 1) == 0;
        // every dimension is a power of two: indices by shifts and masks
        int sl = 0, sr = 0;   // log2 Dl, log2 Dr
        for (int layer = 0; layer < L; ++layer) {
            __syncwarp();
            // the layer's one-qubit gate on the physical index
            const Gate1<T> g = table_gate<T>(gates, gn, ansatz, layer, img, k);
            for (int e = lane; e < (1 << (sl + sr)); e += 32) {
                const int l = e >> sr, r = e & ((1 << sr) - 1);
                const int i0 = ((2 * l) << sr) + r, i1 = i0 + (1 << sr);
                const cx<T> a0 = cur[i0], a1 = cur[i1];
                cur[i0] = cdot2(g.u00, a0, g.u01, a1);
                cur[i1] = cdot2(g.u10, a0, g.u11, a1);
            }
            __syncwarp();
            // the layer's CNOTs: new bond index = old index + old dimension * bond bit
            const int sl2 = k == 0 ? sl : sl + 1;
            const int sr2 = k == n - 1 ? sr : sr + 1;
            for (int e = lane; e < (2 << (sl2 + sr2)); e += 32) {
                const int l2 = e >> (sr2 + 1), s = (e >> sr2) & 1, r2 = e & ((1 << sr2) - 1);
                const int a = l2 >> sl, l = l2 & ((1 << sl) - 1);   // a = 0 at site 0
                cx<T> v;
                if (k == n - 1) {
                    v = cur[((2 * l + (a ^ s)) << sr) + r2];
                } else {
                    const int b = r2 >> sr, r = r2 & ((1 << sr) - 1);
                    if (right_first) v = s == (a ^ b) ? cur[((2 * l + b) << sr) + r] : czero<T>();
                    else v = s == b ? cur[((2 * l + (a ^ b)) << sr) + r] : czero<T>();
                }
                nxt[e] = v;
            }
            cx<T>* t = cur; cur = nxt; nxt = t;
            sl = sl2;
            sr = sr2;
        }
        __syncwarp();
        const int Dl = 1 << sl;
        cx<T>* dst = sites + (size_t)k * 2 * ld * ld;
        for (int e = lane; e < (2 << (sl + sr)); e += 32) {
            const int row = e >> sr, r = e & ((1 << sr) - 1);
            dst[row * ld + r] = cur[e];
        }
        if (lane == 0) bonds_out[mt.bond_off + k] = Dl;
        __syncwarp();
    }
    if (threadIdx.x == 0) {
        bonds_out[mt.bond_off + n] = 1;
        discarded_out[img] = 0.0;
    }
}

// v <- u v with the rounding of cdot2 when one of its two terms is an exact zero (the
// layered kernel's gate application at a half-structured site): each component is one
// rounded product followed by one fma.
template <typename T>
__device__ __forceinline__ cx<T> mpo_mul(cx<T> u, cx<T> v) {
    return mk<T>(fma(-u.im, v.im, mul_rn(u.re, v.re)), fma(u.im, v.re, mul_rn(u.re, v.im)));
}

// The ladder's site tensors in closed form, every element computed on its own (no shared
// memory, no intermediate layers).  With l = sum_j a_j 2^(j-1) and r = sum_j b_j 2^(j-1)
// (a_j, b_j the incoming and outgoing parities of layer j; a = 0 at site 0), an inner
// site's element is zero unless s = b_L, and otherwise
//     A[l][s][r] = y[a_1 xor b_1] * prod_{j = 2..L} U_j[a_j xor b_j][b_(j-1)],
// y = U_1 (cos(pi x / 2), sin(pi x / 2)): before layer j's CNOT the physical index is
// a_j xor b_j and after it b_j, which the next gate reads alone (the other physical
// component is zero).  The last site has no right bond: its physical 2-vector goes
// through v <- X^(a_j) U_j v.  The paper's brick-wall has the same form with the roles
// of the two parities swapped at its even sites (X^a P_b: t = b before and a xor b after
// the CNOTs), and |0> re-encoded by its per-image gate in every layer.  The products are
// rounded in the layered kernel's order (its gate applications add exact zeros), so both
// kernels write the same values.
// Grid: (images, site groups of MPO_DIRECT_WARPS sites); one warp per site.
constexpr int MPO_DIRECT_WARPS = 8;

template <typename T>
__global__ void __launch_bounds__(32 * MPO_DIRECT_WARPS) ladder_mpo_direct_kernel(
    const ImageMeta* __restrict__ meta, int n_images, const int32_t* __restrict__ order,
    const double* __restrict__ pixels, const cx<T>* __restrict__ gates, int gn, int ansatz,
    cx<T>* __restrict__ arena, int32_t* __restrict__ bonds_out, double* __restrict__ discarded_out,
    int* status) {
    constexpr int MAXL = 4;   // 2^L <= MPO_MAXB
    const int slot = blockIdx.x;
    if (slot >= n_images) return;
    const int img = order ? order[slot] : slot;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const ImageMeta mt = meta[img];
    const int n = mt.n, ld = mt.ld, L = mt.L;
    if (L < 0 || L > MAXL || (1 << L) > MPO_MAXB || (1 << L) > ld) {   // the host routes by these bounds
        if (threadIdx.x == 0) raise_status(status, DEV_BOND_OVERFLOW);
        return;
    }
    const double* px = pixels + mt.pixel_off;
    cx<T>* sites = arena + mt.site_off;
    const int k = blockIdx.y * MPO_DIRECT_WARPS + warp;
    if (k < n) {
        // ladder: the encoding R_Y(pi x) on |0>; paper: |0> (it encodes in every layer)
        T sn = T(0), cs = T(1);
        if (ansatz == 0) encode_amplitudes(px[k], &sn, &cs);
        const cx<T> x0 = mk<T>(cs, T(0)), x1 = mk<T>(sn, T(0));
        Gate1<T> g[MAXL];
#pragma unroll
        for (int j = 0; j < MAXL; ++j)
            if (j < L) g[j] = table_gate<T>(gates, gn, ansatz, j, img, k);
        // physical index before (t) and after (p) each layer's CNOTs, as bits j of tb and
        // pb: P_b X^a (ladder, odd brick-wall sites) t = a xor b, p = b; X^a P_b (even
        // brick-wall sites) t = b, p = a xor b
        const bool right_first = ansatz != 0 && (k & 1) == 0;
        const int sl = k == 0 ? 0 : L, sr = k == n - 1 ? 0 : L;   // log2 of the bonds
        cx<T>* dst = sites + (size_t)k * 2 * ld * ld;
        if (k < n - 1) {
            const cx<T> y0 = L > 0 ? cdot2(g[0].u00, x0, g[0].u01, x1) : x0;
            const cx<T> y1 = L > 0 ? cdot2(g[0].u10, x0, g[0].u11, x1) : x1;
            for (int e = lane; e < (2 << (sl + sr)); e += 32) {
                const int row = e >> sr, r = e & ((1 << sr) - 1);
                const int l = row >> 1, s = row & 1;
                const int tb = right_first ? r : (l ^ r), pbits = right_first ? (l ^ r) : r;
                cx<T> v;
                if (L == 0) {
                    v = s ? x1 : x0;
                } else if (s != ((pbits >> (L - 1)) & 1)) {
                    v = czero<T>();
                } else {
                    v = (tb & 1) ? y1 : y0;
#pragma unroll
                    for (int j = 1; j < MAXL; ++j) {
                        if (j < L) {
                            const int t = (tb >> j) & 1, pb = (pbits >> (j - 1)) & 1;
                            const cx<T> u = t ? (pb ? g[j].u11 : g[j].u10) : (pb ? g[j].u01 : g[j].u00);
                            v = mpo_mul(u, v);
                        }
                    }
                }
                dst[row * ld + r] = v;
            }
        } else {
            // last site: one 2-vector per left index l
            for (int l = lane; l < (1 << sl); l += 32) {
                cx<T> v0 = x0, v1 = x1;
#pragma unroll
                for (int j = 0; j < MAXL; ++j) {
                    if (j < L) {
                        const cx<T> w0 = cdot2(g[j].u00, v0, g[j].u01, v1);
                        const cx<T> w1 = cdot2(g[j].u10, v0, g[j].u11, v1);
                        const bool a = (l >> j) & 1;
                        v0 = a ? w1 : w0;
                        v1 = a ? w0 : w1;
                    }
                }
                dst[(2 * l) * ld] = v0;
                dst[(2 * l + 1) * ld] = v1;
            }
        }
        if (lane == 0) bonds_out[mt.bond_off + k] = 1 << sl;
    }
    if (blockIdx.y == 0 && threadIdx.x == 0) {
        bonds_out[mt.bond_off + n] = 1;
        discarded_out[img] = 0.0;
    }
}

template <typename T>
mps_status launch_mpo_t(mps_batch* b, const double* pixels, int ansatz) {
    // the closed form; MPSANO_MPO=layered selects the layer-by-layer kernel (the two
    // write the same values; the tests compare them)
    const char* mode = std::getenv("MPSANO_MPO");
    if (!(mode && std::strcmp(mode, "layered") == 0)) {
        auto kd = ladder_mpo_direct_kernel<T>;
        timing_begin(b, KIND_CIRCUIT);
        const dim3 grid((unsigned)b->run_count, (unsigned)((b->n_max + MPO_DIRECT_WARPS - 1) / MPO_DIRECT_WARPS));
        kd<<<grid, 32 * MPO_DIRECT_WARPS, 0, b->stream>>>(b->meta_d, b->run_count, b->run_order, pixels,
                                                        reinterpret_cast<const cx<T>*>(b->gates), b->gate_n, ansatz,
                                                        reinterpret_cast<cx<T>*>(b->arena), b->bonds_d,
                                                        b->discarded_d, b->status_d);
        timing_end(b);
        CUDA_TRY(cudaGetLastError());
        count_launch();
        return MPS_OK;
    }
    auto k = ladder_mpo_kernel<T>;
    const size_t smem = sizeof(cx<T>) * 2 * MPO_BUF * MPO_WARPS;
    CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    timing_begin(b, KIND_CIRCUIT);
    k<<<b->run_count, 32 * MPO_WARPS, smem, b->stream>>>(b->meta_d, b->run_count, b->run_order, pixels,
                                                      reinterpret_cast<const cx<T>*>(b->gates), b->gate_n, ansatz,
                                                      reinterpret_cast<cx<T>*>(b->arena), b->bonds_d,
                                                      b->discarded_d, b->status_d);
    timing_end(b);
    CUDA_TRY(cudaGetLastError());
    count_launch();
    return MPS_OK;
}

}  // namespace

mps_status launch_ladder_mpo(mps_batch* b, const double* pixels, int ansatz) {
    return b->prec == MPS_FP64 ? launch_mpo_t<double>(b, pixels, ansatz) : launch_mpo_t<float>(b, pixels, ansatz);
}

}  // namespace mpsano
