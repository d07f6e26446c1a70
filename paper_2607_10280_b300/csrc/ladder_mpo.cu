// Ladder circuit as an operator product (Sec. II.B, Eq. 3), and the left environments
// it then needs.
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
// The result is not left-canonical (a layer's operator keeps left orthonormality only
// where the incoming parity is summed, not at site 0), so the Pauli kernel contracts
// the left environments L_k = sum_s A_{k-1}^{s dagger} L_{k-1} A_{k-1}^s (L_0 = 1)
// that lenv_kernel writes, marked per image by META_LENV.
#include <algorithm>

#include "batch.h"
#include "circuit.cuh"
#include "pauli.cuh"

namespace mpsano {
namespace {

constexpr int MPO_MAXB = 16;                       // largest bond 2^L of this path (L <= 4)
constexpr int MPO_BUF = MPO_MAXB * 2 * MPO_MAXB;   // one site tensor, compact [Dl][2][Dr]
constexpr int MPO_WARPS = 4;

// One CTA per image of order[0 .. n_images), its warps taking the sites in turn.
template <typename T>
__global__ void __launch_bounds__(32 * MPO_WARPS) ladder_mpo_kernel(
    const ImageMeta* __restrict__ meta, int n_images, const int32_t* __restrict__ order,
    const double* __restrict__ pixels, const cx<T>* __restrict__ gates, int gn,
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
        // encoding R_Y(pi x) on |0>
        if (lane == 0) {
            double sn, cs;
            sincos(0.5 * M_PI * px[k], &sn, &cs);
            cur[0] = mk<T>(T(cs), T(0));
            cur[1] = mk<T>(T(sn), T(0));
        }
        int Dl = 1, Dr = 1;
        for (int layer = 0; layer < L; ++layer) {
            __syncwarp();
            // the layer's one-qubit gate on the physical index
            const Gate1<T> g = table_gate<T>(gates, gn, 0, layer, img, k);
            for (int e = lane; e < Dl * Dr; e += 32) {
                const int l = e / Dr, r = e - l * Dr;
                const cx<T> a0 = cur[(2 * l) * Dr + r], a1 = cur[(2 * l + 1) * Dr + r];
                cur[(2 * l) * Dr + r] = cdot2(g.u00, a0, g.u01, a1);
                cur[(2 * l + 1) * Dr + r] = cdot2(g.u10, a0, g.u11, a1);
            }
            __syncwarp();
            // the layer's CNOT ladder: new bond index = old index + old dimension * parity
            const int Dl2 = k == 0 ? Dl : 2 * Dl;
            const int Dr2 = k == n - 1 ? Dr : 2 * Dr;
            for (int e = lane; e < Dl2 * 2 * Dr2; e += 32) {
                const int l2 = e / (2 * Dr2), rem = e - l2 * 2 * Dr2;
                const int s = rem / Dr2, r2 = rem - s * Dr2;
                const int a = l2 / Dl, l = l2 - a * Dl;       // a = 0 at site 0 (Dl2 = Dl)
                cx<T> v;
                if (k == n - 1) {
                    v = cur[(2 * l + (a ^ s)) * Dr + r2];
                } else {
                    const int b = r2 / Dr, r = r2 - b * Dr;
                    v = s == b ? cur[(2 * l + (a ^ b)) * Dr + r] : czero<T>();
                }
                nxt[e] = v;
            }
            cx<T>* t = cur; cur = nxt; nxt = t;
            Dl = Dl2;
            Dr = Dr2;
        }
        __syncwarp();
        cx<T>* dst = sites + (size_t)k * 2 * ld * ld;
        for (int e = lane; e < Dl * 2 * Dr; e += 32) {
            const int row = e / Dr, r = e - row * Dr;
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

// Left environments of the images flagged META_LENV (one warp per image; the others
// return at once): L_0 = 1 and L_{k+1}[r][r'] = sum_{l,l',s} conj(A_k[l][s][r])
// L_k[l][l'] A_k[l'][s][r'], stored like the right environments (L_k, D_k x D_k, at
// k * CHI * CHI of the image's block; D_k = left bond of site k).
template <typename T, int CHI>
__global__ void __launch_bounds__(32) lenv_kernel(const ImageMeta* __restrict__ meta, int n_images,
                                                   const cx<T>* __restrict__ arena,
                                                   const int32_t* __restrict__ bonds,
                                                   cx<T>* __restrict__ lenv, int64_t stride) {
    using Lay = PauliLayout<T, CHI>;
    constexpr int CS = Lay::CS, MAT = Lay::MAT, ZS = Lay::ZS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x;
    const int img = blockIdx.x;
    if (img >= n_images) return;
    const ImageMeta mt = meta[img];
    if (!(mt.flags & META_LENV)) return;
    cx<T>* base = reinterpret_cast<cx<T>*>(smem_raw);
    cx<T>* A = base;             // 2 MAT
    cx<T>* Lm = base + 2 * MAT;  // MAT
    cx<T>* S = base + 3 * MAT;   // CHI rows x ZS
    const int n = mt.n, ld = mt.ld;
    const int32_t* bd = bonds + mt.bond_off;
    const cx<T>* sites = arena + mt.site_off;
    cx<T>* lg = lenv + (size_t)img * stride;
    if (lane == 0) Lm[0] = mk<T>(T(1), T(0));
    __syncwarp();
    for (int k = 0; k < n; ++k) {
        const int Dl = bd[k], Dr = bd[k + 1];
        cx<T>* dst = lg + (size_t)k * CHI * CHI;
        team_for_2d<32, 4>(Dl, Dl, lane, [&](int r, int c) { dst[r * CHI + c] = Lm[r * CS + c]; });
        load_site_p<T, CS, 32>(A, sites + (size_t)k * 2 * ld * ld, ld, Dl, Dr, lane);
        __syncwarp();
        // S[l][s Dr + r] = sum_l' L[l][l'] A[2l'+s][r]
        {
            using Tl = Tile<T, CHI, 2 * CHI, 32>;
            team_gemm<T, Tl::MT, Tl::NT, Tl::TM, Tl::TN, 1, false, 1>(
                Lm, [](int l) { return l * CS; }, 1, 0, A, [Dr](int nn) { return (nn / Dr) * CS + (nn % Dr); }, 2 * CS, 0,
                Dl, 2 * Dr, Dl, [](int nn) { return nn; }, [S](int l, int sn, cx<T> v) { S[l * ZS + sn] = v; }, lane);
        }
        __syncwarp();
        // L'[r][r'] = sum_{l,s} conj(A[2l+s][r]) S[l][s Dr + r']
        {
            using Tl = Tile<T, CHI, CHI, 32>;
            team_gemm<T, Tl::MT, Tl::NT, Tl::TM, Tl::TN, 2, true, 1>(
                A, [](int r) { return r; }, 2 * CS, CS, S, [](int nn) { return nn; }, ZS, Dr, Dr, Dr, Dl,
                [](int nn) { return nn; }, [Lm](int r, int sn, cx<T> v) { Lm[r * CS + sn] = v; }, lane);
        }
        __syncwarp();
    }
}

template <typename T>
mps_status launch_mpo_t(mps_batch* b, const double* pixels) {
    auto k = ladder_mpo_kernel<T>;
    const size_t smem = sizeof(cx<T>) * 2 * MPO_BUF * MPO_WARPS;
    CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    timing_begin(b, KIND_CIRCUIT);
    k<<<b->run_count, 32 * MPO_WARPS, smem, b->stream>>>(b->meta_d, b->run_count, b->run_order, pixels,
                                                      reinterpret_cast<const cx<T>*>(b->gates), b->gate_n,
                                                      reinterpret_cast<cx<T>*>(b->arena), b->bonds_d,
                                                      b->discarded_d, b->status_d);
    timing_end(b);
    CUDA_TRY(cudaGetLastError());
    count_launch();
    return MPS_OK;
}

template <typename T, int CHI>
mps_status launch_lenv_t(mps_batch* b) {
    using Lay = PauliLayout<T, CHI>;
    const size_t smem = sizeof(cx<T>) * (3 * Lay::MAT + CHI * Lay::ZS);
    if (smem > (size_t)smem_optin_limit()) return fail(MPS_ERR_UNSUPPORTED, "left environments: %zu B shared memory", smem);
    auto k = lenv_kernel<T, CHI>;
    CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    timing_begin(b, KIND_RENV);
    k<<<b->B, 32, smem, b->stream>>>(b->meta_d, b->B, reinterpret_cast<const cx<T>*>(b->arena), b->bonds_d,
                                     reinterpret_cast<cx<T>*>(b->lenv), b->renv_stride);
    timing_end(b);
    CUDA_TRY(cudaGetLastError());
    count_launch();
    return MPS_OK;
}

template <typename T>
mps_status launch_lenv_b(mps_batch* b) {
    switch (b->chi_tpl) {
        case 4: return launch_lenv_t<T, 4>(b);
        case 8: return launch_lenv_t<T, 8>(b);
        case 16: return launch_lenv_t<T, 16>(b);
        case 32: return launch_lenv_t<T, 32>(b);
    }
    return fail(MPS_ERR_UNSUPPORTED, "bond dimension bucket %d not compiled", b->chi_tpl);
}

}  // namespace

mps_status launch_ladder_mpo(mps_batch* b, const double* pixels) {
    return b->prec == MPS_FP64 ? launch_mpo_t<double>(b, pixels) : launch_mpo_t<float>(b, pixels);
}

mps_status launch_lenv(mps_batch* b) {
    return b->prec == MPS_FP64 ? launch_lenv_b<double>(b) : launch_lenv_b<float>(b);
}

}  // namespace mpsano
