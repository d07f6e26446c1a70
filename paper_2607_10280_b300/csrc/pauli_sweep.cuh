// Pauli cache as one right-to-left sweep per image (Sec. II.C, Eq. 5).
//
// pauli_kernel gives a team one grid column of one image and carries two closing
// matrices at a time, so each of its products is a 16 x 16 complex GEMM that the team
// splits into 2 x 2 register tiles: it spends more issue slots on operand loads, offsets
// and loop control than on multiply-adds.  pauli_sweep_kernel gives a CTA a whole image
// and walks its chain from site n-1 down to site 0.  Arriving at site k it holds
//   R      the right environment R_k (formed by the sweep itself: the environment kernel
//          runs only the left chains of META_LENV images),
//   slots  the closings Q_o = (M_o, C_Z,o) of the sites o > k that still have a pair to
//          close further left, each carried to the bond (k, k+1): origins k+1 .. k+p
//          with the H+V pairs, k+1 .. k+p+1 with the diagonal sets as well (slot o mod ns),
// and then
//   1. forms the left blocks E_a of site k (with L_k for a META_LENV image; at its
//      half-structured sites the left chain stored them, F'_k, on its way);
//   2. closes, one warp per closing, <E_a, R_k> (the single-site terms) and the pairs
//      (k, o) for o = k+1 (horizontal), k+p (vertical), k+p+1 and k+p-1 (the diagonal
//      sets), with the closings of o as carried;
//   3. transfers R and every carried closing that still has a pair further left through
//      site k in two stacked products
//        S_s = [R; M_1; C_Z,1; M_2; ...] A^{sT}       (s = 0, 1: one half of the CTA each)
//        [R_{k-1}, C_Z,k, M_1', C_Z,1', ...] = sum_s conj(A^s) S_s
//      (rows l, l' of a carried closing in the same half of the left bond only, when
//      its next use is a transfer through a half-structured site), and forms the
//      closings of site k from the R rows of S: M_k = 2 conj(A^0) S_1,
//      C_Z,k = conj(A^0) S_0 - conj(A^1) S_1.
// With 13 or more matrices in one product a thread holds a 7 x 4 (first product) or a
// 2 x 9 (second) tile of accumulators.  Every output is accumulated in the order of
// renv_kernel and pauli_kernel, so the two paths give the same bits.
// <psi|psi> = R_{-1} is known only after site 0, so the sweep writes the pair values
// unnormalised and scales them at its end (the [0][0] entry, 1, excepted).
#pragma once
#include "pauli.cuh"

namespace mpsano {

// Register-tile caps (complex accumulators per thread) of the first and second product.
#ifndef MPS_SWEEP_TILE1
#define MPS_SWEEP_TILE1 16
#endif
#ifndef MPS_SWEEP_TILE2
#define MPS_SWEEP_TILE2 24
#endif

// Carried-closing slots for images of side p: origins k+1 .. k+p are live at site k with
// the H+V pairs (the last one closes there), one more with the diagonal sets.
__host__ __device__ constexpr int sweep_slots(int p, bool diag) { return p + (diag ? 1 : 0); }

__host__ __device__ constexpr int sweep_imax(int a, int b) { return a > b ? a : b; }
__host__ __device__ constexpr int sweep_imin(int a, int b) { return a < b ? a : b; }

// Layout of a sweep CTA's shared memory (elements of E unless noted):
//   A (two buffers of 2 MAT: site k, and site k-1 arriving by cp.async) | L (MAT: L_k,
//   then L_{k-1} arriving) | R (MAT) | slots (ns x 2 MAT: M at +0, C_Z at +MAT) | S (two
//   planes of srows rows of stride CS; the left blocks use the same space) | bonds and
//   tables (ints) | dot sums (5 sets x 12) and single-site sums (3 per site) (scalars)
// HALF: every image is half-structured, so a carried closing needs h = D_r / 2 rows of a
// plane at a site with D_r >= HALF_SPLIT_MIN (dense sites then have D_r < that).
template <typename E, int CHI, bool HALF>
struct SweepLayout {
    using T = typename elem_traits<E>::scalar;
    static constexpr int CS = CHI + 1, MAT = CHI * CS, ZS = 2 * CHI + 1;
    // the R block and two blocks per carried closing (at most ns - 1 are transferred)
    __host__ __device__ static constexpr int srows(int ns) {
        return HALF ? sweep_imax(CHI * ns, sweep_imin(CHI, HALF_SPLIT_MIN - 1) * (2 * ns - 1))
                    : CHI * (2 * ns - 1);
    }
    __host__ __device__ static constexpr int s_elems(int ns) { return sweep_imax(2 * srows(ns) * CS, 3 * CHI * ZS); }
    static constexpr int MAXB = 36;                    // blocks per product (ns <= 18)
    static constexpr int TAB = 32 + 4 * MAXB;          // ints
    static constexpr int DOTS = 5 * 12;                // scalars
    static constexpr int OFF_A0 = 0, OFF_A1 = 2 * MAT, OFF_L = 4 * MAT, OFF_R = 5 * MAT, OFF_SLOT = 6 * MAT;
    __host__ __device__ static constexpr size_t elems(int ns) { return (size_t)(OFF_SLOT + 2 * ns * MAT + s_elems(ns)); }
    __host__ __device__ static constexpr size_t bytes(int ns, int n_max) {
        return sizeof(E) * elems(ns) + sizeof(int) * (TAB + (size_t)n_max + 1) +
               sizeof(T) * (DOTS + 3 * (size_t)n_max);
    }
};

// Table entries (ints) written by warp 0 at each site.
enum : int {
    SW_NSETS = 0,   // closing sets, set 0 being <E_a, R_k>
    SW_NG1 = 1,     // blocks of the first product (R first)
    SW_NF = 3,      // full blocks of the second product (R_{k-1} first)
    SW_ND = 4,      // diagonal-block-only blocks of the second product
    SW_NEW = 5,     // offset of the slot receiving the closings of site k, or -1
    SW_ORIG = 8,    // 8 .. 11: origin of closing set 1 .. 4
    SW_PAIR = 12,   // 12 .. 15: its pair index
    SW_G1 = 32,                 // source offset of each block of the first product
    SW_G2ROW = 32 + 36,         // S row of each block of the second product
    SW_G2DST = 32 + 72          // its destination offset
};

// floor(t / d) for t < 2048 and 1 <= d <= 32 as (t * m) >> 16, m = ceil(2^16 / d): the
// error t (m - 2^16 / d) / 2^16 < 1/32 <= 1/d never carries across an integer.
__host__ __device__ __forceinline__ int sweep_recip(int d) { return (65536 + d - 1) / d; }
__device__ __forceinline__ int sweep_div(int t, int m) { return (t * m) >> 16; }

// Left chains of the META_LENV images for the sweep, one CTA of NTHR threads per image
// (the environment kernel gives a chain one warp and runs it beside the right chain):
// L_k into lenv and the compact left blocks F'_k of the half-structured sites into fblk,
// env_stride elements per image.
template <typename T, int CHI, int NTHR, bool REAL>
__global__ void __launch_bounds__(NTHR) lenv_kernel(const ImageMeta* __restrict__ meta, int n_images,
                                                    const cx<T>* __restrict__ arena,
                                                    const int32_t* __restrict__ bonds, cx<T>* __restrict__ lenv_c,
                                                    cx<T>* __restrict__ fblk_c, int64_t env_stride) {
    using E = std::conditional_t<REAL, T, cx<T>>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int img = blockIdx.x;
    if (img >= n_images) return;
    const ImageMeta mt = meta[img];
    if (!(mt.flags & META_LENV)) return;
    lenv_image<E, CHI, true, NTHR>(mt, arena, bonds, reinterpret_cast<E*>(lenv_c) + (size_t)img * env_stride,
                                   reinterpret_cast<E*>(fblk_c) + (size_t)img * env_stride,
                                   reinterpret_cast<E*>(smem_raw), threadIdx.x);
}

// One CTA of NTHR threads per image.  lenv: left environments (META_LENV images), as
// written by renv_kernel; norms: <psi|psi> per image (written here); out: the Pauli
// cache; ns, n_max: the slots and the most sites of any image the launch was sized for.
template <typename T, int CHI, int NTHR, bool DIAG, bool REAL, bool HALF>
__global__ void __launch_bounds__(NTHR, (sizeof(T) == 4 && CHI <= 16 && NTHR <= 128) ? 3 : 1) pauli_sweep_kernel(
        const ImageMeta* __restrict__ meta, int n_images, const cx<T>* __restrict__ arena,
        const int32_t* __restrict__ bonds, const cx<T>* __restrict__ lenv_c, const cx<T>* __restrict__ fblk_c,
        int64_t env_stride, T* __restrict__ norms, T* __restrict__ out, int ns, int n_max, int* status) {
    using E = std::conditional_t<REAL, T, cx<T>>;
    using Lay = SweepLayout<E, CHI, HALF>;
    constexpr int CS = Lay::CS, MAT = Lay::MAT;
    constexpr int HT = NTHR / 2;   // threads of one half of the CTA
    static_assert(HT >= 32 && (HT & (HT - 1)) == 0, "two halves of whole warps");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int img = blockIdx.x;
    if (img >= n_images) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int grp = tid / HT, gl = tid & (HT - 1);

    E* base = reinterpret_cast<E*>(smem_raw);
    constexpr int OFF_R = Lay::OFF_R, OFF_SLOT = Lay::OFF_SLOT;
    const int off_s = OFF_SLOT + 2 * ns * MAT;
    const int srows = Lay::srows(ns);
    const int plane = srows * CS;                    // elements of one plane of S
    E* R = base + OFF_R;
    E* Ls = base + Lay::OFF_L;
    E* S = base + off_s;
    int* tab = reinterpret_cast<int*>(base + Lay::elems(ns));
    int* bd = tab + Lay::TAB;                        // the image's bond dimensions
    T* dots = reinterpret_cast<T*>(bd + n_max + 1);
    T* singles = dots + Lay::DOTS;

    const ImageMeta mt = meta[img];
    const int p = mt.p, n = mt.n, ld = mt.ld;
    const bool half_img = (mt.flags & META_HALF) != 0;
    if (sweep_slots(p, DIAG) > ns || n > n_max || (HALF && !half_img)) {
        if (tid == 0) raise_status(status, DEV_BAD_SHAPE);
        return;
    }
    for (int i = tid; i <= n; i += NTHR) bd[i] = bonds[mt.bond_off + i];
    const cx<T>* sites = arena + mt.site_off;
    const E* lenv = reinterpret_cast<const E*>(lenv_c);
    const E* lgb = (lenv && (mt.flags & META_LENV)) ? lenv + (size_t)img * env_stride : nullptr;
    // the compact left blocks F'_k the left chain stored for the half-structured sites
    const E* fgb = (lgb && fblk_c) ? reinterpret_cast<const E*>(fblk_c) + (size_t)img * env_stride : nullptr;
    // site k into A buffer (n-1-k) % 2 and L_k into Ls, by cp.async (real elements take
    // the real parts of the complex64 storage)
    auto prefetch_site = [=](int k) {
        E* dstA = base + (((n - 1 - k) & 1) ? Lay::OFF_A1 : Lay::OFF_A0);
        const cx<T>* src = sites + (size_t)k * 2 * ld * ld;
        team_for_2d<NTHR, 4>(2 * bd[k], bd[k + 1], tid, [=](int r, int c) {
            if constexpr (REAL) cp_async_re(dstA + r * CS + c, src + r * ld + c);
            else cp_async_same(dstA + r * CS + c, src + r * ld + c);
        });
    };
    auto half_at = [half_img, n, bd](int i) { return half_img && i < n - 1 && bd[i + 1] >= 2; };
    // site k's left blocks come ready from the left chain (F'_k), or are formed here from L_k
    auto fpre = [=](int k) { return fgb != nullptr && half_at(k); };
    auto prefetch_lenv = [=](int k) {
        const bool f = fpre(k);
        const E* src = (f ? fgb : lgb) + (size_t)k * CHI * CHI;
        const int D = f ? bd[k + 1] : bd[k];
        team_for_2d<NTHR, 4>(D, D, tid, [=](int r, int c) { cp_async_same(Ls + r * CS + c, src + r * CHI + c); });
    };
    auto half_tr = [half_img, n, bd](int i) { return half_img && i < n - 1 && bd[i + 1] >= HALF_SPLIT_MIN; };
    T* outp = out + (size_t)(DIAG ? mt.pair_off_d : mt.pair_off) * 16;
    const int nh = p * (p - 1);
    const int base_dd = 2 * p * (p - 1);
    const int base_da = base_dd + (p - 1) * (p - 1);
    const int npairs = DIAG ? base_da + (p - 1) * (p - 1) : base_dd;

    // first (leftmost) site at which origin o closes a pair, n if none; whether o
    // closes one at site u
    auto last_use = [p, n](int o) {
        const int r = o / p, c = o - r * p;
        int u = n;
        if (c >= 1) u = o - 1;
        if (r >= 1) u = o - p;
        if (DIAG && r >= 1 && c >= 1) u = o - p - 1;
        return u;
    };
    auto used_at = [p](int o, int u) {
        const int r = o / p, c = o - r * p;
        if (c >= 1 && u == o - 1) return true;
        if (r >= 1 && u == o - p) return true;
        if (DIAG && r >= 1 && c <= p - 2 && u == o - p + 1) return true;
        if (DIAG && r >= 1 && c >= 1 && u == o - p - 1) return true;
        return false;
    };
    auto slot_of = [ns](int o) { return OFF_SLOT + (o % ns) * 2 * MAT; };

    if (tid == 0) R[0] = eone<E>();
    __syncthreads();
    for (int i = 0; i <= n; ++i)
        if (bd[i] > CHI || bd[i] < 1) {
            if (tid == 0) raise_status(status, DEV_BOND_OVERFLOW);
            return;
        }
    prefetch_site(n - 1);
    if (lgb) prefetch_lenv(n - 1);
    cp_async_commit();
    for (int k = n - 1; k >= 0; --k) {
        const int row = k / p, col = k - row * p;
        const int Dl = bd[k], Dr = bd[k + 1];
        const E* A = base + (((n - 1 - k) & 1) ? Lay::OFF_A1 : Lay::OFF_A0);
        const bool htr = half_tr(k);
        const int h = Dr >> 1;
        const int hs = htr ? h : 0;              // column offset of the odd segment's half
        const int K1 = htr ? h : Dr;             // depth of one segment (= rows of a carried block)
        // diagonal blocks alone for a carried closing whose next use is the transfer
        // through site k-1 (half-structured there)
        const bool dg = k >= 1 && half_tr(k - 1) && (Dl & 1) == 0;
        const bool has_new = k >= 1 && last_use(k) < k;
        cp_async_wait_all();
        if (warp == 0) {
            // carried closings: lane l looks at origin k+1+l
            const int o = k + 1 + lane;
            const bool carried = lane < ns - 1 && o <= n - 1 && last_use(o) < k;
            const bool full = carried && (!dg || used_at(o, k - 1));
            const unsigned cm = __ballot_sync(0xffffffffu, carried), fm = __ballot_sync(0xffffffffu, full);
            const unsigned lt = (1u << lane) - 1u;
            const int nc = __popc(cm), nfc = __popc(fm);
            if (carried) {
                const int j = __popc(cm & lt);
                tab[SW_G1 + 1 + 2 * j] = slot_of(o);
                tab[SW_G1 + 2 + 2 * j] = slot_of(o) + MAT;
                // second product: full blocks (R_{k-1}, then the closings used at k-1 or
                // not followed by a half-structured transfer), then diagonal-only blocks
                const int pos = full ? 1 + 2 * __popc(fm & lt) : 1 + 2 * nfc + 2 * __popc(cm & ~fm & lt);
                tab[SW_G2ROW + pos] = Dr + 2 * j * K1;
                tab[SW_G2ROW + pos + 1] = Dr + (2 * j + 1) * K1;
                tab[SW_G2DST + pos] = slot_of(o);
                tab[SW_G2DST + pos + 1] = slot_of(o) + MAT;
            }
            if (lane == 0) {
                tab[SW_G1] = OFF_R;
                tab[SW_NG1] = 1 + 2 * nc;
                tab[SW_G2ROW] = 0;
                tab[SW_G2DST] = OFF_R;
                tab[SW_NF] = 1 + 2 * nfc;
                tab[SW_ND] = 2 * (nc - nfc);
                tab[SW_NEW] = has_new ? slot_of(k) : -1;
                // closing sets: <E_a, R_k>, then the pairs (k, o)
                int ns_ = 1;
                if (col < p - 1) { tab[SW_ORIG + ns_ - 1] = k + 1; tab[SW_PAIR + ns_ - 1] = row * (p - 1) + col; ++ns_; }
                if (row < p - 1) { tab[SW_ORIG + ns_ - 1] = k + p; tab[SW_PAIR + ns_ - 1] = nh + k; ++ns_; }
                if (DIAG && row < p - 1 && col < p - 1) {
                    tab[SW_ORIG + ns_ - 1] = k + p + 1; tab[SW_PAIR + ns_ - 1] = base_dd + row * (p - 1) + col; ++ns_;
                }
                if (DIAG && row < p - 1 && col >= 1) {
                    tab[SW_ORIG + ns_ - 1] = k + p - 1; tab[SW_PAIR + ns_ - 1] = base_da + row * (p - 1) + col - 1; ++ns_;
                }
                tab[SW_NSETS] = ns_;
            }
        }
        __syncthreads();
        // site k-1 into the other A buffer (last read by the transfer through site k+1)
        if (k >= 1) prefetch_site(k - 1);
        cp_async_commit();
        // 1. left blocks of site k: F'_k as stored by the left chain (in Ls), or formed here
        //    into S (from L_k in Ls, or the identity)
        const bool fp = fpre(k);
        if (!fp) {
            left_blocks_env<E, CHI, NTHR, CS>(A, lgb ? Ls : nullptr, S, Dl, Dr, tid, half_at(k));
            __syncthreads();
        }
        // 2. closings, one warp per set (sums into dots, written out after the next barrier)
        const int nsets = tab[SW_NSETS];
        for (int set = warp; set < nsets; set += NTHR / 32) {
            const E* C = set == 0 ? nullptr : base + slot_of(tab[SW_ORIG + set - 1]);
            T d[12];
            left_dots_warp<E, CHI>(fp ? Ls : S + CHI * Lay::ZS, fp ? CS : Lay::ZS, C, R, Dr, d, lane, half_at(k));
            if (lane == 0)
#pragma unroll
                for (int i = 0; i < 12; ++i) dots[12 * set + i] = d[i];
        }
        // the first product overwrites S (which holds the blocks unless they came stored)
        if (!fp) __syncthreads();
        // 3. transfer through site k
        const int g1 = tab[SW_NG1];
        const int Ms = Dr + (g1 - 1) * K1;
        if (Ms > srows) {
            if (tid == 0) raise_status(status, DEV_SMEM_OVERFLOW);
            return;
        }
        {
            // S_s[m][l'] = sum_k X_m[s hs + k] A[2l'+s][s hs + k], X_m the m-th row of the
            // stack; R's rows are stored rotated by s hs (row t of plane s is row
            // (t + s hs) mod D_r), so that every block of the second product finds the
            // rows of its odd segment at the same plane offset
            const int s = grp;
            const int mk = sweep_recip(K1);
            // tile rows: the R block and 2 (ns - 1) carried blocks of half a bond each at a
            // half-structured site (7 CHI rows for 7 x 7 images with H+V pairs)
            using Tl = Tile<E, (DIAG ? 8 : 7) * CHI, CHI, HT, MPS_SWEEP_TILE1>;
            const int* g1src = tab + SW_G1;
            team_gemm<E, Tl::MT, Tl::NT, Tl::TM, Tl::TN, 1, false, 2>(
                base,
                [=](int m) {
                    if (m < Dr) {
                        int r = m + s * hs;
                        if (r >= Dr) r -= Dr;
                        return OFF_R + r * CS + s * hs;
                    }
                    const int t = m - Dr, jb = sweep_div(t, mk), i = t - jb * K1;
                    return g1src[1 + jb] + (s * hs + i) * CS + s * hs;
                },
                1, 0, A, [=](int nn) { return (2 * nn + s) * CS + s * hs; }, 1, 0, Ms, Dl, K1,
                [](int nn) { return nn; }, [=](int m, int sn, E v) { S[s * plane + m * CS + sn] = v; }, gl);
        }
        __syncthreads();
        // Ls has been read: the left blocks (or L) of site k-1 into it
        if (lgb && k >= 1) prefetch_lenv(k - 1);
        cp_async_commit();
        if (tid < 3) singles[3 * k + tid] = dots[4 * tid + 3];
        if (tid < 16 * (nsets - 1)) {
            const int set = 1 + (tid >> 4), e = tid & 15, a = e >> 2, b = e & 3;
            const int o = tab[SW_ORIG + set - 1];
            T v;
            if (a == 0 && b == 0) v = T(1);
            else if (b == 0) v = dots[4 * (a - 1) + 3];
            else if (a == 0) v = singles[3 * o + b - 1];
            else v = dots[12 * set + 4 * (a - 1) + (b - 1)];
            outp[(size_t)tab[SW_PAIR + set - 1] * 16 + e] = v;
        }
        {
            // second product, rows l in half q of the left bond (one half of the CTA each)
            const int nf = tab[SW_NF], nd = tab[SW_ND];
            const int g = dg ? Dl >> 1 : (Dl + 1) >> 1;
            const int q = grp, q0 = q ? g : 0, Mq = q ? Dl - g : g;
            const int Nq = nf * Dl + nd * g;
            const int* rowb = tab + SW_G2ROW;
            const int* dst = tab + SW_G2DST;
            const int mD = sweep_recip(Dl), mg = sweep_recip(g > 0 ? g : 1);
            // column nn -> (block, column of the block)
            auto colb = [=](int nn, int& lp) {
                if (nn < nf * Dl) {
                    const int fb = sweep_div(nn, mD);
                    lp = nn - fb * Dl;
                    return fb;
                }
                const int t = nn - nf * Dl, db = sweep_div(t, mg);
                lp = q0 + t - db * g;
                return nf + db;
            };
            // columns: R_{k-1}, one full carried pair and the rest diagonal-only (8 CHI for
            // 7 x 7 images with H+V pairs)
            using Tl = Tile<E, CHI / 2, (DIAG ? 9 : 8) * CHI, HT, MPS_SWEEP_TILE2>;
            team_gemm<E, Tl::MT, Tl::NT, Tl::TM, Tl::TN, 2, true, 2>(
                A, [=](int l) { return 2 * (q0 + l) * CS; }, 1, CS + hs,
                S, [=](int nn) { int lp; const int b = colb(nn, lp); return rowb[b] * CS + lp; }, CS, plane, Mq, Nq,
                K1, [=](int nn) { int lp; const int b = colb(nn, lp); return dst[b] + lp; },
                [=](int m, int sn, E v) { base[sn + (q0 + m) * CS] = v; }, gl);
            // closings of site k from the R rows of S: M_k = 2 conj(A^0) S_1 (the R rows of
            // half 0, stored from row D_r - hs of plane 1), C_Z,k = conj(A^0) S_0 - conj(A^1) S_1
            const int nw = tab[SW_NEW];
            if (nw >= 0) {
                const int rot1 = htr ? Dr - hs : 0;
                using Tm = Tile<E, CHI, CHI, NTHR>;
                team_gemm<E, Tm::MT, Tm::NT, Tm::TM, Tm::TN, 1, true, 2>(
                    A, [](int l) { return 2 * l * CS; }, 1, 0, S,
                    [=](int nn) { return plane + rot1 * CS + nn; }, CS, 0, Dl, Dl, K1, [](int nn) { return nn; },
                    [=](int l, int sn, E v) { base[nw + l * CS + sn] = v + v; }, tid);
                team_gemm<E, Tm::MT, Tm::NT, Tm::TM, Tm::TN, 2, true, 2, true>(
                    A, [](int l) { return 2 * l * CS; }, 1, CS + hs, S, [](int nn) { return nn; }, CS, plane, Dl,
                    Dl, K1, [](int nn) { return nn; },
                    [=](int l, int sn, E v) { base[nw + MAT + l * CS + sn] = v; }, tid);
            }
        }
        __syncthreads();
    }
    // <psi|psi> = R_{-1}; scale the sweep's unnormalised values
    const T nrm = ereal(R[0]);
    const T inv_norm = T(1) / nrm;
    if (tid == 0) norms[img] = nrm;
    for (int i = tid; i < npairs * 16; i += NTHR)
        if (i & 15) outp[i] = outp[i] * inv_norm;
}

}  // namespace mpsano
