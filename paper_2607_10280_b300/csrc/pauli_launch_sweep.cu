// Launches of the per-image sweep Pauli kernel (pauli_sweep.cuh) under the mixed
// precisions: complex64 elements, or real ones for a real state, bonds up to 16.
#include <algorithm>

#include "batch.h"
#include "pauli_sweep.cuh"

namespace mpsano {
namespace {

// threads per image (three images per SM fit the shared memory of the 7x7, bond-16 case)
#ifndef MPS_SWEEP_THREADS
#define MPS_SWEEP_THREADS 128
#endif
constexpr int SWEEP_THREADS = MPS_SWEEP_THREADS;
// threads per left chain
#ifndef MPS_LENV_THREADS
#define MPS_LENV_THREADS 64
#endif
constexpr int LENV_THREADS = MPS_LENV_THREADS;

template <int CHI, bool DIAG, bool REAL, bool HALF>
mps_status launch_sweep(mps_batch* b, void* out, int ns, size_t smem) {
    using E = std::conditional_t<REAL, float, cx<float>>;
    if (b->any_lenv) {
        // left chains of the operator-product images (the sweep forms the right
        // environments itself), storing the compact left blocks of their half-structured
        // sites in the otherwise unused right-environment buffer
        using Lp = PauliLayout<E, CHI>;
        auto lk = lenv_kernel<float, CHI, LENV_THREADS, REAL>;
        CUDA_TRY(cudaFuncSetAttribute(lk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Lp::env_bytes));
        timing_begin(b, KIND_RENV);
        lk<<<b->B, LENV_THREADS, Lp::env_bytes, b->stream>>>(
            b->meta_d, b->B, reinterpret_cast<const cx<float>*>(b->arena), b->bonds_d,
            reinterpret_cast<cx<float>*>(b->lenv), reinterpret_cast<cx<float>*>(b->renv), b->renv_stride);
        timing_end(b);
        CUDA_TRY(cudaGetLastError());
        count_launch();
    }
    auto sk = pauli_sweep_kernel<float, CHI, SWEEP_THREADS, DIAG, REAL, HALF>;
    CUDA_TRY(cudaFuncSetAttribute(sk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    timing_begin(b, KIND_PAULI);
    sk<<<b->B, SWEEP_THREADS, smem, b->stream>>>(
        b->meta_d, b->B, reinterpret_cast<const cx<float>*>(b->arena), b->bonds_d,
        reinterpret_cast<const cx<float>*>(b->any_lenv ? b->lenv : nullptr),
        reinterpret_cast<const cx<float>*>(b->any_lenv ? b->renv : nullptr), b->renv_stride,
        reinterpret_cast<float*>(b->norms), reinterpret_cast<float*>(out), ns, b->n_max, b->status_d);
    timing_end(b);
    CUDA_TRY(cudaGetLastError());
    count_launch();
    return MPS_OK;
}

template <int CHI, bool DIAG, bool REAL, bool HALF>
bool sweep_fits(mps_batch* b, int ns, size_t* smem) {
    using E = std::conditional_t<REAL, float, cx<float>>;
    *smem = SweepLayout<E, CHI, HALF>::bytes(ns, b->n_max);
    return ns <= SweepLayout<E, CHI, HALF>::MAXB / 2 && *smem <= (size_t)smem_optin_limit();
}

template <int CHI, bool DIAG>
mps_status try_sweep(mps_batch* b, void* out, int ns, bool* taken) {
    size_t smem = 0;
    *taken = false;
    if (b->real) {
        if (!sweep_fits<CHI, DIAG, true, false>(b, ns, &smem)) return MPS_OK;
        *taken = true;
        return launch_sweep<CHI, DIAG, true, false>(b, out, ns, smem);
    }
    if (b->all_half) {
        if (!sweep_fits<CHI, DIAG, false, true>(b, ns, &smem)) return MPS_OK;
        *taken = true;
        return launch_sweep<CHI, DIAG, false, true>(b, out, ns, smem);
    }
    if (!sweep_fits<CHI, DIAG, false, false>(b, ns, &smem)) return MPS_OK;
    *taken = true;
    return launch_sweep<CHI, DIAG, false, false>(b, out, ns, smem);
}

}  // namespace

mps_status launch_pauli_sweep(mps_batch* b, void* out, bool diag, bool* taken) {
    *taken = false;
    if (b->pauli_sweep == MPS_PAULI_COLUMN || b->B == 0) return MPS_OK;
    int p_max = 1, p_min = 1 << 30;
    for (const ImageMeta& m : b->meta_h) {
        p_max = std::max(p_max, (int)m.p);
        p_min = std::min(p_min, (int)m.p);
    }
    // the automatic choice: batches of equal-size half-structured images (operator-product
    // ladder images), where the sweep's stacked products and stored left blocks pay; the
    // column walk measured faster on dense sites (fewer sweep CTAs fit an SM) and on
    // mixed sizes (slots sized for the largest image, whose chain sets the time)
    if (b->pauli_sweep == MPS_PAULI_AUTO && (!b->all_half || p_min != p_max)) return MPS_OK;
    const int ns = sweep_slots(p_max, diag);
    switch (b->chi_tpl) {
        case 4: return diag ? try_sweep<4, true>(b, out, ns, taken) : try_sweep<4, false>(b, out, ns, taken);
        case 8: return diag ? try_sweep<8, true>(b, out, ns, taken) : try_sweep<8, false>(b, out, ns, taken);
        case 16: return diag ? try_sweep<16, true>(b, out, ns, taken) : try_sweep<16, false>(b, out, ns, taken);
    }
    return MPS_OK;
}

}  // namespace mpsano
