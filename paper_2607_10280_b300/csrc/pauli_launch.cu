// Right-environment and Pauli-cache kernel launches.
#include <algorithm>

#include "batch.h"
#include "pauli.cuh"

namespace mpsano {
namespace {

template <typename T, int CHI, int UW, bool DIAG, bool HALF = false>
mps_status launch_pauli_uw(mps_batch* b, void* out) {
    constexpr bool diag = DIAG;
    using Lay = PauliLayout<cx<T>, CHI, HALF>;
    const int limit = smem_optin_limit();
    const size_t smem = Lay::team_bytes(UW, diag);
    if (smem > (size_t)limit) return fail(MPS_ERR_UNSUPPORTED, "Pauli kernel shared memory %zu B", smem);
    auto pk = pauli_kernel<T, CHI, UW, DIAG, false, false, HALF>;
    CUDA_TRY(cudaFuncSetAttribute(pk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    timing_begin(b, KIND_PAULI);
    pk<<<b->n_units, 32 * UW, smem, b->stream>>>(
        b->meta_d, b->n_units, b->units_d, reinterpret_cast<const cx<T>*>(b->arena), b->bonds_d,
        reinterpret_cast<const cx<T>*>(b->renv), b->renv_stride,
        reinterpret_cast<const cx<T>*>(b->any_lenv ? b->lenv : nullptr),
        reinterpret_cast<const T*>(b->norms), reinterpret_cast<T*>(out), nullptr, b->status_d);
    timing_end(b);
    CUDA_TRY(cudaGetLastError());
    count_launch();
    return MPS_OK;
}

template <typename T, int CHI>
mps_status launch_pauli(mps_batch* b, void* out, bool diag) {
    using Lay = PauliLayout<cx<T>, CHI>;
    const int limit = smem_optin_limit();
    const size_t smem = Lay::env_bytes;
    if (smem > (size_t)limit) return fail(MPS_ERR_UNSUPPORTED, "environment kernel shared memory %zu B", smem);
    auto rk = renv_kernel<T, CHI>;
    CUDA_TRY(cudaFuncSetAttribute(rk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    timing_begin(b, KIND_RENV);
    // right environments of every image; with operator-product images also their left
    // environments, in the same launch (CTAs B .. 2B)
    rk<<<b->any_lenv ? 2 * b->B : b->B, 32, smem, b->stream>>>(
        b->meta_d, b->B, reinterpret_cast<const cx<T>*>(b->arena), b->bonds_d,
        reinterpret_cast<cx<T>*>(b->renv), b->renv_stride,
        reinterpret_cast<cx<T>*>(b->any_lenv ? b->lenv : nullptr), reinterpret_cast<T*>(b->norms), nullptr, 0, nullptr);
    timing_end(b);
    CUDA_TRY(cudaGetLastError());
    count_launch();
    // the diagonal pair sets are compiled for 2-warp teams only
    if (diag) return launch_pauli_uw<T, CHI, 2, true>(b, out);
    // every image half-structured (operator-product ladder images): the smaller scratch,
    // more resident teams
    if constexpr (sizeof(T) == 4) {
        if (b->all_half && b->pauli_warps == 2) return launch_pauli_uw<T, CHI, 2, false, true>(b, out);
    }
    switch (b->pauli_warps) {
        case 1: return launch_pauli_uw<T, CHI, 1, false>(b, out);
        case 4: return launch_pauli_uw<T, CHI, 4, false>(b, out);
        default: return launch_pauli_uw<T, CHI, 2, false>(b, out);
    }
}

template <typename T>
mps_status dispatch_pauli(mps_batch* b, void* out, bool diag) {
    if constexpr (sizeof(T) == 4) {
        // bonds up to 16: one sweep per image (pauli_sweep.cuh), where its buffers fit
        bool taken = false;
        const mps_status st = launch_pauli_sweep(b, out, diag, &taken);
        if (taken || st != MPS_OK) return st;
    }
    // a real state (paper ansatz) up to bond 32: real-element kernels
    if (sizeof(T) == 4 && b->real && b->chi_tpl <= 32) return launch_pauli_real(b, out, diag);
    switch (b->chi_tpl) {
        case 4: return launch_pauli<T, 4>(b, out, diag);
        case 8: return launch_pauli<T, 8>(b, out, diag);
        case 16: return launch_pauli<T, 16>(b, out, diag);
        case 32: return launch_pauli<T, 32>(b, out, diag);
        case 64:
        case 128: return launch_pauli_large(b, out, diag, sizeof(T) == 8);
    }
    return fail(MPS_ERR_UNSUPPORTED, "bond dimension bucket %d not compiled", b->chi_tpl);
}


}  // namespace

mps_status launch_pauli_fp64(mps_batch* b, void* out, bool diag) { return dispatch_pauli<double>(b, out, diag); }
mps_status launch_pauli_mixed(mps_batch* b, void* out, bool diag) { return dispatch_pauli<float>(b, out, diag); }

}  // namespace mpsano
