// Circuit-kernel launch templates (included by one .cu per precision).
#pragma once
#include <algorithm>

#include "batch.h"
#include "circuit.cuh"

namespace mpsano {
namespace {

template <typename T, typename TQ, int CHI, bool TRUNC>
mps_status launch_circuit(mps_batch* b, const double* pixels, const double* params, int params_n, int ansatz) {
    using Lay = CircuitLayout<T, TQ, CHI, TRUNC>;
    const int limit = smem_optin_limit();
    int ipc = std::max(1, b->images_per_cta);
    while (ipc > 1 && (size_t)ipc * Lay::bytes > (size_t)limit) --ipc;
    const size_t smem = (size_t)ipc * Lay::bytes;
    if (smem > (size_t)limit)
        return fail(MPS_ERR_UNSUPPORTED, "circuit kernel needs %zu B shared memory per warp (limit %d)",
                    Lay::bytes, limit);
    auto kern = circuit_kernel<T, TQ, CHI, TRUNC>;
    CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = (b->B + ipc - 1) / ipc;
    timing_begin(b, KIND_CIRCUIT);
    kern<<<grid, 32 * ipc, smem, b->stream>>>(b->meta_d, b->B, pixels, params, params_n, ansatz,
                                                reinterpret_cast<cx<T>*>(b->arena), b->bonds_d,
                                                b->discarded_d, b->status_d);
    timing_end(b);
    CUDA_TRY(cudaGetLastError());
    count_launch();
    return MPS_OK;
}

template <typename T, typename TQ, int CHI>
mps_status dispatch_trunc(mps_batch* b, bool trunc, const double* px, const double* pr, int pn, int an) {
    if (trunc) return launch_circuit<T, TQ, CHI, true>(b, px, pr, pn, an);
    return launch_circuit<T, TQ, CHI, false>(b, px, pr, pn, an);
}

template <typename T, typename TQ>
mps_status dispatch_chi(mps_batch* b, int chi_tpl, bool trunc, const double* px, const double* pr, int pn, int an) {
    switch (chi_tpl) {
        case 4: return dispatch_trunc<T, TQ, 4>(b, trunc, px, pr, pn, an);
        case 8: return dispatch_trunc<T, TQ, 8>(b, trunc, px, pr, pn, an);
        case 16: return dispatch_trunc<T, TQ, 16>(b, trunc, px, pr, pn, an);
        case 32: return dispatch_trunc<T, TQ, 32>(b, trunc, px, pr, pn, an);
    }
    return fail(MPS_ERR_UNSUPPORTED, "bond dimension bucket %d not compiled", chi_tpl);
}


}  // namespace
}  // namespace mpsano
