// Circuit-kernel launch templates (included by one .cu per precision).
#pragma once
#include <algorithm>

#include "batch.h"
#include "circuit.cuh"

namespace mpsano {
namespace {

template <typename T, typename TQ, int CHI, bool TRUNC, int NTHR>
mps_status launch_circuit_team(mps_batch* b, const double* pixels, int ansatz) {
    using Lay = CircuitLayout<T, TQ, CHI, TRUNC>;
    const int limit = smem_optin_limit();
    int per_cta = 1;   // images per CTA
    if (NTHR == 32) {
        per_cta = std::max(1, b->images_per_cta);
        while (per_cta > 1 && (size_t)per_cta * Lay::bytes > (size_t)limit) --per_cta;
    }
    const size_t smem = (size_t)per_cta * Lay::bytes;
    if (smem > (size_t)limit)
        return fail(MPS_ERR_UNSUPPORTED, "circuit kernel needs %zu B shared memory per image (limit %d)",
                    Lay::bytes, limit);
    auto kern = circuit_kernel<T, TQ, CHI, TRUNC, NTHR>;
    CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = (b->B + per_cta - 1) / per_cta;
    timing_begin(b, KIND_CIRCUIT);
    kern<<<grid, NTHR * per_cta, smem, b->stream>>>(b->meta_d, b->B, pixels,
                                                   reinterpret_cast<const cx<T>*>(b->gates), b->gate_n, ansatz,
                                                   reinterpret_cast<cx<T>*>(b->arena), b->bonds_d,
                                                   b->discarded_d, b->status_d);
    timing_end(b);
    CUDA_TRY(cudaGetLastError());
    count_launch();
    return MPS_OK;
}

// Teams wider than a warp pay off only for the larger tiles; smaller buckets run
// one warp per image.
template <typename T, typename TQ, int CHI, bool TRUNC>
mps_status launch_circuit(mps_batch* b, const double* pixels, int ansatz) {
    if constexpr (CHI >= 16 && sizeof(T) == 4 && sizeof(TQ) == 4) {
        if (b->circuit_threads == 64) return launch_circuit_team<T, TQ, CHI, TRUNC, 64>(b, pixels, ansatz);
        if (b->circuit_threads == 128) return launch_circuit_team<T, TQ, CHI, TRUNC, 128>(b, pixels, ansatz);
    }
    return launch_circuit_team<T, TQ, CHI, TRUNC, 32>(b, pixels, ansatz);
}

template <typename T, typename TQ, bool TRUNC>
mps_status dispatch_chi(mps_batch* b, int chi_tpl, const double* px, int an) {
    switch (chi_tpl) {
        case 4: return launch_circuit<T, TQ, 4, TRUNC>(b, px, an);
        case 8: return launch_circuit<T, TQ, 8, TRUNC>(b, px, an);
        case 16: return launch_circuit<T, TQ, 16, TRUNC>(b, px, an);
        case 32: return launch_circuit<T, TQ, 32, TRUNC>(b, px, an);
    }
    return fail(MPS_ERR_UNSUPPORTED, "bond dimension bucket %d not compiled", chi_tpl);
}

}  // namespace
}  // namespace mpsano
