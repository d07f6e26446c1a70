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
    auto kern = circuit_kernel<T, TQ, CHI, TRUNC, NTHR>;
    int dev = 0, sms = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if constexpr (NTHR > 32) {
      if (Lay::bytes > (size_t)limit) {
        // bonds above 32: the team's buffers live in global memory (a slice per CTA,
        // one team per CTA), two CTAs per SM at most
        const int grid = std::max(1, std::min(b->run_count, 2 * sms));
        const mps_status st = ensure_gws(b, (size_t)grid * Lay::bytes);
        if (st != MPS_OK) return st;
        CUDA_TRY(cudaMemsetAsync(b->queue_d, 0, sizeof(int), b->stream));
        timing_begin(b, KIND_CIRCUIT);
        kern<<<grid, NTHR, 0, b->stream>>>(b->meta_d, b->run_count, b->run_order, b->queue_d, pixels,
                                           reinterpret_cast<const cx<T>*>(b->gates), b->gate_n, ansatz,
                                           reinterpret_cast<cx<T>*>(b->arena), b->bonds_d, b->discarded_d,
                                           b->status_d, static_cast<unsigned char*>(b->gws));
        timing_end(b);
        CUDA_TRY(cudaGetLastError());
        count_launch();
        return MPS_OK;
      }
    }
    int per_cta = 1;   // images per CTA
    if (NTHR == 32) {
        per_cta = std::max(1, b->images_per_cta);
        while (per_cta > 1 && (size_t)per_cta * Lay::bytes > (size_t)limit) --per_cta;
    }
    const size_t smem = (size_t)per_cta * Lay::bytes;
    if (smem > (size_t)limit)
        return fail(MPS_ERR_UNSUPPORTED, "circuit kernel needs %zu B shared memory per image (limit %d)",
                    Lay::bytes, limit);
    CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // persistent grid: as many CTAs as stay resident, capped by the work
    int per_sm = 0;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NTHR * per_cta, smem));
    const int needed = (b->run_count + per_cta - 1) / per_cta;
    const int grid = std::max(1, std::min(needed, std::max(1, per_sm) * sms));
    CUDA_TRY(cudaMemsetAsync(b->queue_d, 0, sizeof(int), b->stream));
    timing_begin(b, KIND_CIRCUIT);
    kern<<<grid, NTHR * per_cta, smem, b->stream>>>(b->meta_d, b->run_count, b->run_order, b->queue_d, pixels,
                                                   reinterpret_cast<const cx<T>*>(b->gates), b->gate_n, ansatz,
                                                   reinterpret_cast<cx<T>*>(b->arena), b->bonds_d,
                                                   b->discarded_d, b->status_d, nullptr);
    timing_end(b);
    CUDA_TRY(cudaGetLastError());
    count_launch();
    return MPS_OK;
}

// Layer-pipelined kernel (ladder ansatz, no truncation, at most WAVE_LAYERS layers):
// one CTA of one warp per layer for each image of b->run_order[0 .. run_count).  Its
// buffers only depend on min(CHI, 16) since a ladder bond is at most 2^layers.
template <typename T, typename TQ, int CHI>
mps_status launch_circuit_wave(mps_batch* b, const double* pixels) {
    constexpr int CW = CHI < 16 ? CHI : 16;
    using Lay = WaveLayout<T, TQ, CW>;
    const size_t smem = Lay::bytes;
    if (smem > (size_t)smem_optin_limit())
        return fail(MPS_ERR_UNSUPPORTED, "layer-pipelined circuit kernel needs %zu B shared memory", smem);
    auto kern = circuit_wave_kernel<T, TQ, CW>;
    CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int warps = std::max(1, std::min(b->L_max, WAVE_LAYERS));
    timing_begin(b, KIND_CIRCUIT);
    kern<<<b->run_count, 32 * warps, smem, b->stream>>>(b->meta_d, b->run_count, b->run_order, pixels,
                                                reinterpret_cast<const cx<T>*>(b->gates), b->gate_n,
                                                reinterpret_cast<cx<T>*>(b->arena), b->bonds_d,
                                                b->discarded_d, b->status_d);
    timing_end(b);
    CUDA_TRY(cudaGetLastError());
    count_launch();
    return MPS_OK;
}

// Wider teams are compiled only for the mixed path at bond bucket 16 without
// truncation (the benchmark shape); measured on B300 they do not beat one warp per
// image, so every other combination runs one warp per image.
// Shared memory of one block on B300 (opt-in); layouts above it run on a global-memory
// workspace, one 256-thread team per image.
constexpr size_t SMEM_BLOCK_MAX = 232448;

template <typename T, typename TQ, int CHI, bool TRUNC>
mps_status launch_circuit(mps_batch* b, const double* pixels, int ansatz) {
    if constexpr (CHI > 32 || CircuitLayout<T, TQ, CHI, TRUNC>::bytes > SMEM_BLOCK_MAX) {
        // bonds above 32, and FP64 truncation at bond 32 (its refined eigen-decomposition
        // needs about 270 KB): one 256-thread team per image, workspace in global memory
        return launch_circuit_team<T, TQ, CHI, TRUNC, 256>(b, pixels, ansatz);
    } else {
    if constexpr (!TRUNC) {
        if (b->use_wave) return launch_circuit_wave<T, TQ, CHI>(b, pixels);
    }
    if constexpr (CHI == 16 && !TRUNC && sizeof(T) == 4 && sizeof(TQ) == 4) {
        if (b->circuit_threads == 64) return launch_circuit_team<T, TQ, CHI, TRUNC, 64>(b, pixels, ansatz);
    }
    // FP64 truncation chains up to bond 16 on 128-thread teams: the chain's FP64 work
    // spreads over the SM's four FP64 pipes instead of one, which shortens each chain
    // when few images run at once (serving); full batches keep one warp per image
    if constexpr (TRUNC && sizeof(T) == 8 && CHI <= 16) {
        if (b->circuit_threads == 128) return launch_circuit_team<T, TQ, CHI, TRUNC, 128>(b, pixels, ansatz);
    }
    return launch_circuit_team<T, TQ, CHI, TRUNC, 32>(b, pixels, ansatz);
    }
}

}  // namespace
}  // namespace mpsano
