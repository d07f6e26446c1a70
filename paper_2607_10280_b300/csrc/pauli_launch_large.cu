// Environment and Pauli-cache launches for bonds above 32 (buckets 64 and 128): the
// same kernels with their workspace in global memory (a block's shared memory holds
// neither a 64-wide site pair nor its GEMM scratch), one 128-thread team per CTA.
#include <algorithm>

#include "batch.h"
#include "pauli.cuh"

namespace mpsano {
namespace {

template <typename T, int CHI>
mps_status launch_large(mps_batch* b, void* out, bool diag) {
    if (diag) return fail(MPS_ERR_UNSUPPORTED, "the diagonal pair sets are built for bonds up to 32");
    using Lay = PauliLayout<cx<T>, CHI>;
    constexpr int UW = 4;
    const int renv_ctas = b->any_lenv ? 2 * b->B : b->B;
    int dev = 0, sms = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int pauli_ctas = std::max(1, std::min(b->n_units, 4 * sms));
    const size_t pws = (Lay::team_bytes(UW, false) + 255) & ~size_t(255);
    const size_t need = std::max((size_t)renv_ctas * Lay::env_bytes, (size_t)pauli_ctas * pws);
    const mps_status st = ensure_gws(b, need);
    if (st != MPS_OK) return st;
    timing_begin(b, KIND_RENV);
    renv_kernel<T, CHI, true><<<renv_ctas, 32, 0, b->stream>>>(
        b->meta_d, b->B, reinterpret_cast<const cx<T>*>(b->arena), b->bonds_d,
        reinterpret_cast<cx<T>*>(b->renv), b->renv_stride,
        reinterpret_cast<cx<T>*>(b->any_lenv ? b->lenv : nullptr), reinterpret_cast<T*>(b->norms),
        static_cast<unsigned char*>(b->gws), 0, nullptr);
    timing_end(b);
    CUDA_TRY(cudaGetLastError());
    count_launch();
    timing_begin(b, KIND_PAULI);
    pauli_kernel<T, CHI, UW, false, true><<<pauli_ctas, 32 * UW, 0, b->stream>>>(
        b->meta_d, b->n_units, b->units_d, reinterpret_cast<const cx<T>*>(b->arena), b->bonds_d,
        reinterpret_cast<const cx<T>*>(b->renv), b->renv_stride,
        reinterpret_cast<const cx<T>*>(b->any_lenv ? b->lenv : nullptr),
        reinterpret_cast<const T*>(b->norms), reinterpret_cast<T*>(out), static_cast<unsigned char*>(b->gws),
        b->status_d);
    timing_end(b);
    CUDA_TRY(cudaGetLastError());
    count_launch();
    return MPS_OK;
}

}  // namespace

mps_status launch_pauli_large(mps_batch* b, void* out, bool diag, bool f64) {
    if (f64) return b->chi_tpl == 64 ? launch_large<double, 64>(b, out, diag) : launch_large<double, 128>(b, out, diag);
    return b->chi_tpl == 64 ? launch_large<float, 64>(b, out, diag) : launch_large<float, 128>(b, out, diag);
}

}  // namespace mpsano
