// Environment and Pauli-cache launches for a real state (every amplitude real, as for
// the paper ansatz, whose gates H, R_Y and CNOT are real): the same kernels on real
// elements, a quarter of the multiply-adds of the complex contractions and half their
// shared-memory traffic; every Pauli with one Y vanishes exactly.  Complex64 storage
// of the state stays as it is (imaginary parts exactly zero); the environments are
// stored as reals.  Bonds up to 32, 64-thread Pauli teams.
#include <algorithm>

#include "batch.h"
#include "pauli.cuh"

namespace mpsano {
namespace {

template <int CHI, bool DIAG>
mps_status launch_real(mps_batch* b, void* out) {
    using Lay = PauliLayout<float, CHI>;
    constexpr int UW = 2;
    const int limit = smem_optin_limit();
    auto rk = renv_kernel<float, CHI, false, true>;
    CUDA_TRY(cudaFuncSetAttribute(rk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Lay::env_bytes));
    timing_begin(b, KIND_RENV);
    rk<<<b->any_lenv ? 2 * b->B : b->B, 32, Lay::env_bytes, b->stream>>>(
        b->meta_d, b->B, reinterpret_cast<const cx<float>*>(b->arena), b->bonds_d,
        reinterpret_cast<cx<float>*>(b->renv), b->renv_stride,
        reinterpret_cast<cx<float>*>(b->any_lenv ? b->lenv : nullptr), reinterpret_cast<float*>(b->norms), nullptr, 0, nullptr);
    timing_end(b);
    CUDA_TRY(cudaGetLastError());
    count_launch();
    const size_t smem = Lay::team_bytes(UW, DIAG);
    if (smem > (size_t)limit) return fail(MPS_ERR_UNSUPPORTED, "Pauli kernel shared memory %zu B", smem);
    auto pk = pauli_kernel<float, CHI, UW, DIAG, false, true>;
    CUDA_TRY(cudaFuncSetAttribute(pk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    timing_begin(b, KIND_PAULI);
    pk<<<b->n_units, 32 * UW, smem, b->stream>>>(
        b->meta_d, b->n_units, b->units_d, reinterpret_cast<const cx<float>*>(b->arena), b->bonds_d,
        reinterpret_cast<const cx<float>*>(b->renv), b->renv_stride,
        reinterpret_cast<const cx<float>*>(b->any_lenv ? b->lenv : nullptr),
        reinterpret_cast<const float*>(b->norms), reinterpret_cast<float*>(out), nullptr, b->status_d);
    timing_end(b);
    CUDA_TRY(cudaGetLastError());
    count_launch();
    return MPS_OK;
}

template <bool DIAG>
mps_status dispatch_real(mps_batch* b, void* out) {
    switch (b->chi_tpl) {
        case 4: return launch_real<4, DIAG>(b, out);
        case 8: return launch_real<8, DIAG>(b, out);
        case 16: return launch_real<16, DIAG>(b, out);
        case 32: return launch_real<32, DIAG>(b, out);
    }
    return fail(MPS_ERR_UNSUPPORTED, "bond dimension bucket %d has no real-element kernel", b->chi_tpl);
}

}  // namespace

mps_status launch_pauli_real(mps_batch* b, void* out, bool diag) {
    return diag ? dispatch_real<true>(b, out) : dispatch_real<false>(b, out);
}

}  // namespace mpsano
