// Circuit kernel instantiations: state float, QR/LQ in float, without the SVD-truncation branch.
#include "circuit_launch.cuh"

namespace mpsano {
mps_status launch_circuit_mixed_t0(mps_batch* b, int chi_tpl, const double* px, int ansatz) {
    return dispatch_chi<float, float, false>(b, chi_tpl, px, ansatz);
}
}  // namespace mpsano
