// Circuit kernel instantiations: state float, QR/LQ in double, without the SVD-truncation branch.
#include "circuit_launch.cuh"

namespace mpsano {
mps_status launch_circuit_orth64_t0(mps_batch* b, int chi_tpl, const double* px, int ansatz) {
    return dispatch_chi<float, double, false>(b, chi_tpl, px, ansatz);
}
}  // namespace mpsano
