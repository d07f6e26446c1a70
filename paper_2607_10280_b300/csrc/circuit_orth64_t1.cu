// Circuit kernel instantiations: state float, QR/LQ in double, with the SVD-truncation branch.
#include "circuit_launch.cuh"

namespace mpsano {
mps_status launch_circuit_orth64_t1(mps_batch* b, int chi_tpl, const double* px, int ansatz) {
    return dispatch_chi<float, double, true>(b, chi_tpl, px, ansatz);
}
}  // namespace mpsano
