// Circuit kernel instantiations: state float, QR/LQ in float.
#include "circuit_launch.cuh"

namespace mpsano {
mps_status launch_circuit_mixed(mps_batch* b, int chi_tpl, bool trunc, const double* px, const double* pr,
                               int pn, int ansatz) {
    return dispatch_chi<float, float>(b, chi_tpl, trunc, px, pr, pn, ansatz);
}
}  // namespace mpsano
