// Circuit kernel instantiations: state float, QR/LQ in double.
#include "circuit_launch.cuh"

namespace mpsano {
mps_status launch_circuit_orth64(mps_batch* b, int chi_tpl, bool trunc, const double* px, const double* pr,
                               int pn, int ansatz) {
    return dispatch_chi<float, double>(b, chi_tpl, trunc, px, pr, pn, ansatz);
}
}  // namespace mpsano
