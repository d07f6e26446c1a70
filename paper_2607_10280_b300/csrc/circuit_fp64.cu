// Circuit kernel instantiations: state double, QR/LQ in double.
#include "circuit_launch.cuh"

namespace mpsano {
mps_status launch_circuit_fp64(mps_batch* b, int chi_tpl, bool trunc, const double* px, const double* pr,
                               int pn, int ansatz) {
    return dispatch_chi<double, double>(b, chi_tpl, trunc, px, pr, pn, ansatz);
}
}  // namespace mpsano
