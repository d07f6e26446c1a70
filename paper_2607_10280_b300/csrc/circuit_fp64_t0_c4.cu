// Circuit kernel instantiation: state double, QR/LQ in double, without the SVD-truncation branch, bond bucket 4.
#include "circuit_launch.cuh"

namespace mpsano {
mps_status launch_circuit_fp64_t0_c4(mps_batch* b, const double* px, int ansatz) {
    return launch_circuit<double, double, 4, false>(b, px, ansatz);
}
}  // namespace mpsano
