// Circuit kernel instantiation: state float, QR/LQ in double, with the SVD-truncation branch, bond bucket 16.
#include "circuit_launch.cuh"

namespace mpsano {
mps_status launch_circuit_orth64_t1_c16(mps_batch* b, const double* px, int ansatz) {
    return launch_circuit<float, double, 16, true>(b, px, ansatz);
}
}  // namespace mpsano
