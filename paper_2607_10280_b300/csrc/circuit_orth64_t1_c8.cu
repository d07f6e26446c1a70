// Circuit kernel instantiation: state float, QR/LQ in double, with the SVD-truncation branch, bond bucket 8.
#include "circuit_launch.cuh"

namespace mpsano {
mps_status launch_circuit_orth64_t1_c8(mps_batch* b, const double* px, int ansatz) {
    return launch_circuit<float, double, 8, true>(b, px, ansatz);
}
}  // namespace mpsano
