// Circuit kernel instantiation: state float, QR/LQ in float, without the SVD-truncation branch, bond bucket 8.
#include "circuit_launch.cuh"

namespace mpsano {
mps_status launch_circuit_mixed_t0_c8(mps_batch* b, const double* px, int ansatz) {
    return launch_circuit<float, float, 8, false>(b, px, ansatz);
}
}  // namespace mpsano
