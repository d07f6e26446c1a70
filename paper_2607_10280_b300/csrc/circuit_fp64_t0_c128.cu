// Circuit kernel instantiation: state double, QR/LQ in double, without the SVD-truncation branch, bond bucket 128 (workspace in global memory).
#include "circuit_launch.cuh"

namespace mpsano {
mps_status launch_circuit_fp64_t0_c128(mps_batch* b, const double* px, int ansatz) {
    return launch_circuit<double, double, 128, false>(b, px, ansatz);
}
}  // namespace mpsano
