// Circuit kernel instantiation: state double, QR/LQ in double, with the SVD-truncation branch, bond bucket 64 (workspace in global memory).
#include "circuit_launch.cuh"

namespace mpsano {
mps_status launch_circuit_fp64_t1_c64(mps_batch* b, const double* px, int ansatz) {
    return launch_circuit<double, double, 64, true>(b, px, ansatz);
}
}  // namespace mpsano
