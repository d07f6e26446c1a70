// Dispatch of the circuit kernel over precision, truncation branch and bond bucket.
#include "batch.h"

namespace mpsano {
mps_status launch_circuit_fp64_t0_c4(mps_batch* b, const double* px, int ansatz);
mps_status launch_circuit_fp64_t0_c8(mps_batch* b, const double* px, int ansatz);
mps_status launch_circuit_fp64_t0_c16(mps_batch* b, const double* px, int ansatz);
mps_status launch_circuit_fp64_t0_c32(mps_batch* b, const double* px, int ansatz);
mps_status launch_circuit_fp64_t1_c4(mps_batch* b, const double* px, int ansatz);
mps_status launch_circuit_fp64_t1_c8(mps_batch* b, const double* px, int ansatz);
mps_status launch_circuit_fp64_t1_c16(mps_batch* b, const double* px, int ansatz);
mps_status launch_circuit_fp64_t1_c32(mps_batch* b, const double* px, int ansatz);
mps_status launch_circuit_mixed_t0_c4(mps_batch* b, const double* px, int ansatz);
mps_status launch_circuit_mixed_t0_c8(mps_batch* b, const double* px, int ansatz);
mps_status launch_circuit_mixed_t0_c16(mps_batch* b, const double* px, int ansatz);
mps_status launch_circuit_mixed_t0_c32(mps_batch* b, const double* px, int ansatz);
mps_status launch_circuit_mixed_t1_c4(mps_batch* b, const double* px, int ansatz);
mps_status launch_circuit_mixed_t1_c8(mps_batch* b, const double* px, int ansatz);
mps_status launch_circuit_mixed_t1_c16(mps_batch* b, const double* px, int ansatz);
mps_status launch_circuit_mixed_t1_c32(mps_batch* b, const double* px, int ansatz);
mps_status launch_circuit_fp64_t0_c64(mps_batch* b, const double* px, int ansatz);
mps_status launch_circuit_fp64_t0_c128(mps_batch* b, const double* px, int ansatz);
mps_status launch_circuit_fp64_t1_c64(mps_batch* b, const double* px, int ansatz);
mps_status launch_circuit_fp64_t1_c128(mps_batch* b, const double* px, int ansatz);
mps_status launch_circuit_mixed_t0_c64(mps_batch* b, const double* px, int ansatz);
mps_status launch_circuit_mixed_t0_c128(mps_batch* b, const double* px, int ansatz);
mps_status launch_circuit_mixed_t1_c64(mps_batch* b, const double* px, int ansatz);
mps_status launch_circuit_mixed_t1_c128(mps_batch* b, const double* px, int ansatz);
mps_status launch_circuit_orth64_t0_c4(mps_batch* b, const double* px, int ansatz);
mps_status launch_circuit_orth64_t0_c8(mps_batch* b, const double* px, int ansatz);
mps_status launch_circuit_orth64_t0_c16(mps_batch* b, const double* px, int ansatz);
mps_status launch_circuit_orth64_t0_c32(mps_batch* b, const double* px, int ansatz);
mps_status launch_circuit_orth64_t1_c4(mps_batch* b, const double* px, int ansatz);
mps_status launch_circuit_orth64_t1_c8(mps_batch* b, const double* px, int ansatz);
mps_status launch_circuit_orth64_t1_c16(mps_batch* b, const double* px, int ansatz);
mps_status launch_circuit_orth64_t1_c32(mps_batch* b, const double* px, int ansatz);

mps_status launch_circuit_fp64_t0(mps_batch* b, int chi_tpl, const double* px, int ansatz) {
    switch (chi_tpl) {
        case 4: return launch_circuit_fp64_t0_c4(b, px, ansatz);
        case 8: return launch_circuit_fp64_t0_c8(b, px, ansatz);
        case 16: return launch_circuit_fp64_t0_c16(b, px, ansatz);
        case 32: return launch_circuit_fp64_t0_c32(b, px, ansatz);
        case 64: return launch_circuit_fp64_t0_c64(b, px, ansatz);
        case 128: return launch_circuit_fp64_t0_c128(b, px, ansatz);
    }
    return fail(MPS_ERR_UNSUPPORTED, "bond dimension bucket %d not compiled", chi_tpl);
}

mps_status launch_circuit_fp64_t1(mps_batch* b, int chi_tpl, const double* px, int ansatz) {
    switch (chi_tpl) {
        case 4: return launch_circuit_fp64_t1_c4(b, px, ansatz);
        case 8: return launch_circuit_fp64_t1_c8(b, px, ansatz);
        case 16: return launch_circuit_fp64_t1_c16(b, px, ansatz);
        case 32: return launch_circuit_fp64_t1_c32(b, px, ansatz);
        case 64: return launch_circuit_fp64_t1_c64(b, px, ansatz);
        case 128: return launch_circuit_fp64_t1_c128(b, px, ansatz);
    }
    return fail(MPS_ERR_UNSUPPORTED, "bond dimension bucket %d not compiled", chi_tpl);
}

mps_status launch_circuit_mixed_t0(mps_batch* b, int chi_tpl, const double* px, int ansatz) {
    switch (chi_tpl) {
        case 4: return launch_circuit_mixed_t0_c4(b, px, ansatz);
        case 8: return launch_circuit_mixed_t0_c8(b, px, ansatz);
        case 16: return launch_circuit_mixed_t0_c16(b, px, ansatz);
        case 32: return launch_circuit_mixed_t0_c32(b, px, ansatz);
        case 64: return launch_circuit_mixed_t0_c64(b, px, ansatz);
        case 128: return launch_circuit_mixed_t0_c128(b, px, ansatz);
    }
    return fail(MPS_ERR_UNSUPPORTED, "bond dimension bucket %d not compiled", chi_tpl);
}

mps_status launch_circuit_mixed_t1(mps_batch* b, int chi_tpl, const double* px, int ansatz) {
    switch (chi_tpl) {
        case 4: return launch_circuit_mixed_t1_c4(b, px, ansatz);
        case 8: return launch_circuit_mixed_t1_c8(b, px, ansatz);
        case 16: return launch_circuit_mixed_t1_c16(b, px, ansatz);
        case 32: return launch_circuit_mixed_t1_c32(b, px, ansatz);
        case 64: return launch_circuit_mixed_t1_c64(b, px, ansatz);
        case 128: return launch_circuit_mixed_t1_c128(b, px, ansatz);
    }
    return fail(MPS_ERR_UNSUPPORTED, "bond dimension bucket %d not compiled", chi_tpl);
}

mps_status launch_circuit_orth64_t0(mps_batch* b, int chi_tpl, const double* px, int ansatz) {
    switch (chi_tpl) {
        case 4: return launch_circuit_orth64_t0_c4(b, px, ansatz);
        case 8: return launch_circuit_orth64_t0_c8(b, px, ansatz);
        case 16: return launch_circuit_orth64_t0_c16(b, px, ansatz);
        case 32: return launch_circuit_orth64_t0_c32(b, px, ansatz);
    }
    return fail(MPS_ERR_UNSUPPORTED, "bond dimension bucket %d not compiled", chi_tpl);
}

mps_status launch_circuit_orth64_t1(mps_batch* b, int chi_tpl, const double* px, int ansatz) {
    switch (chi_tpl) {
        case 4: return launch_circuit_orth64_t1_c4(b, px, ansatz);
        case 8: return launch_circuit_orth64_t1_c8(b, px, ansatz);
        case 16: return launch_circuit_orth64_t1_c16(b, px, ansatz);
        case 32: return launch_circuit_orth64_t1_c32(b, px, ansatz);
    }
    return fail(MPS_ERR_UNSUPPORTED, "bond dimension bucket %d not compiled", chi_tpl);
}

}  // namespace mpsano
