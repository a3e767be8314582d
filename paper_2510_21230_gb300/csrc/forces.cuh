// forces.cuh -- one LJ + ATM force evaluation on built cells (host side).
#pragma once
#include "atm3_internal.cuh"
#include "md_kernels.cuh"

namespace atm3 {

constexpr int ATM_MCAP_LIMIT = 2047;  // staged molecules per unit (queue entries pack 11-bit indices)

struct ForceJob {
    Grid g;
    long long n;
    const double* xl;        // sorted cell-local coordinates FP64, SoA [3n]
    const float* xl32;       // the same in FP32
    const int* start;        // cell_start [ncell + 1]
    const int* cell_sorted;  // [n]
    double* f_lj;            // [3n] sorted order, fully written
    double* f_atm;           // [3n] sorted order
    double* lj_ew;
    unsigned long long* lj_cnt;
    double* unit_ew;
    unsigned long long* unit_cnt;
    int* status;
    double rc, nu, lj_eps, lj_sigma;
    int lj_shift;
    int trav, trunc, prec;
    int mcap;   // largest unit of the traversal (staged molecules)
    int optin;  // opt-in shared memory per block of the device
    cudaStream_t st;
};

cudaError_t enqueue_lj(const ForceJob& j);
// *capacity is set when no kernel configuration fits the unit size
cudaError_t enqueue_atm(const ForceJob& j, size_t* smem_set, bool* capacity);

}  // namespace atm3
