// md_kernels.cuh -- argument structs and host launchers of md_kernels.cu.
#pragma once
#include "atm3_internal.cuh"

namespace atm3 {

template <typename R>
struct LjArgs {
    Grid g;
    long long n;
    const R* xl;              // sorted cell-local coordinates, SoA [3n]
    const int* cell_start;    // [ncell + 1]
    const int* cell_sorted;   // [n] cell of each sorted slot
    double* fs;               // sorted-order LJ force, SoA [3n] (fully written)
    double* part_ew;          // [2 * blocks]: E2, W2 per block
    unsigned long long* part_cnt;  // [2 * blocks]: candidates, visits
    R w[3];
    R rc2, sig2, eps4, eps24, eps48, ushift;
    // FP64 path: FP32 prefilter of the cutoff test (FP32 coordinates, cell
    // edges, and the band outside which the FP32 value decides; see atm_common.cuh)
    const float* xl32;
    float wf[3];
    float p_lo, p_hi;
};

// device-side copy of atm_result (same layout)
struct ResultDev {
    double e2, e3, w2, w3, ekin;
    unsigned long long n_cand3, n_int3, n_cand2, n_int2;
};

struct ReduceArgs {
    const double* unit_ew;
    const unsigned long long* unit_cnt;
    long long n_units;
    const double* lj_ew;
    const unsigned long long* lj_cnt;
    long long n_lj;
    const double* ke_part;
    long long n_ke;
    ResultDev* out;
};

constexpr int LJ_BLOCK = 128;
constexpr int MD_BLOCK = 256;

// maxocc[0] = largest cell occupancy, maxocc[1..3] = largest unit of 3c01, 3c18, 3c08
cudaError_t launch_build_cells(const Grid& g, long long n, double* x, int* cell_of, int* rank,
                               int* count, int* start, int* perm, double* xl, float* xl32,
                               int* cell_sorted, int* maxocc, int* status, cudaStream_t st);
cudaError_t launch_lj(int prec, const LjArgs<double>& a64, const LjArgs<float>& a32,
                      cudaStream_t st);
cudaError_t launch_kick(long long n, const int* perm, const double* f_lj, const double* f_atm,
                        double* x, double* v, double half_dt, double dt, int drift,
                        double* ke_part, cudaStream_t st);
cudaError_t launch_kinetic(long long n, const double* v, double* ke_part, cudaStream_t st);
cudaError_t launch_check_finite(long long m, const double* a, int* status, cudaStream_t st);
cudaError_t launch_final_reduce(const ReduceArgs& r, cudaStream_t st);
cudaError_t launch_gather_forces(long long n, const int* perm, const double* f_lj,
                                 const double* f_atm, int which, double* out, cudaStream_t st);

}  // namespace atm3
