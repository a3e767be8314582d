// md_kernels.cuh -- argument structs and host launchers of md_kernels.cu.
#pragma once
#include "atm3_internal.cuh"

namespace atm3 {

template <typename R>
struct LjArgs {
    Batch b;
    long long n;              // SoA stride = b.ntot
    const R* xl;              // sorted cell-local coordinates, SoA [3n]
    const float* xl32;        // FP32 copy (prefilter of the FP64 path)
    const int* cell_start;    // [ncell + 1]
    const int* cell_sorted;   // [n] global cell of each sorted slot
    double* fs;               // sorted-order LJ force, SoA [3n] (fully written)
    double* mol_ew;           // [2n] per sorted molecule: half of its pair energies, virials
    unsigned* mol_cnt;        // [2n] per sorted molecule: half-shell candidates, interacting pairs
};

// device-side copy of atm_result (same layout)
struct ResultDev {
    double e2, e3, w2, w3, ekin;
    unsigned long long n_cand3, n_int3, n_cand2, n_int2;
};

struct ReduceArgs {
    Batch b;
    const double* unit_ew;
    const unsigned long long* unit_cnt;
    const double* mol_ew;
    const unsigned* mol_cnt;
    const double* ke;         // [n] kinetic energy per molecule
    // non-null when the ATM units evaluated LJ too: E2, W2 and the pair counts
    // per unit ([2 ncell] each) replace mol_ew / mol_cnt
    const double* unit_ew2 = nullptr;
    const unsigned long long* unit_cnt2 = nullptr;
    ResultDev* part;          // [R * REDUCE_PARTS] partial sums
    ResultDev* out;           // [R]
};

constexpr int REDUCE_PARTS = 64;  // partial sums per replica of the two-level reduction

constexpr int LJ_BLOCK = 128;
constexpr int MD_BLOCK = 256;

// maxocc[0] = largest cell occupancy, maxocc[1..5] = largest unit of 3c01, 3c18, 3c08, 3cw,
// corner-anchored 3c08 (3cw's only when wide; 0 otherwise)
cudaError_t launch_build_cells(const Batch& b, double* x, int* cell_of, int* rank, int* count,
                               int* start, int* perm, double* xl, float* xl32, int* cell_sorted,
                               int* maxocc, int* status, bool wide, cudaStream_t st);
cudaError_t launch_lj(int prec, const LjArgs<double>& a64, const LjArgs<float>& a32,
                      cudaStream_t st);
cudaError_t launch_kick(const Batch& b, const int* perm, const double* f_lj, const double* f_atm,
                        double* x, double* v, int drift, double* ke, cudaStream_t st);
cudaError_t launch_kinetic(long long n, const double* v, double* ke, cudaStream_t st);
// first half kick + drift with a total force in the original order
cudaError_t launch_kick_orig(const Batch& b, const double* f, double* x, double* v, double* ke,
                             cudaStream_t st);
// v *= sqrt(T_r (3 N_r - 3) / (2 K_r)) per replica (K_r = res[r].ekin)
cudaError_t launch_rescale(const Batch& b, double* v, double* ke, const ResultDev* res,
                           const double* t_target, cudaStream_t st);
cudaError_t launch_check_finite(long long m, const double* a, int* status, cudaStream_t st);
cudaError_t launch_final_reduce(const ReduceArgs& r, cudaStream_t st);
// pair bitmaps of the FP32 pair-rule decisions: pm[(k - 13) n + s] bit j is
// set when molecule s (cell-sorted) and the j-th molecule of the cell at
// offset27(k) from its cell, k = 13 (the cell itself; molecules after s only)
// .. 26 (the forward cells), are closer than r_c by the canonical FP32
// displacement (xl_t - xl_s) + delta w, the value the block kernels' own
// decisions compute; grid n x PM_WORDS.  A neighbour cell of more than
// PM_CELL_MAX molecules sets ST_CAPACITY in status (its words stay 0).
cudaError_t launch_pair_masks(const Batch& b, const int* start, const float* xl32,
                              const int* cell_sorted, unsigned* pm, int* status, cudaStream_t st);
cudaError_t launch_gather_forces(long long n, const int* perm, const double* f_lj,
                                 const double* f_atm, int which, double* out, cudaStream_t st);
// adds the pair-distance histogram (nbins equal bins over [0, rmax), every
// pair once, rmax at most the smallest cell edge) of every replica to
// counts[R * nbins]
cudaError_t launch_rdf(const Batch& b, const double* xl, const int* start, const int* cell_sorted,
                       double rmax, int nbins, unsigned long long* counts, cudaStream_t st);
// adds the histogram of coordinate `axis` (nbins equal bins over [0, L_axis))
// of every replica's wrapped positions to counts[R * nbins]
cudaError_t launch_density(const Batch& b, const double* x, int axis, int nbins,
                           unsigned long long* counts, cudaStream_t st);
// unit size classes of a block traversal (trav 1, 2 or 4) on built cells:
// zeroes counts[ncls], then lists the units of class k (staged molecules
// <= cut0, <= cut1 with three classes, the rest last) in ulist[k * ncell ..]
// and counts them in counts[k]
cudaError_t launch_unit_classes(const Batch& b, const int* start, int trav, int ncls, int cut0,
                                int cut1, int* ulist, int* counts, cudaStream_t st);
// in place: m signed 64-bit fixed-point sums in units of 2^-bits (the
// deterministic mode's force accumulator) become doubles
cudaError_t launch_fix_to_double(double* f, long long m, int bits, cudaStream_t st);

}  // namespace atm3
