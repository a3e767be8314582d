// forces.cuh -- host side of one LJ + ATM force evaluation on built cells,
// and the replica descriptors; shared by the context API and the
// allocation-free entry point.
#pragma once
#include "atm3.h"
#include "atm3_internal.cuh"
#include "md_kernels.cuh"

namespace atm3 {

constexpr int ATM_MCAP_LIMIT = 2047;  // staged molecules per unit (queue entries pack 11-bit indices)

// Fill a replica descriptor from the public parameters: linked-cell grid
// (n_d = largest k with L_d / k >= r_c, at least 3), cutoffs in FP64 and
// FP32, LJ constants, FP32 prefilter bands of the FP64 decisions (derivation
// in atm_common.cuh).  Returns ATM_OK, ATM_E_INVALID or ATM_E_BOX_TOO_SMALL.
atm_status make_rep(const atm_params& p, long long n, long long mol0, long long cell0, Rep& r);

struct ForceJob {
    Batch b;                 // device replica table
    const Rep* rep_host;     // [R] host copy (plan sizing)
    const double* xl;        // sorted cell-local coordinates FP64, SoA [3n]
    const float* xl32;       // the same in FP32
    const int* start;        // cell_start [ncell + 1]
    const int* cell_sorted;  // [n]
    double* f_lj;            // [3n] sorted order, fully written
    double* f_atm;           // [3n] sorted order
    double* mol_ew;          // [2n]
    unsigned* mol_cnt;       // [2n]
    double* unit_ew;         // [2 ncell]
    unsigned long long* unit_cnt;
    int* status;
    int* work;               // unit counter of the persistent launch
    int trav, trunc, prec;
    int mcap;                // largest unit of the traversal (staged molecules)
    int optin;               // opt-in shared memory per block of the device
    int sms;                 // SMs of the device
    int persistent;          // 1: persistent grid over a unit counter
    int nwarps;              // 0: the plan's default, else 4 or 8
    cudaStream_t st;
    // 3c08 / corner-anchored 3c08 / 3c18, pair rule: LJ evaluated inside the
    // ATM units (f_atm receives LJ + ATM, f_lj is zeroed; E2, W2 and the pair
    // counts go to unit_ew2 / unit_cnt2 instead of mol_ew / mol_cnt)
    int lj = 0;
    double* unit_ew2 = nullptr;
    unsigned long long* unit_cnt2 = nullptr;
    // block traversals: unit size classes (ncls 2 or 3; 1 = none).  Units of
    // at most cuts[0] (then cuts[1]) staged molecules run in launches sized for
    // that bound (2 warps when it is at most 64), the rest in one sized for
    // mcap; ulist [ncls * ncell], ucount [ncls] and work [ncls] are scratch
    int ncls = 1;
    int cuts[2] = {0, 0};
    int* ulist = nullptr;
    int* ucount = nullptr;
    // with a side stream the first class runs on it, forked from st after the
    // class kernel and joined back before the evaluation ends
    cudaStream_t side_st = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // deterministic mode: fixed work order; the block traversals sum their
    // terms in 64-bit fixed point and f_atm is converted back after them
    int det = 0;
    // FP32 pair rule of the block traversals: [PM_WORDS n] words for the pair
    // bitmaps, computed by one kernel ahead of the units, which assemble
    // their adjacency from them (nullptr: the units decide their own pairs).
    // The caller passes it only when every cell holds at most PM_CELL_MAX
    // molecules (a fuller cell found on the device sets ST_CAPACITY)
    unsigned* pmask = nullptr;
    // pair rule of the block traversals: edge-table capacity in 1/16 edges per
    // staged molecule (256: 16), and where the units record their need
    // (nullptr: not recorded)
    int gpm16 = 256;
    int* emax = nullptr;
};

cudaError_t enqueue_lj(const ForceJob& j);
// *capacity is set when no kernel configuration fits the unit size
cudaError_t enqueue_atm(const ForceJob& j, size_t* smem_set, bool* capacity);
// the job runs its units in size classes (one more kernel, ncls ATM launches)
bool atm_split_active(const ForceJob& j);
// the job's units take their pairs from bitmaps (one more kernel ahead of them)
bool atm_uses_pair_masks(const ForceJob& j);

}  // namespace atm3
