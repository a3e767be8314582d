// ctx.cuh -- the context behind the C ABI (a batch of one or more replicas
// with its device buffers) and the helpers that capi.cu shares with the
// surrogate's entry points (sur_capi.cu).
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "atm3.h"
#include "atm3_internal.cuh"
#include "md_kernels.cuh"

namespace atm3 {
struct SurState;
}

struct atm_ctx {
    int R = 1;
    std::vector<atm_params> params;
    std::vector<atm3::Rep> reps;  // host copy
    long long n = 0, ncell = 0;
    int device = 0;
    cudaStream_t st = nullptr;
    atm3::Batch b{};
    atm3::Rep* d_rep = nullptr;
    int* d_rep_of_cell = nullptr;
    int* d_rep_of_mol = nullptr;
    double* x = nullptr;   // [3n] positions, original order (wrapped by the cell build)
    double* v = nullptr;   // [3n] velocities, original order
    double* x0 = nullptr;  // [3n] snapshot at the start of a graph-mode run
    double* v0 = nullptr;
    double* xl = nullptr;  // [3n] sorted cell-local FP64
    float* xl32 = nullptr; // [3n] sorted cell-local FP32
    int* cell_of = nullptr;
    int* rank = nullptr;
    int* count = nullptr;
    int* start = nullptr;
    int* perm = nullptr;
    int* cell_sorted = nullptr;
    double* f_lj = nullptr;   // [3n] sorted order
    double* f_atm = nullptr;  // [3n] sorted order
    double* f_out = nullptr;  // [3n] original-order scratch for atm_get_forces
    double* unit_ew = nullptr;
    unsigned long long* unit_cnt = nullptr;
    double* unit_ew2 = nullptr;             // [2 ncell] LJ E2, W2 of the units (fused steps)
    unsigned long long* unit_cnt2 = nullptr;
    double* mol_ew = nullptr;
    unsigned* mol_cnt = nullptr;
    double* ke = nullptr;
    atm3::ResultDev* d_res = nullptr;  // [R]
    atm3::ResultDev* d_part = nullptr; // [R * REDUCE_PARTS] partial sums
    atm3::ResultDev* h_res = nullptr;  // [R] pinned
    int* d_status = nullptr;
    int* h_status = nullptr;
    int* d_chk = nullptr;  // finiteness flag of a state or force copied in
    int* h_chk = nullptr;
    int* d_maxocc = nullptr;
    int* h_maxocc = nullptr;
    int* d_work = nullptr;    // [4] persistent unit counters (one per unit size class)
    int* d_ulist = nullptr;   // [3 * ncell] unit lists of the size classes
    int* d_ucount = nullptr;  // [4] their lengths
    unsigned long long* d_dens = nullptr;  // [R * DENS_MAX_BINS]
    unsigned long long* d_rdf = nullptr;   // [R * DENS_MAX_BINS]
    double* d_ttarget = nullptr;           // [R] thermostat temperatures
    double rdf_rmax = 0.0;
    int rdf_nbins = 0;
    long long rdf_samples = 0;
    int dens_axis = -1, dens_nbins = 0;
    long long dens_samples = 0;
    int maxocc = 0;
    int unit_max[atm3::ATM_NTRAV] = {};  // largest unit (staged molecules) of 3c01, 3c18, 3c08, 3cw
    // pair rule of the block traversals outside the deterministic mode: the
    // edge table's capacity in 1/16 edges per staged molecule, from the
    // largest need the units of this context recorded (d_maxocc[1 + NTRAV +
    // trav], read with the unit sizes) plus a margin; 256 before any
    int gpm16[atm3::ATM_NTRAV] = {256, 256, 256, 256, 256};
    bool have_x = false, cells_built = false, forces_valid = false;
    int f_trav = -1, f_trunc = -1, f_prec = -1;
    bool f_fused = false;  // the current forces came from units that also did LJ
    bool wide_cells = false;  // cell builds also size the wide traversal's 5^3 units
    // forces of the current state given by the caller (original order, total),
    // for the combination f_in_key = (traversal, truncation, precision)
    double* f_in = nullptr;
    bool f_in_valid = false;
    int f_in_key[3] = {-1, -1, -1};
    size_t smem_set[2][atm3::ATM_NTRAV][2] = {};
    int smem_optin = 0, sms = 0;
    // launch options: persistent ATM grid, warps per block-kernel CTA (0 =
    // default), CUDA-graph steps; tuned choices per (prec, trav, trunc)
    int opt_persistent = 0, opt_nwarps = 0, opt_graph = 0;
    int opt_cls[3] = {1, 0, 0};  // unit size classes: count, bounds of the first two
    int det = 0;                 // deterministic mode (atm_set_deterministic)
    // FP32 pair-rule decisions of the block traversals from per-molecule pair
    // bitmaps ([27 n] words) when every cell holds at most 32 molecules
    // (atm_set_pair_masks; on by default); pm_3c18: every replica's cells are
    // wide enough in FP32 that cells two apart hold no pair within r_c
    unsigned* pmask = nullptr;
    int opt_pmask = 1;
    bool pm_3c18 = false;
    // 0 = not tuned, else 1 + persistent + 2 * (nwarps == 8) + 4 * size-class choice
    int tuned[2][atm3::ATM_NTRAV][2] = {};
    // untuned FP32 pair rule of the block traversals: warps per CTA chosen by
    // resident warps per SM, cached for a band of unit sizes (mcap / 8)
    int nw_auto[atm3::ATM_NTRAV][2][2] = {};  // [trav][trunc] = {mcap band + 1, warps}
    // graph of one step, valid for (trav, trunc, prec, mcap, launch choice)
    cudaStream_t cap_st = nullptr;
    // size classes: the small-unit class runs on side_st beside the rest
    // (forked from and joined to the context's stream by the two events)
    cudaStream_t side_st = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // host round trips (atm_step_host): the input checks and the copy of the
    // last step's positions run on io_st beside the context's stream
    cudaStream_t io_st = nullptr;
    cudaEvent_t ev_io = nullptr, ev_io_done = nullptr;
    double* x_host_out = nullptr;  // where the last step copies its positions early
    bool x_out_issued = false;     // that copy is in flight on io_st
    cudaGraphExec_t graph = nullptr;
    int graph_key[9] = {-1, -1, -1, -1, -1, -1, -1, -1, -1};
    // profiling: event pairs around launch groups, summed per kind
    int prof = 0;  // profiling: 0 off, 1 every launch group, 2 force evaluations only
    struct EvRec {
        cudaEvent_t a, b;
        int kind;
    };
    std::vector<EvRec> ev_live;
    std::vector<cudaEvent_t> ev_pool;
    double prof_ms[4] = {0, 0, 0, 0};  // cells, lj, atm, md
    long long n_launch = 0, n_atm = 0;
    atm3::SurState* sur = nullptr;  // learned surrogate: model, data set, training state
    char err[256] = "no error";
};


namespace atm3 {

// record the reason of a failure in the context and return the status
atm_status ctx_fail(atm_ctx* c, atm_status s, const char* fmt, ...);
// wait for the stream, fold the device status word into a status
atm_status ctx_sync_and_check(atm_ctx* c);
// LJ + ATM (exact or surrogate) forces of the current cells
// the wide traversal's units are sized by cell builds only once it is in use:
// its first request rebuilds the (unchanged) cells with that size
atm_status ctx_want_wide(atm_ctx* c, int trav);
// fuse_lj: 3c08 / corner-anchored 3c08 under the pair rule evaluate LJ inside
// the ATM units (only the total force is kept apart from the energies)
atm_status ctx_enqueue_forces(atm_ctx* c, int trav, int trunc, int prec, int mcap,
                              bool fuse_lj = false);
// profiling of a launch group (kind: 0 cells, 1 LJ, 2 ATM, 3 MD)
cudaEvent_t ctx_prof_begin(atm_ctx* c, int kind);
void ctx_prof_end(atm_ctx* c, int kind, cudaEvent_t a);

// surrogate hooks (sur_capi.cu)
atm_status sur_enqueue_atm(atm_ctx* c);       // surrogate force into f_atm; unit sums zeroed
atm_status sur_enqueue_monitor(atm_ctx* c);   // compare the surrogate with the current exact f_atm
bool sur_exact_due(atm_ctx* c);               // this ATM_SURROGATE step uses the exact traversal
void sur_count_step(atm_ctx* c);
int sur_exact_every(const atm_ctx* c);
void sur_free(atm_ctx* c);

}  // namespace atm3

#define CU(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return atm3::ctx_fail(c, ATM_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)
