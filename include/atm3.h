/*
 * atm3.h -- C ABI of the GB300 (sm_103a) library for Axilrod-Teller-Muto
 * three-body forces over linked-cell triplets, next to Lennard-Jones pair
 * forces, after "Linked Cell Traversal Algorithms for Three-Body Interactions
 * in Molecular Dynamics" (arXiv 2510.21230).
 *
 * Problem statement (paper section 2 and section 3 opening): N molecules in a
 * periodic orthorhombic box [0,Lx)x[0,Ly)x[0,Lz), reduced LJ units
 * (eps = sigma = m = 1 by default), one cutoff radius r_c for pairs and
 * triplets, ATM strength nu.  Linked cells have edge w_d = L_d / n_d with n_d
 * the largest integer such that L_d / n_d >= r_c; n_d >= 3 is required.
 *
 * Conventions shared by every entry point
 *  - Every call returns an atm_status; nothing exits, aborts or throws across
 *    the ABI.  atm_last_error() gives a one-line reason for the last failure.
 *  - Arrays of 3-vectors are SoA: x[0..n), y[0..n), z[0..n) back to back
 *    (3n doubles), in the caller's ("original") molecule order.
 *  - Host pointers are caller-owned and only read or written during the call.
 *    `_dev` variants take device pointers on the context's device; the data
 *    is copied on the context's stream and the caller keeps ownership.
 *  - Work is enqueued on params.cuda_stream (NULL = the legacy default
 *    stream).  Calls that return host data (atm_get_*, or any call given a
 *    non-NULL atm_result*) synchronise that stream before returning.
 *  - The context owns all its device memory (allocated in atm_create, freed in
 *    atm_destroy).  A context is not thread-safe: one host thread at a time.
 */
#ifndef ATM3_H
#define ATM3_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ATM3_ABI_VERSION 3

typedef enum {
    ATM_OK = 0,
    ATM_E_INVALID = 1,       /* bad argument (NULL pointer, n < 0, unknown enum, rc <= 0 ...) */
    ATM_E_BOX_TOO_SMALL = 2, /* fewer than 3 cells along some axis */
    ATM_E_CUDA = 3,          /* a CUDA runtime call or kernel launch failed */
    ATM_E_TIMEOUT = 4,       /* a bounded device-side wait gave up */
    ATM_E_NONFINITE = 5,     /* a position or velocity is NaN or infinite */
    ATM_E_STATE = 6,         /* call out of order (e.g. forces before a state was set) */
    ATM_E_CAPACITY = 7,      /* a cell holds more molecules than the kernels stage (see atm_create) */
    ATM_E_RANGE = 8          /* deterministic mode: a force term beyond its fixed-point range */
} atm_status;

/* Cell-triplet traversals (paper section 4, and one wide traversal).
 *  3C01: no Newton-3; for every molecule i of a base cell, every pair {j,k} of
 *        other molecules in its 27-cell neighbourhood; only F_i is written and
 *        u/3 is added per visit.
 *  3C18: Newton-3; base cell, its 13 forward neighbours ((dz,dy,dx)
 *        lexicographically > 0) and every pair of those neighbours
 *        (1 + 13 + 78 cell tasks per base cell, Algorithm 1).
 *  3C08: Newton-3; 2x2x2 block anchored at the base cell; every cell multiset
 *        of the block whose bounding box starts at the anchor
 *        (1 + 13 + 44 cell tasks per block). */
/*  3CW:  not in the paper.  Like 3C01 (owner computes, u/3 per visit) over the
 *        5x5x5 cells around the base cell: for i in the base cell, every pair
 *        {j, k} of molecules within R_w = 2 min(w_d) of i (within r_c under the
 *        pair rule) whose third side is below R_w too.  Under the product rule it finds every interacting
 *        triplet with all sides below R_w -- every one, once the closest pair
 *        is r_min apart with (r_min + sqrt(r_min^2 + 4 r_c^3 / r_min)) / 2 <=
 *        R_w -- and so measures what the paper's traversals miss.  Needs 5
 *        cells per axis (BOX_TOO_SMALL otherwise).  n_cand3 counts the
 *        partner pairs of every owner, n_int3 the owner visits. */
/*  3C08A: the 3c08 of the paper's text (section 4, Fig. c08traversal): the
 *        procedure of 3C18 with the partners of the base cell restricted to
 *        the other 7 cells of the 2x2x2 block in front of it, so every task
 *        holds the block's corner cell (1 + 14 + 21 tasks per block).  A
 *        triplet whose cells form a block triple without its corner cell
 *        (e.g. the three face neighbours of a cell) is never visited: these
 *        are interactions the paper says 3c08 omits.  Newton-3, same units
 *        and launch plans as 3C08. */
typedef enum { ATM_3C01 = 0, ATM_3C18 = 1, ATM_3C08 = 2, ATM_3CW = 3, ATM_3C08A = 4 } atm_traversal;

/* Truncation conditions (paper section 2).  A triplet interacts iff
 *  PAIR:    r_ij < r_c and r_ik < r_c and r_jk < r_c;
 *  PRODUCT: r_ij r_ik r_jk < r_c^3, decided as (p*q)*s < r_c^6 on the three
 *           squared sides sorted ascending (p <= q <= s). */
typedef enum { ATM_TRUNC_PAIR = 0, ATM_TRUNC_PRODUCT = 1 } atm_truncation;

/* Arithmetic of the force evaluation.
 *  FP64:  every decision and every force, energy and virial term in FP64.
 *  FP32C: decisions and per-triplet arithmetic in FP32 on FP32 cell-local
 *         coordinates (every pair decision on the canonical displacement
 *         (xl_q - xl_p) + (o_q - o_p) w; the pair-rule block traversals then
 *         evaluate triplets and forces on the FP32-rounded unit-frame
 *         positions xl + o w).  Force sums: 3C18 / 3C08 / 3C08A add each triplet's
 *         three pair scalars to per-edge FP32 sums, then each molecule's share
 *         of a unit is a plain FP32 sum over its edges, and the shares of
 *         different units are added in FP64; 3C01 / 3CW keep compensated
 *         (Kahan) FP32 per-lane sums of F_i, combined in FP64.  Energy and
 *         virial: Kahan-compensated FP32 per lane, reduced in FP64.  (The
 *         deterministic mode sums the block traversals' terms in fixed
 *         point instead, see atm_set_deterministic.)
 *  SURROGATE: the ATM force comes from the learned per-molecule model below
 *         (atm_surrogate_*), not from triplets; LJ runs in FP32.  The model
 *         gives forces only: E3, W3 and the triplet counts are reported as 0.
 *         Traversal and truncation select the exact evaluation that atm_step
 *         interleaves every `exact_every` steps (atm_surrogate_options). */
typedef enum { ATM_FP64 = 0, ATM_FP32C = 1, ATM_SURROGATE = 2 } atm_precision;

typedef struct {
    double box[3];      /* L_x, L_y, L_z > 0 */
    double rc;          /* cutoff radius for pairs and triplets, > 0 */
    double nu;          /* ATM strength (0.073 argon-like reduced units) */
    double lj_eps;      /* LJ epsilon (1) */
    double lj_sigma;    /* LJ sigma (1) */
    double dt;          /* velocity-Verlet time step used by atm_step */
    int lj_shift;       /* 1: LJ energy shifted to 0 at r_c; 0: plain truncation */
    int device;         /* CUDA device ordinal */
    void* cuda_stream;  /* cudaStream_t to enqueue on; NULL = default stream */
} atm_params;

/* Scalars of one force evaluation (section 5 estimators).
 * e2, e3: LJ and ATM potential energy; w2, w3: pair and three-body virial
 * W = sum r_ab . F_ab (Eq. P_3); the caller assembles the virial pressure as
 * P = rho T + (w2 + w3) / (3 V).  ekin = 1/2 sum v^2 (unit mass).
 * n_cand3 / n_int3: candidate / interacting triplets of the traversal
 * (3C01 counts owner visits); n_cand2 / n_int2: candidate / interacting
 * pairs of the half-shell pair traversal (each pair once). */
typedef struct {
    double e2, e3, w2, w3, ekin;
    uint64_t n_cand3, n_int3, n_cand2, n_int2;
} atm_result;

typedef struct atm_ctx atm_ctx;

/* Create a context for n molecules (n >= 0).  Allocates every device buffer.
 * Errors: INVALID, BOX_TOO_SMALL, CUDA.  *out is NULL on failure. */
atm_status atm_create(const atm_params* params, int64_t n, atm_ctx** out);

/* Destroy a context and free its device memory; NULL is allowed. */
atm_status atm_destroy(atm_ctx* ctx);

/* One-line description of the last error on ctx (never NULL). */
const char* atm_last_error(const atm_ctx* ctx);

/* ABI version number (ATM3_ABI_VERSION). */
int atm_abi_version(void);

/* Set positions x[3n] (any real values; wrapped into the box by
 * atm_build_cells) and velocities v[3n] (NULL = zero) from host memory.  The
 * copies are checked for NaN / Inf on the device; the call synchronises the
 * stream, so the caller may reuse its buffers on return.
 * Errors: INVALID, NONFINITE, CUDA. */
atm_status atm_set_state(atm_ctx* ctx, const double* x, const double* v);
/* Same from device memory (x_dev required, v_dev may be NULL).  The values
 * are checked for finiteness on the device; a failure surfaces as NONFINITE
 * from the next synchronising call. */
atm_status atm_set_state_dev(atm_ctx* ctx, const double* x_dev, const double* v_dev);

/* Linked cells (section 3): wrap positions into the box, bin them with the
 * cell-edge rule above, and sort molecules by (cell id, original index) with
 * cell id = (c_z n_y + c_y) n_x + c_x.  Also reads the largest cell occupancy
 * back to size the force kernels (synchronises the stream).
 * Errors: STATE (no positions), CUDA. */
atm_status atm_build_cells(atm_ctx* ctx);

/* Copy the cell arrays to caller-owned host memory (any pointer may be NULL):
 * cell_of[n] (original order), cell_start[ncell+1], perm[n] (sorted slot ->
 * original index).  ncell3[3] (may be NULL) receives n_x, n_y, n_z. */
atm_status atm_get_cells(atm_ctx* ctx, int32_t* cell_of, int32_t* cell_start, int32_t* perm,
                         int32_t* ncell3);

/* LJ pair forces plus ATM three-body forces with the given traversal,
 * truncation and precision (cells must be built).  If out is non-NULL the
 * stream is synchronised and the scalars are written to *out.
 * Errors: INVALID, STATE, CUDA, CAPACITY (the staged neighbourhood of the
 * fullest cell does not fit in shared memory: more than about 60 molecules per
 * cell for 3C01 in FP64, far more for 3C18/3C08). */
atm_status atm_compute_forces(atm_ctx* ctx, atm_traversal trav, atm_truncation trunc,
                              atm_precision prec, atm_result* out);

/* Forces of the last evaluation in original order: which = 0 total,
 * 1 LJ only, 2 ATM only.  f[3n] host (synchronises) or device. */
atm_status atm_get_forces(atm_ctx* ctx, double* f, int which);
atm_status atm_get_forces_dev(atm_ctx* ctx, double* f_dev, int which);

/* Current (wrapped) positions and velocities, host, either may be NULL. */
atm_status atm_get_state(atm_ctx* ctx, double* x, double* v);

/* nsteps velocity-Verlet NVE steps of size params.dt (unit mass):
 * v += dt/2 F; x += dt v; rebuild cells; F = LJ + ATM; v += dt/2 F.
 * The first step computes F at the start if no evaluation is current.
 * If last is non-NULL the scalars after the final step are written there
 * (synchronises).  Errors: as atm_compute_forces. */
atm_status atm_step(atm_ctx* ctx, int nsteps, atm_traversal trav, atm_truncation trunc,
                    atm_precision prec, atm_result* last);

/* A round trip through host memory for callers that keep the state on the
 * host: x[3n] and v[3n] (host, original order) become the state and f[3n]
 * (host, or NULL) its total force as computed with (trav, trunc, prec), as
 * atm_set_forces takes it (NULL: the first step evaluates it; with
 * ATM_SURROGATE f must be NULL); then nsteps steps as atm_step; then the new
 * (wrapped) positions and velocities are written back into x and v, the total
 * force of the new state into f (when given), and the scalars into *last (when
 * non-NULL).  The result equals atm_set_state, atm_set_forces, atm_step,
 * atm_get_state and atm_get_forces(..., 0) in sequence, but the stream is
 * synchronised only by the steps' cell builds and once at the end (those calls
 * synchronise one by one), and the input checks and the copy of the last
 * step's positions run beside the other copies and the force evaluation on
 * a second stream of the context.  The inputs are checked for NaN / Inf on the
 * device: a non-finite input returns NONFINITE, after which the contents of x,
 * v and f are unspecified and the context has no state.  Host memory that is
 * page-locked (cudaHostAlloc / cudaHostRegister) is copied fastest.
 * Errors: as atm_step, NONFINITE. */
atm_status atm_step_host(atm_ctx* ctx, int nsteps, atm_traversal trav, atm_truncation trunc,
                         atm_precision prec, double* x, double* v, double* f, atm_result* last);

/* ---- Batches of independent replicas ------------------------------------
 * A context may hold nrep independent periodic systems ("replicas", e.g. an
 * ensemble of uneven N, density and temperature).  Every kernel of a force
 * evaluation or of a step covers all replicas in one launch (cells of all
 * replicas are numbered back to back, every CTA looks its replica up).
 * State arrays are the replicas' SoA arrays back to back: replica r occupies
 * molecules [sum_{s<r} n[s], sum_{s<=r} n[s]) of every coordinate row, so
 * x[d * ntot + i] is coordinate d of molecule i.  atm_create(p, n) is the
 * batch of one.  Per-replica parameters (box, rc, nu, LJ, dt) may differ;
 * device and cuda_stream are taken from params[0].
 * Errors: as atm_create. */
atm_status atm_batch_create(const atm_params* params, const int64_t* n, int nrep, atm_ctx** out);
/* Number of replicas and total molecules. */
atm_status atm_batch_size(const atm_ctx* ctx, int* nrep, int64_t* ntot);
/* Total cells of all replicas (the length of atm_get_cells' cell_start is
 * this + 1).  Errors: INVALID (NULL). */
atm_status atm_batch_cells(const atm_ctx* ctx, int64_t* ncell);

/* The linked-cell grid of one system (paper section 3, the cell-edge rule
 * above): ncell3[3] receives n_x, n_y, n_z.  Host arithmetic, no device.
 * Errors: INVALID (NULL, non-positive or non-finite box or rc),
 * BOX_TOO_SMALL (fewer than 3 cells along some axis). */
atm_status atm_cell_grid(const atm_params* params, int32_t* ncell3);
/* Scalars of the last evaluation for every replica: out[nrep] (synchronises).
 * (atm_compute_forces / atm_step return replica 0's.) */
atm_status atm_get_results(atm_ctx* ctx, atm_result* out);

/* Launch options.  persistent = 1: the ATM kernel runs as a persistent grid
 * (resident CTAs x SMs) whose CTAs take traversal units from a global counter
 * instead of one CTA per unit.  nwarps = 4 or 8 warps per 3C18/3C08 CTA (0 =
 * default).  graph = 1: atm_step captures one step in a CUDA graph (on a
 * stream of its own) and replays it, with no host synchronisation between
 * steps; the graph sizes the kernels for the current largest unit plus
 * headroom (at most a quarter of it, the largest amount that keeps the
 * resident CTAs per SM of the current size, else 4 molecules), and a step
 * that outgrows it is detected on the device, after
 * which the run is restarted from its initial state without the graph.
 * Options reset any autotuned choice.  Errors: INVALID. */
atm_status atm_set_options(atm_ctx* ctx, int persistent, int nwarps, int graph);

/* Domain decomposition (the paper's outlook: distributed memory).  The
 * replica owns only the cell layers z_lo <= c_z < z_hi of its grid (0 <= z_lo
 * < z_hi <= n_z; all layers by default): ATM units whose base cell (3C01,
 * 3C18, 3CW) or anchor cell (3C08, 3C08A) lies in another layer, and the LJ
 * pair terms of molecules in another layer, are skipped, so energies,
 * virials and counts are those of the owned units and molecules.  A context
 * that holds a domain's molecules plus one halo layer of the neighbouring
 * domains' molecules below and above then gives: the complete force of each
 * owned molecule under 3C01 and LJ (owner computes); under 3C18 / 3C08 /
 * 3C08A the owned units' share, with the forces those units put on the halo
 * layer above to be added to its owner's molecules (their units reach one
 * layer up); the global sums are the sums over the domains.  The host side
 * (partition, halo exchange, force return, sums) is
 * paper_2510_21230_gb300/domain.py.  The surrogate evaluates whole replicas:
 * it returns INVALID while layers are restricted.  Resets the current
 * forces.  Errors: INVALID, CUDA. */
atm_status atm_set_owned_layers(atm_ctx* ctx, int replica, int z_lo, int z_hi);

/* Deterministic mode (on = 1; 0 = off, the default).  Repeated evaluations
 * and steps of the same state with the same launch options give bit-identical
 * forces, energies, virials and counts (without it, forces, energies and
 * virials vary at the rounding level from run to run: warps take work from
 * counters in the order they arrive and floating-point atomic additions
 * round in the order they happen).  In this mode
 *  - every warp takes its work in a fixed order (cell-triplet edge groups and
 *    candidate tasks of the block traversals, base molecules of 3C01 / 3CW),
 *    so each lane's energy and virial sums are the same every time;
 *  - the block traversals (3C18, 3C08, 3C08A) sum their pair scalars, their
 *    per-molecule fallback accumulators and the forces of different units as
 *    signed 64-bit integers in units of 2^-32 (FP32C) or 2^-44 (FP64): each
 *    term is rounded once to that grid and the sums do not depend on the
 *    order of the additions, so the forces are also the same for every launch
 *    form (one CTA per unit or persistent, warps per CTA, size classes);
 *    energies and virials then depend on the launch form only through the
 *    lanes' partial sums;
 *  - a term of size 2^26 (FP32C) or 2^14 = 16,384 (FP64) or more, which a
 *    liquid never reaches, makes the evaluation fail with ATM_E_RANGE.
 * 3C01 and 3CW write each force once (owner computes) and the LJ kernel owns
 * its molecules' sums, so they need no fixed point.  The surrogate is
 * unaffected (its kernels already sum in a fixed order).  Resets any tuned
 * choice and the current forces (the next step evaluates them).
 * Errors: INVALID. */
atm_status atm_set_deterministic(atm_ctx* ctx, int on);

/* Pair bitmaps for the FP32C pair rule of the block traversals (on = 1, the
 * default; 0 = off).  With them on, each force evaluation first decides every
 * pair of molecules in neighbouring cells once, in one kernel and its
 * transposition: 27 words per molecule (4 bytes each, held by the context),
 * bit j of word k set when the molecule and the j-th molecule of the
 * neighbour cell at offset k are closer
 * than r_c by the same FP32 arithmetic the units use (the canonical
 * displacement (xl_q - xl_p) + (o_q - o_p) w), and the 3C18 / 3C08 / 3C08A
 * units assemble their adjacency from those words instead of deciding each
 * pair of their 14 or 8 cells again.  The decisions, so the triplets and the
 * counts, are the same either way.  Used when every cell holds at most 32
 * molecules (the cell build's largest occupancy; graph steps whose cells fill
 * beyond that restart without the graph) and, for 3C18, when the cells are
 * wide enough in FP32 that cells two apart hold no pair within r_c.  Drops
 * any tuned choice and graph.  Errors: INVALID. */
atm_status atm_set_pair_masks(atm_ctx* ctx, int on);

/* Unit size classes of the block traversals (3C18, 3C08, 3C08A) for
 * evaluations and steps without an autotuned choice.  nclass = 1: every unit
 * in one launch sized for the largest unit (the default).  nclass = 2 or 3:
 * every force evaluation first lists, on the device, the units of at most
 * cuts[0] staged molecules, then (nclass = 3) those of at most cuts[1], then
 * the rest, and launches the block kernel once per class with shared memory
 * sized for the class bound (2 warps when it is at most 64): small units of
 * a batch of uneven replicas then share an SM with more of their kind.  The
 * first class runs on a stream the context owns, forked from the context's
 * stream after the sorting kernel and joined back before the evaluation
 * ends, so later work on the context's stream sees its results.  Counts are
 * those of one launch; energies and forces agree with it to rounding (the
 * class plans' warps and tables change the order of the additions).  cuts
 * (host, nclass - 1 values) must rise within 1 .. 2047.  Resets any
 * autotuned choice.  Errors: INVALID. */
atm_status atm_set_unit_classes(atm_ctx* ctx, int nclass, const int* cuts);

typedef struct {
    int persistent;     /* chosen launch form */
    int nwarps;         /* chosen warps per CTA */
    double ms_per_eval; /* device time of one LJ + ATM evaluation with it */
    int nclass;         /* unit size classes (1: all units in one launch) */
    int cut[2];         /* staged-molecule bounds of the first classes */
} atm_tuning;

/* Autotuner: times `reps` force evaluations on the current cells, in the form
 * steps take them (LJ inside the ATM units for the 3C18/3C08/3C08A pair
 * rule), for every launch form (one CTA per unit or persistent; 4 or 8 warps
 * for 3C18/3C08;
 * for 3C18/3C08/3C08A also unit size classes: {all}, {<= 64, rest},
 * {<= 48, <= 96, rest}, {<= 64, <= 128, rest}, where every force evaluation
 * sorts the units by their staged molecules on the device and launches each
 * class with shared memory sized for its bound, 2 warps for bounds up to 64)
 * and keeps the fastest for this (trav, trunc, prec); later evaluations and
 * steps use it.  Cells must be built.  out may be NULL.
 * Errors: INVALID, STATE, CAPACITY, CUDA. */
atm_status atm_autotune(atm_ctx* ctx, atm_traversal trav, atm_truncation trunc,
                        atm_precision prec, int reps, atm_tuning* out);

/* ---- Density profile (section 5, vapour-liquid slab) ---------------------
 * Adds, for every replica, the histogram of coordinate `axis` of the current
 * wrapped positions over nbins equal bins of [0, L_axis) (bin = floor(x / h),
 * h = L_axis / nbins, clamped to [0, nbins)) to a device accumulator.  Cells
 * must be built (the build wraps positions).  1 <= nbins <= 4096; the axis and
 * bin count must stay the same until atm_density_reset.
 * Errors: INVALID, STATE, CUDA. */
atm_status atm_density_accumulate(atm_ctx* ctx, int axis, int nbins);
/* counts[nrep * nbins] (replica-major) and the number of accumulated samples;
 * either may be NULL (synchronises). */
atm_status atm_density_get(atm_ctx* ctx, uint64_t* counts, int64_t* samples);
atm_status atm_density_reset(atm_ctx* ctx);

/* Allocation-free force evaluation.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc -- code that runs inside
 * a host application which owns and budgets all device memory up front, a
 * plug-in that is handed only raw device pointers, or a process whose
 * allocator must not be touched after start-up.  It does what atm_create +
 * atm_set_state_dev + atm_build_cells + atm_compute_forces + atm_get_forces_dev
 * (which = 0) do for one set of positions, but allocates nothing: every
 * intermediate array lives in one fixed __device__ array of about 6.7 MB that
 * this library reserves on every GPU it is loaded on, until the process exits.
 *
 *   params  box, rc, nu, LJ parameters, device, cuda_stream (dt is unused)
 *   n       molecules, 0 <= n <= ATM_NOALLOC_MAX_N
 *   x_dev   [3n] device positions (SoA, any real values; only read)
 *   f_dev   [3n] device output: total LJ + ATM force in the caller's order
 *   out     host scalars of the evaluation (ekin = 0), may be NULL
 *
 * Accepted: traversals ATM_3C01, ATM_3C18, ATM_3C08 and ATM_3C08A with either
 * truncation, precisions ATM_FP64 and ATM_FP32C.  ATM_3CW and ATM_SURROGATE
 * return INVALID (the wide traversal's 5^3 unit sizes and the surrogate's
 * model live in a context).
 * Errors: INVALID (NULL pointer, unknown enum, ATM_3CW, ATM_SURROGATE, device
 * index >= 64), BOX_TOO_SMALL, CAPACITY (n > ATM_NOALLOC_MAX_N, more than
 * ATM_NOALLOC_MAX_CELLS cells, or a unit that does not fit shared memory),
 * NONFINITE, CUDA.  There is no context, so no message: the status code is
 * the error.
 * The call makes params.device current while it runs and restores the
 * caller's current device before it returns.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress, with that device
 * current); make that first call before any stream capture.  The call
 * synchronises params.cuda_stream.  All
 * calls share the one array and leave their data in it (what must start at
 * zero is cleared on every call); calls whose GPU work overlaps -- on two
 * streams, or from two host threads -- race on it and must be serialised by
 * the caller. */
#define ATM_NOALLOC_MAX_N 32768
#define ATM_NOALLOC_MAX_CELLS 32768
atm_status atm_compute_forces_noalloc(const atm_params* params, int64_t n, const double* x_dev,
                                      atm_traversal trav, atm_truncation trunc,
                                      atm_precision prec, double* f_dev, atm_result* out);

/* ------------------------------------------------------------------------
 * Learned ATM force surrogate.  The paper has no counterpart: it evaluates
 * the triplet sum of Eq. atm / Eq. forcepairs exactly.  The surrogate replaces
 * that sum by a per-molecule model of the same force, for runs that trade a
 * stated force error for speed:
 *   neighbours j with r = |r_j - r_i| < r_c, rhat = (r_j - r_i) / r, cutoff
 *   f_c = (cos(pi r / r_c) + 1) / 2;
 *   D[0..15]  = sum_j exp(-eta_g (r - mu_k)^2) f_c, mu_k = 0.8 + k d_g,
 *               d_g = (r_c - 0.8) / 15, eta_g = 1 / (2 d_g^2);
 *   phi_a     = exp(-eta_v (r - nu_a)^2) f_c, nu_a = 0.8 + (a + 1/2) d_v,
 *               d_v = (r_c - 0.8) / 4, eta_v = 1 / (2 d_v^2), a = 0..3;
 *   p_a       = sum_j phi_a rhat, T_a = sum_j phi_a (rhat rhat^T - I/3) (a < 3);
 *   D[16..25] = p_a . p_b for ab = 00 01 02 03 11 12 13 22 23 33;
 *   D[26..31] = tr(T_a T_b) for ab = 00 01 02 11 12 22;
 *   vectors   v_m = p_m (m < 4), v_{4 + 4a + b} = T_a p_b (a < 3, b < 4);
 *   w = W3^T silu(W2^T silu(W1^T xn + b1) + b2) + b3 (16 outputs),
 *   xn = (D - mean) / scale;
 *   F_i = sum_m w_m v_m.
 * Parameters: ATM_SUR_NPARAM floats laid out W1[32][64], b1[64], W2[64][64],
 * b2[64], W3[64][16], b3[16] (row-major, input index first), plus mean[32] and
 * scale[32] (> 0).  Inference: inputs, weights and the two hidden layers in
 * bfloat16 on the tensor cores, FP32 sums.  Training: FP32 master weights;
 * gradients by default on the tensor cores (the inference arithmetic forward,
 * then the backward GEMMs with bfloat16 operands -- inputs, activations,
 * weights, dL/dw and the pre-activation gradients -- and FP32 sums), or in
 * FP32 on the CUDA cores (atm_surrogate_training_arithmetic); FP32
 * gradients, Adam (beta1 0.9, beta2 0.999, eps 1e-8) on the loss
 *   L = sum_i |F_i - F_i^ref|^2 / (3 B sigma2)
 * over a minibatch of B rows, sigma2 = mean squared target force component of
 * the data set (L = 1 for the zero model).
 * Descriptor / vector rows are float [rows][32] and [rows][48] (v_0 .. v_15),
 * targets float [rows][3]; all host arrays, caller-owned.
 * ------------------------------------------------------------------------ */
#define ATM_SUR_NDESC 32
#define ATM_SUR_NVEC 48
#define ATM_SUR_NOUT 16
#define ATM_SUR_NPARAM 7312

/* Set / get the model.  set_model copies (and validates: finite, scale > 0)
 * the parameters and resets the Adam state.  get_model accepts NULL for any
 * output.  STATE if no model was set or initialised. */
atm_status atm_surrogate_set_model(atm_ctx* ctx, const float* params, const float* mean,
                                   const float* scale);
atm_status atm_surrogate_get_model(atm_ctx* ctx, float* params, float* mean, float* scale);

/* Initialise a model for the current data set: mean / scale from its
 * descriptor columns (population deviation, 1 where below 1e-12), weights
 * uniform in +-sqrt(6 / (fan_in + fan_out)) from a splitmix64 stream of
 * `seed` (output layer times 0.1), biases 0.  STATE if the data set is empty. */
atm_status atm_surrogate_init(atm_ctx* ctx, uint64_t seed);

/* Model file: 8-byte tag "ATMSUR01", int32 parameter count, int32 descriptor
 * count, then params, mean, scale as little-endian float32.  IO errors return
 * INVALID with the reason in atm_last_error(). */
atm_status atm_surrogate_save(atm_ctx* ctx, const char* path);
atm_status atm_surrogate_load(atm_ctx* ctx, const char* path);

/* Descriptors and vectors of every molecule of the current cells (original
 * order), computed by the same kernel as the inference.  STATE without cells. */
atm_status atm_surrogate_descriptors(atm_ctx* ctx, float* desc, float* vec);

/* Inference on given rows (no neighbour search): w[rows][16] and
 * force[rows][3] = sum_m w_m vec_m.  STATE without a model. */
atm_status atm_surrogate_mlp(atm_ctx* ctx, int64_t rows, const float* desc, const float* vec,
                             float* w, float* force);

/* Loss and gradient of the current master parameters on given rows (the whole
 * set is one batch), in the arithmetic atm_surrogate_training_arithmetic
 * selects.  loss may be NULL; grad has ATM_SUR_NPARAM floats. */
atm_status atm_surrogate_loss_grad(atm_ctx* ctx, int64_t rows, const float* desc,
                                   const float* vec, const float* target, double sigma2,
                                   double* loss, float* grad);

/* Data set.  add_frame evaluates the exact ATM force (traversal, truncation,
 * precision FP64 or FP32C) on the current cells and appends one row per
 * molecule (its descriptors, vectors and that force).  add_rows appends given
 * rows.  The data set lives on the device and grows as needed. */
atm_status atm_surrogate_add_frame(atm_ctx* ctx, atm_traversal trav, atm_truncation trunc,
                                   atm_precision prec);
atm_status atm_surrogate_add_rows(atm_ctx* ctx, int64_t rows, const float* desc,
                                  const float* vec, const float* target);
atm_status atm_surrogate_dataset(atm_ctx* ctx, int64_t* rows, double* sigma2);
atm_status atm_surrogate_clear(atm_ctx* ctx);

/* `steps` Adam steps of learning rate lr.  batch <= 0 or >= the data-set size:
 * every step uses all rows in order; else each step draws `batch` rows with
 * replacement, row = splitmix64(seed, step, b) mod size.  loss (may be NULL)
 * receives the minibatch loss of each step.  STATE without model or data. */
atm_status atm_surrogate_train(atm_ctx* ctx, int64_t steps, int64_t batch, double lr,
                               uint64_t seed, double* loss);

/* Arithmetic of the gradients of atm_surrogate_train and atm_surrogate_loss_grad:
 * tensor_cores = 1 (the default): tcgen05 GEMMs with bfloat16 operands and
 * FP32 accumulators, 128 samples per tile, the forward pass in the inference
 * kernel's arithmetic; 0: FP32 on the CUDA cores (64 samples per block,
 * FP32 activations).  Errors: INVALID. */
atm_status atm_surrogate_training_arithmetic(atm_ctx* ctx, int tensor_cores);

/* atm_step with ATM_SURROGATE: every `exact_every` steps (0 = never; default
 * 50) the step uses the exact FP32C traversal instead and the surrogate is
 * compared with it on that configuration.  atm_surrogate_error returns the
 * accumulated comparison: RMS of the force difference and of the exact force
 * (per component) and the number of comparisons; reset != 0 clears it. */
atm_status atm_surrogate_options(atm_ctx* ctx, int exact_every);
atm_status atm_surrogate_error(atm_ctx* ctx, double* rms_diff, double* rms_exact,
                               int64_t* checks, int reset);

/* Give the total force of the state just set (host memory, f[3n], original
 * order, as atm_get_forces(..., 0) returns it) as computed with (trav, trunc,
 * prec): the next atm_step with that combination uses it for its first half
 * kick instead of evaluating the forces of the state again -- velocity
 * Verlet carries the force with the state, so a caller that keeps the state
 * on the host between steps keeps it too.  Must follow atm_set_state (which
 * forgets it); the library does not check that it belongs to the state.
 * Errors: INVALID (surrogate or unknown combination, NULL), STATE (no state),
 * NONFINITE, CUDA. */
atm_status atm_set_forces(atm_ctx* ctx, const double* f, atm_traversal trav, atm_truncation trunc,
                          atm_precision prec);

/* Velocity-rescaling thermostat for the NVT runs of section 5.1 (the paper
 * names no thermostat): the velocities of replica r are scaled by
 * sqrt(T_r (3 N_r - 3) / (2 K_r)) so that its kinetic temperature
 * 2 K / (3 N - 3) becomes t_target[r] (host array of R values >= 0,
 * INVALID otherwise); a replica with K = 0 or N < 2 is left alone.  Called
 * between atm_step calls (every k steps); synchronises; the results then
 * report the new kinetic energy.  STATE without a state. */
atm_status atm_thermostat(atm_ctx* ctx, const double* t_target);

/* Radial distribution (paper section 5, Fig. rdfs): adds to a per-replica
 * integer histogram every pair once with r < r_max, bin floor(r / (r_max /
 * nbins)), r from the FP64 canonical displacement of the linked cells.
 * r_max must not exceed the smallest cell edge (INVALID); needs built cells
 * (STATE); range and bins are fixed until reset.  get copies counts
 * [R][nbins] (uint64) and the number of accumulated configurations.
 * g(r) = counts / (samples * N / 2 * rho * shell volume). */
atm_status atm_rdf_accumulate(atm_ctx* ctx, double r_max, int nbins);
atm_status atm_rdf_get(atm_ctx* ctx, uint64_t* counts, int64_t* samples);
atm_status atm_rdf_reset(atm_ctx* ctx);

/* Long-range corrections of the truncated (unshifted) LJ pair terms of a
 * homogeneous system (section 5 applies them to E2 and P2; the standard
 * tail integrals): e_tail = 8/3 pi N rho eps sigma^3 [(sigma/r_c)^9 / 3 -
 * (sigma/r_c)^3], p_tail = 16/3 pi rho^2 eps sigma^3 [2/3 (sigma/r_c)^9 -
 * (sigma/r_c)^3], rho = N / V.  Host arithmetic; either output may be NULL. */
atm_status atm_lj_tail(const atm_params* params, int64_t n, double* e_tail, double* p_tail);

/* Measured fused multiply-add throughput of the device (TFLOP/s, one FMA = 2
 * flops): a kernel of independent FMA chains in FP32 (fp64 = 0) or FP64,
 * best of three timed launches.  Roofline context for the ALU-bound kernels;
 * the paper has no counterpart. */
atm_status atm_measure_fma_peak(int device, int fp64, double* tflops);
/* Measured FP32 reciprocal-square-root throughput (rsqrtf, the special-function
 * unit) in G operations/s, measured the same way; it bounds the one rsqrt per
 * triplet.  Errors: INVALID (NULL output, negative device), CUDA. */
atm_status atm_measure_rsqrt_peak(int device, double* gops);

/* Device-time profile of the library's own kernels (CUDA events recorded on
 * the context's stream around each group of launches while profiling is on).
 * ms_*: summed device time since profiling was (re)enabled; n_launches: kernels
 * this library launched since then (profiling on or off: counted always since
 * the last atm_set_profiling call); n_atm_launches: ATM triplet kernels among them. */
typedef struct {
    double ms_cells, ms_lj, ms_atm, ms_md;
    int64_t n_launches, n_atm_launches;
} atm_profile;

/* on = 1: start recording every launch group (and reset the sums and
 * counters); on = 2: the same for the force evaluations only (ms_atm; the
 * other sums stay 0), which puts fewer timestamps between a step's kernels;
 * 0: stop. */
atm_status atm_set_profiling(atm_ctx* ctx, int on);
/* Synchronises the stream and returns the sums. */
atm_status atm_get_profile(atm_ctx* ctx, atm_profile* out);

#ifdef __cplusplus
}
#endif
#endif
