// capi.cu -- the C ABI declared in include/atm3.h: context (a batch of one or
// more replicas), buffers, call order, CUDA-graph steps, autotuning.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "atm3.h"
#include "atm3_internal.cuh"
#include "forces.cuh"
#include "md_kernels.cuh"
#include "ctx.cuh"
#include "surrogate.cuh"

using namespace atm3;

namespace {
constexpr int DENS_MAX_BINS = 4096;
constexpr int CELL_KERNELS = 5;  // wrap/bin, scan, unit sizes, scatter, per-cell order

// steps under the 3c08, corner-anchored 3c08 or 3c18 pair rule evaluate LJ inside the ATM units
static bool lj_fused(int trav, int trunc, int prec)
{
    return (trav == ATM_3C08 || trav == ATM_3C08A || trav == ATM_3C18) && trunc == ATM_TRUNC_PAIR &&
           prec != ATM_SURROGATE;
}

// unit size classes the autotuner chooses among for the block traversals:
// {classes, bound of the first, bound of the second}
constexpr int N_SPLITS = 4;
constexpr int SPLITS[N_SPLITS][3] = {{1, 0, 0}, {2, 64, 0}, {3, 48, 96}, {3, 64, 128}};

// kernels of one step: two kicks, the cell build and the force kernels (with
// ncls > 1 size classes: the class kernel and one ATM launch per class)
static int kernels_per_step(int trav, int trunc, int prec, int ncls)
{
    int forces = prec == ATM_SURROGATE ? SUR_LAUNCHES : (lj_fused(trav, trunc, prec) ? 1 : 2);
    if (ncls > 1 && prec != ATM_SURROGATE) forces += ncls;
    return 2 + CELL_KERNELS + forces;
}
}  // namespace


enum { PK_CELLS = 0, PK_LJ = 1, PK_ATM = 2, PK_MD = 3 };

cudaEvent_t atm3::ctx_prof_begin(atm_ctx* c, int kind)
{
    // level 2 times the force evaluations only: fewer timestamps between the
    // step's other kernels
    if (!c->prof || (c->prof == 2 && kind != PK_ATM)) return nullptr;
    cudaEvent_t e = nullptr;
    if (!c->ev_pool.empty()) {
        e = c->ev_pool.back();
        c->ev_pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        return nullptr;
    }
    cudaEventRecord(e, c->st);
    return e;
}

void atm3::ctx_prof_end(atm_ctx* c, int kind, cudaEvent_t a)
{
    if (!c->prof || !a) return;
    cudaEvent_t b = nullptr;
    if (!c->ev_pool.empty()) {
        b = c->ev_pool.back();
        c->ev_pool.pop_back();
    } else if (cudaEventCreate(&b) != cudaSuccess) {
        c->ev_pool.push_back(a);
        return;
    }
    cudaEventRecord(b, c->st);
    c->ev_live.push_back({a, b, kind});
}

// fold completed event pairs into the sums (call after a stream synchronisation)
static void prof_drain(atm_ctx* c)
{
    for (auto& r : c->ev_live) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) c->prof_ms[r.kind] += ms;
        c->ev_pool.push_back(r.a);
        c->ev_pool.push_back(r.b);
    }
    c->ev_live.clear();
    cudaGetLastError();
}

atm_status atm3::ctx_fail(atm_ctx* c, atm_status s, const char* fmt, ...)
{
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return s;
}


static void drop_graph(atm_ctx* c)
{
    if (c->graph) cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
    for (int& k : c->graph_key) k = -1;
}

static void free_all(atm_ctx* c)
{
    drop_graph(c);
    sur_free(c);
    void* dev[] = {c->d_rep, c->d_rep_of_cell, c->d_rep_of_mol, c->x, c->v, c->x0, c->v0, c->xl,
                   c->xl32, c->cell_of, c->rank, c->count, c->start, c->perm, c->cell_sorted,
                   c->f_lj, c->f_atm, c->f_out, c->unit_ew, c->unit_cnt, c->mol_ew, c->mol_cnt,
                   c->ke, c->d_res, c->d_part, c->d_status, c->d_maxocc, c->d_work, c->d_dens,
                   c->d_rdf, c->d_ttarget, c->unit_ew2, c->unit_cnt2, c->f_in, c->d_chk,
                   c->d_ulist, c->d_ucount, c->pmask};
    for (void* p : dev)
        if (p) cudaFree(p);
    if (c->h_res) cudaFreeHost(c->h_res);
    if (c->h_status) cudaFreeHost(c->h_status);
    if (c->h_chk) cudaFreeHost(c->h_chk);
    if (c->h_maxocc) cudaFreeHost(c->h_maxocc);
    if (c->cap_st) cudaStreamDestroy(c->cap_st);
    if (c->side_st) cudaStreamDestroy(c->side_st);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->io_st) cudaStreamDestroy(c->io_st);
    if (c->ev_io) cudaEventDestroy(c->ev_io);
    if (c->ev_io_done) cudaEventDestroy(c->ev_io_done);
    for (auto& r : c->ev_live) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    c->ev_live.clear();
    c->ev_pool.clear();
}

static atm_status check_status(atm_ctx* c)
{
    int s = *c->h_status;
    if (s == 0) return ATM_OK;
    *c->h_status = 0;
    cudaMemsetAsync(c->d_status, 0, sizeof(int), c->st);
    // capacity first: a unit skipped for capacity during graph steps leaves its
    // molecules without forces, and what follows (overlaps, non-finite
    // positions) is its consequence; graph steps restart on ATM_E_CAPACITY
    if (s & ST_CAPACITY)
        return ctx_fail(c, ATM_E_CAPACITY, "a traversal unit holds more molecules than staged");
    if (s & ST_NONFINITE) return ctx_fail(c, ATM_E_NONFINITE, "non-finite position or velocity");
    if (s & ST_TIMEOUT)
        return ctx_fail(c, ATM_E_TIMEOUT, "a device-side wait for the tensor cores gave up");
    if (s & ST_RANGE)
        return ctx_fail(c, ATM_E_RANGE,
                        "deterministic mode: a force term exceeds the fixed-point range");
    return ctx_fail(c, ATM_E_CUDA, "device status %d", s);
}

atm_status atm3::ctx_sync_and_check(atm_ctx* c)
{
    CU(cudaMemcpyAsync(c->h_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    CU(cudaStreamSynchronize(c->st));
    // the profiling events are folded in by atm_get_profile, or here once
    // many are pending: a step's own synchronisation (the cell build's) is on
    // its critical path, and querying events there would lengthen it
    if (c->ev_live.size() >= 4096) prof_drain(c);
    return check_status(c);
}

extern "C" int atm_abi_version(void) { return ATM3_ABI_VERSION; }

extern "C" const char* atm_last_error(const atm_ctx* c)
{
    return c ? c->err : "null context";
}

extern "C" atm_status atm_batch_create(const atm_params* params, const int64_t* n, int nrep,
                                       atm_ctx** out)
{
    if (!out) return ATM_E_INVALID;
    *out = nullptr;
    if (!params || !n || nrep < 1 || nrep > (1 << 20)) return ATM_E_INVALID;
    atm_ctx* c = new (std::nothrow) atm_ctx();
    if (!c) return ATM_E_INVALID;
    c->R = nrep;
    c->device = params[0].device;
    c->st = (cudaStream_t)params[0].cuda_stream;
    long long ntot = 0, ncell = 0;
    for (int r = 0; r < nrep; r++) {
        if (n[r] < 0 || ntot + n[r] > (long long)0x7fffffff - 1) {
            delete c;
            return ATM_E_INVALID;
        }
        Rep rp;
        atm_status s = make_rep(params[r], n[r], ntot, ncell, rp);
        if (s != ATM_OK) {
            delete c;
            return s;
        }
        c->params.push_back(params[r]);
        c->reps.push_back(rp);
        ntot += n[r];
        ncell += rp.g.ncell;
        if (ncell > (1ll << 30)) {
            delete c;
            return ATM_E_INVALID;
        }
    }
    c->n = ntot;
    c->ncell = ncell;
    // a pair two cells apart is at least a cell edge w apart along that axis,
    // and its FP32 squared distance at least fl(wf * wf): no pair within r_c
    // when that is not below the FP32 r_c^2 (the 3c18 units' outer slots)
    c->pm_3c18 = true;
    for (const atm3::Rep& r : c->reps)
        for (int d = 0; d < 3; d++) {
            volatile float wf = r.wf[d];
            volatile float w2 = wf * wf;
            if (!(w2 >= r.rc2f)) c->pm_3c18 = false;
        }
    auto alloc = [&](void** ptr, size_t bytes) -> bool {
        return cudaMalloc(ptr, bytes > 0 ? bytes : 16) == cudaSuccess;
    };
    bool ok = cudaSetDevice(c->device) == cudaSuccess;
    const size_t N = (size_t)(ntot > 0 ? ntot : 1), NC = (size_t)ncell;
    ok = ok && alloc((void**)&c->d_rep, nrep * sizeof(Rep));
    ok = ok && alloc((void**)&c->d_rep_of_cell, NC * sizeof(int));
    ok = ok && alloc((void**)&c->d_rep_of_mol, N * sizeof(int));
    ok = ok && alloc((void**)&c->x, 3 * N * sizeof(double));
    ok = ok && alloc((void**)&c->v, 3 * N * sizeof(double));
    ok = ok && alloc((void**)&c->x0, 3 * N * sizeof(double));
    ok = ok && alloc((void**)&c->v0, 3 * N * sizeof(double));
    ok = ok && alloc((void**)&c->xl, 3 * N * sizeof(double));
    ok = ok && alloc((void**)&c->xl32, 3 * N * sizeof(float));
    ok = ok && alloc((void**)&c->cell_of, N * sizeof(int));
    ok = ok && alloc((void**)&c->rank, N * sizeof(int));
    ok = ok && alloc((void**)&c->count, NC * sizeof(int));
    ok = ok && alloc((void**)&c->start, (NC + 1) * sizeof(int));
    ok = ok && alloc((void**)&c->perm, N * sizeof(int));
    ok = ok && alloc((void**)&c->cell_sorted, N * sizeof(int));
    ok = ok && alloc((void**)&c->f_lj, 3 * N * sizeof(double));
    ok = ok && alloc((void**)&c->f_atm, 3 * N * sizeof(double));
    ok = ok && alloc((void**)&c->f_out, 3 * N * sizeof(double));
    ok = ok && alloc((void**)&c->f_in, 3 * N * sizeof(double));
    ok = ok && alloc((void**)&c->d_chk, sizeof(int));
    ok = ok && alloc((void**)&c->unit_ew, 2 * NC * sizeof(double));
    ok = ok && alloc((void**)&c->unit_cnt, 2 * NC * sizeof(unsigned long long));
    ok = ok && alloc((void**)&c->unit_ew2, 2 * NC * sizeof(double));
    ok = ok && alloc((void**)&c->unit_cnt2, 2 * NC * sizeof(unsigned long long));
    ok = ok && alloc((void**)&c->mol_ew, 2 * N * sizeof(double));
    ok = ok && alloc((void**)&c->mol_cnt, 2 * N * sizeof(unsigned));
    ok = ok && alloc((void**)&c->ke, N * sizeof(double));
    ok = ok && alloc((void**)&c->d_res, nrep * sizeof(ResultDev));
    ok = ok && alloc((void**)&c->d_part, (size_t)nrep * REDUCE_PARTS * sizeof(ResultDev));
    ok = ok && alloc((void**)&c->d_status, sizeof(int));
    // largest cell, largest unit per traversal, edge-table need per traversal
    ok = ok && alloc((void**)&c->d_maxocc, (1 + 2 * ATM_NTRAV) * sizeof(int));
    ok = ok && cudaMemset(c->d_maxocc, 0, (1 + 2 * ATM_NTRAV) * sizeof(int)) == cudaSuccess;
    ok = ok && alloc((void**)&c->d_work, 4 * sizeof(int));
    ok = ok && alloc((void**)&c->d_ulist, 3 * NC * sizeof(int));
    ok = ok && alloc((void**)&c->d_ucount, 4 * sizeof(int));
    ok = ok && alloc((void**)&c->d_dens, (size_t)nrep * DENS_MAX_BINS * sizeof(unsigned long long));
    ok = ok && alloc((void**)&c->d_rdf, (size_t)nrep * DENS_MAX_BINS * sizeof(unsigned long long));
    ok = ok && alloc((void**)&c->d_ttarget, nrep * sizeof(double));
    ok = ok && alloc((void**)&c->pmask, atm3::PM_WORDS * N * sizeof(unsigned));
    ok = ok && cudaMallocHost((void**)&c->h_res, nrep * sizeof(ResultDev)) == cudaSuccess;
    ok = ok && cudaMallocHost((void**)&c->h_status, sizeof(int)) == cudaSuccess;
    ok = ok && cudaMallocHost((void**)&c->h_chk, sizeof(int)) == cudaSuccess;
    ok = ok && cudaMallocHost((void**)&c->h_maxocc, (1 + 2 * ATM_NTRAV) * sizeof(int)) == cudaSuccess;
    ok = ok && cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                                      c->device) == cudaSuccess;
    ok = ok && cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device) ==
                   cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&c->cap_st, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&c->side_st, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&c->io_st, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&c->ev_io, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&c->ev_io_done, cudaEventDisableTiming) == cudaSuccess;
    if (ok) {
        std::vector<int> roc(NC), rom(N, 0);
        for (int r = 0; r < nrep; r++) {
            for (long long q = 0; q < c->reps[r].g.ncell; q++) roc[c->reps[r].cell0 + q] = r;
            for (long long q = 0; q < c->reps[r].n; q++) rom[c->reps[r].mol0 + q] = r;
        }
        ok = ok && cudaMemcpy(c->d_rep, c->reps.data(), nrep * sizeof(Rep),
                              cudaMemcpyHostToDevice) == cudaSuccess;
        ok = ok && cudaMemcpy(c->d_rep_of_cell, roc.data(), NC * sizeof(int),
                              cudaMemcpyHostToDevice) == cudaSuccess;
        ok = ok && cudaMemcpy(c->d_rep_of_mol, rom.data(), N * sizeof(int),
                              cudaMemcpyHostToDevice) == cudaSuccess;
    }
    ok = ok && cudaMemsetAsync(c->d_status, 0, sizeof(int), c->st) == cudaSuccess;
    ok = ok && cudaMemsetAsync(c->v, 0, 3 * N * sizeof(double), c->st) == cudaSuccess;
    ok = ok && cudaMemsetAsync(c->mol_ew, 0, 2 * N * sizeof(double), c->st) == cudaSuccess;
    ok = ok && cudaMemsetAsync(c->mol_cnt, 0, 2 * N * sizeof(unsigned), c->st) == cudaSuccess;
    ok = ok && cudaMemsetAsync(c->unit_ew, 0, 2 * NC * sizeof(double), c->st) == cudaSuccess;
    ok = ok && cudaMemsetAsync(c->unit_cnt, 0, 2 * NC * sizeof(unsigned long long), c->st) ==
                   cudaSuccess;
    ok = ok && cudaMemsetAsync(c->d_dens, 0, (size_t)nrep * DENS_MAX_BINS * 8, c->st) == cudaSuccess;
    ok = ok && cudaMemsetAsync(c->d_rdf, 0, (size_t)nrep * DENS_MAX_BINS * 8, c->st) == cudaSuccess;
    ok = ok && cudaStreamSynchronize(c->st) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_all(c);
        delete c;
        return ATM_E_CUDA;
    }
    c->b.rep = c->d_rep;
    c->b.rep_of_cell = c->d_rep_of_cell;
    c->b.rep_of_mol = c->d_rep_of_mol;
    c->b.R = nrep;
    c->b.ntot = ntot;
    c->b.ncell = ncell;
    *c->h_status = 0;
    *out = c;
    return ATM_OK;
}

extern "C" atm_status atm_create(const atm_params* params, int64_t n, atm_ctx** out)
{
    return atm_batch_create(params, &n, 1, out);
}

extern "C" atm_status atm_batch_size(const atm_ctx* c, int* nrep, int64_t* ntot)
{
    if (!c) return ATM_E_INVALID;
    if (nrep) *nrep = c->R;
    if (ntot) *ntot = c->n;
    return ATM_OK;
}

extern "C" atm_status atm_batch_cells(const atm_ctx* c, int64_t* ncell)
{
    if (!c || !ncell) return ATM_E_INVALID;
    *ncell = c->ncell;
    return ATM_OK;
}

extern "C" atm_status atm_cell_grid(const atm_params* p, int32_t* ncell3)
{
    if (!p || !ncell3) return ATM_E_INVALID;
    atm3::Rep r;
    const atm_status st = atm3::make_rep(*p, 0, 0, 0, r);
    if (st != ATM_OK) return st;
    for (int d = 0; d < 3; d++) ncell3[d] = r.g.nc[d];
    return ATM_OK;
}

extern "C" atm_status atm_destroy(atm_ctx* c)
{
    if (!c) return ATM_OK;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->st);
    free_all(c);
    delete c;
    return ATM_OK;
}

static void invalidate(atm_ctx* c)
{
    c->cells_built = false;
    c->forces_valid = false;
    c->f_in_valid = false;
}

// copies m doubles from host memory to dev and checks them for NaN / Inf on
// the device (the copy's data, one pass); synchronises, so the caller may
// reuse its buffer on return.  *bad: a non-finite element was found
// copies host arrays (a, and b when given, m doubles each) to the device,
// checks them for non-finite values there and waits once for their result
static atm_status copy_in_checked(atm_ctx* c, double* dev_a, const double* host_a, double* dev_b,
                                  const double* host_b, long long m, bool* bad)
{
    *bad = false;
    if (m <= 0) return ATM_OK;
    CU(cudaMemsetAsync(c->d_chk, 0, sizeof(int), c->st));
    CU(cudaMemcpyAsync(dev_a, host_a, (size_t)m * sizeof(double), cudaMemcpyHostToDevice, c->st));
    CU(launch_check_finite(m, dev_a, c->d_chk, c->st));
    c->n_launch += 1;
    if (host_b) {
        CU(cudaMemcpyAsync(dev_b, host_b, (size_t)m * sizeof(double), cudaMemcpyHostToDevice, c->st));
        CU(launch_check_finite(m, dev_b, c->d_chk, c->st));
        c->n_launch += 1;
    }
    CU(cudaMemcpyAsync(c->h_chk, c->d_chk, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    CU(cudaStreamSynchronize(c->st));
    *bad = *c->h_chk != 0;
    return ATM_OK;
}

extern "C" atm_status atm_set_state(atm_ctx* c, const double* x, const double* v)
{
    if (!c) return ATM_E_INVALID;
    if (!x && c->n > 0) return ctx_fail(c, ATM_E_INVALID, "positions are required");
    CU(cudaSetDevice(c->device));
    const long long m = 3 * c->n;
    bool bad = false;
    if (!v && m > 0) CU(cudaMemsetAsync(c->v, 0, (size_t)m * sizeof(double), c->st));
    atm_status s = copy_in_checked(c, c->x, x, c->v, v, m, &bad);
    if (s != ATM_OK) return s;
    c->have_x = !bad;
    invalidate(c);
    if (bad) {
        long long q = 0;
        while (q < m && std::isfinite(x[q]) && (!v || std::isfinite(v[q]))) q++;
        return ctx_fail(c, ATM_E_NONFINITE, "non-finite input at element %lld", q);
    }
    return ATM_OK;
}

extern "C" atm_status atm_set_state_dev(atm_ctx* c, const double* x_dev, const double* v_dev)
{
    if (!c) return ATM_E_INVALID;
    if (!x_dev && c->n > 0) return ctx_fail(c, ATM_E_INVALID, "positions are required");
    CU(cudaSetDevice(c->device));
    size_t bytes = 3 * (size_t)c->n * sizeof(double);
    if (bytes) {
        CU(cudaMemcpyAsync(c->x, x_dev, bytes, cudaMemcpyDeviceToDevice, c->st));
        if (v_dev)
            CU(cudaMemcpyAsync(c->v, v_dev, bytes, cudaMemcpyDeviceToDevice, c->st));
        else
            CU(cudaMemsetAsync(c->v, 0, bytes, c->st));
        CU(launch_check_finite(3 * c->n, c->x, c->d_status, c->st));
        CU(launch_check_finite(3 * c->n, c->v, c->d_status, c->st));
        c->n_launch += 2;
    }
    c->have_x = true;
    invalidate(c);
    return ATM_OK;
}

// cell build kernels only (no host synchronisation; capturable)
static atm_status launch_cells(atm_ctx* c)
{
    cudaEvent_t ev = ctx_prof_begin(c, PK_CELLS);
    CU(launch_build_cells(c->b, c->x, c->cell_of, c->rank, c->count, c->start, c->perm, c->xl,
                          c->xl32, c->cell_sorted, c->d_maxocc, c->d_status, c->wide_cells,
                          c->st));
    ctx_prof_end(c, PK_CELLS, ev);
    c->n_launch += c->n > 0 ? CELL_KERNELS : 2;
    return ATM_OK;
}

// the unit sizes of the last cell build and the edge-table needs recorded by
// the units so far (h_maxocc, after a synchronisation): each traversal's
// table capacity becomes its need plus a quarter edge per staged molecule
// (the needs only grow, so a system that changes slowly keeps its capacity)
static void take_unit_sizes(atm_ctx* c)
{
    c->maxocc = c->h_maxocc[0];
    for (int t = 0; t < ATM_NTRAV; t++) {
        c->unit_max[t] = c->h_maxocc[1 + t];
        const int need = c->h_maxocc[1 + ATM_NTRAV + t];
        const int g = need > 0 ? std::min(256, need + 4) : c->gpm16[t];
        if (g != c->gpm16[t]) {
            c->gpm16[t] = g;
            memset(c->nw_auto[t], 0, sizeof(c->nw_auto[t]));  // keyed by unit size only
        }
    }
}

// cell build + read back of the occupancy maxima that size the force kernels
static atm_status enqueue_cells(atm_ctx* c)
{
    atm_status s = launch_cells(c);
    if (s != ATM_OK) return s;
    CU(cudaMemcpyAsync(c->h_maxocc, c->d_maxocc, (1 + 2 * ATM_NTRAV) * sizeof(int),
                       cudaMemcpyDeviceToHost, c->st));
    s = ctx_sync_and_check(c);
    if (s != ATM_OK) return s;
    take_unit_sizes(c);
    c->cells_built = true;
    c->forces_valid = false;
    return ATM_OK;
}

// the wide traversal's units are sized by cell builds only once it is in use:
// the first request rebuilds the (unchanged) cells with that size
atm_status atm3::ctx_want_wide(atm_ctx* c, int trav)
{
    if (trav != ATM_3CW || c->wide_cells) return ATM_OK;
    c->wide_cells = true;
    drop_graph(c);
    return c->cells_built ? enqueue_cells(c) : ATM_OK;
}

extern "C" atm_status atm_build_cells(atm_ctx* c)
{
    if (!c) return ATM_E_INVALID;
    if (!c->have_x) return ctx_fail(c, ATM_E_STATE, "no state set");
    CU(cudaSetDevice(c->device));
    return enqueue_cells(c);
}

extern "C" atm_status atm_get_cells(atm_ctx* c, int32_t* cell_of, int32_t* cell_start,
                                    int32_t* perm, int32_t* ncell3)
{
    if (!c) return ATM_E_INVALID;
    if (ncell3)
        for (int d = 0; d < 3; d++) ncell3[d] = c->reps[0].g.nc[d];
    if (!c->cells_built) return ctx_fail(c, ATM_E_STATE, "cells not built");
    CU(cudaSetDevice(c->device));
    if (cell_of && c->n)
        CU(cudaMemcpyAsync(cell_of, c->cell_of, c->n * sizeof(int), cudaMemcpyDeviceToHost, c->st));
    if (cell_start)
        CU(cudaMemcpyAsync(cell_start, c->start, (c->ncell + 1) * sizeof(int),
                           cudaMemcpyDeviceToHost, c->st));
    if (perm && c->n)
        CU(cudaMemcpyAsync(perm, c->perm, c->n * sizeof(int), cudaMemcpyDeviceToHost, c->st));
    CU(cudaStreamSynchronize(c->st));
    return ATM_OK;
}

// launch options of one force evaluation: the tuned choice, else the context's
// options; cls = {classes, first bound, second bound} (1 class: all units in
// one launch)
static int atm_ctas_per_sm(const atm_ctx* c, int trav, int trunc, int prec, int nwarps, int mcap);

static void launch_choice(atm_ctx* c, int trav, int trunc, int prec, int mcap, int& persistent,
                          int& nwarps, int cls[3])
{
    int t = c->tuned[prec][trav][trunc];
    if (t) {
        persistent = (t - 1) & 1;
        nwarps = ((t - 1) & 2) ? 8 : 4;
        for (int k = 0; k < 3; k++) cls[k] = SPLITS[(t - 1) >> 2][k];
    } else {
        persistent = c->opt_persistent;
        nwarps = c->opt_nwarps;
        for (int k = 0; k < 3; k++) cls[k] = c->opt_cls[k];
        if (nwarps == 0 && prec == ATM_FP32C && trunc == ATM_TRUNC_PAIR && !c->det &&
            (trav == ATM_3C18 || trav == ATM_3C08 || trav == ATM_3C08A) && mcap > 0) {
            // without a tuned choice: 4 or 8 warps, whichever keeps more warps
            // resident per SM for this unit size (4 on a tie).  Measured
            // (256k / 32k liquids): 3c08 1.20 / 0.27 ms at 4 and 1.50 / 0.23 ms
            // at 8 warps, 3c18 1.98 / 0.85 at 4 and 1.70 / 0.55 at 8.  (Not
            // the deterministic mode: its 8-byte scalars change the balance,
            // and 8 warps measured slower there, 1.87 against 1.70 ms.)
            int* e = c->nw_auto[trav][trunc];
            const int band = mcap / 8 + 1;
            if (e[0] != band) {
                const int w4 = 4 * atm_ctas_per_sm(c, trav, trunc, prec, 4, mcap);
                const int w8 = 8 * atm_ctas_per_sm(c, trav, trunc, prec, 8, mcap);
                e[0] = band;
                e[1] = w8 > w4 ? 8 : 4;
            }
            nwarps = e[1];
        }
    }
    if (trav == ATM_3C01 || trav == ATM_3CW) {
        nwarps = 0;
        cls[0] = 1;
    }
}

// pair rule of a block traversal outside the deterministic mode (whose
// results must not depend on the context's history): the units record their
// edge-table need and the table is sized from it
static bool measured_edges(const atm_ctx* c, int trav, int trunc)
{
    return trunc == ATM_TRUNC_PAIR && !c->det &&
           (trav == ATM_3C18 || trav == ATM_3C08 || trav == ATM_3C08A);
}

// edge-table capacity of a launch, 1/16 edges per staged molecule
static int edge_capacity(const atm_ctx* c, int trav, int trunc)
{
    return measured_edges(c, trav, trunc) ? c->gpm16[trav] : 256;
}

// FP32 pair rule of a block traversal, bitmaps enabled, every cell within 32
static bool use_pair_masks(const atm_ctx* c, int trav, int trunc, int prec)
{
    return c->opt_pmask && c->pmask && prec == ATM_FP32C && trunc == ATM_TRUNC_PAIR &&
           (trav == ATM_3C08 || trav == ATM_3C08A || (trav == ATM_3C18 && c->pm_3c18)) &&
           c->maxocc <= atm3::PM_CELL_MAX;
}

// LJ + ATM force kernels for the current cells; mcap = staged-molecule capacity
atm_status atm3::ctx_enqueue_forces(atm_ctx* c, int trav, int trunc, int prec, int mcap,
                                    bool fuse_lj)
{
    const bool fused = fuse_lj && lj_fused(trav, trunc, prec);
    if (prec == ATM_SURROGATE)
        for (const Rep& r : c->reps)
            if (r.own_z0 != 0 || r.own_z1 != r.g.nc[2])
                return ctx_fail(c, ATM_E_INVALID, "the surrogate evaluates whole replicas (owned layers set)");
    if (trav == ATM_3CW)
        for (const Rep& r : c->reps)
            if (r.g.nc[0] < 5 || r.g.nc[1] < 5 || r.g.nc[2] < 5)
                return ctx_fail(c, ATM_E_BOX_TOO_SMALL, "the wide traversal needs 5 cells per axis");
    ForceJob j;
    j.b = c->b;
    j.rep_host = c->reps.data();
    j.xl = c->xl;
    j.xl32 = c->xl32;
    j.start = c->start;
    j.cell_sorted = c->cell_sorted;
    j.f_lj = c->f_lj;
    j.f_atm = c->f_atm;
    j.mol_ew = c->mol_ew;
    j.mol_cnt = c->mol_cnt;
    j.unit_ew = c->unit_ew;
    j.unit_cnt = c->unit_cnt;
    j.lj = fused ? 1 : 0;
    j.unit_ew2 = c->unit_ew2;
    j.unit_cnt2 = c->unit_cnt2;
    j.status = c->d_status;
    j.work = c->d_work;
    j.trav = trav;
    j.trunc = trunc;
    // the surrogate runs LJ in FP32
    j.prec = prec == ATM_SURROGATE ? ATM_FP32C : prec;
    j.mcap = mcap > 0 ? mcap : 1;
    j.optin = c->smem_optin;
    j.sms = c->sms;
    j.persistent = 0;
    j.nwarps = 0;
    int cls[3] = {1, 0, 0};
    // (the warps follow the current unit size, also when a graph sizes the
    // launch for more)
    if (prec != ATM_SURROGATE)
        launch_choice(c, trav, trunc, prec, c->unit_max[trav], j.persistent, j.nwarps, cls);
    j.ncls = cls[0];
    j.cuts[0] = cls[1];
    j.cuts[1] = cls[2];
    j.ulist = c->d_ulist;
    j.ucount = c->d_ucount;
    j.st = c->st;
    j.side_st = c->side_st;
    j.ev_fork = c->ev_fork;
    j.ev_join = c->ev_join;
    j.det = c->det;
    j.pmask = use_pair_masks(c, trav, trunc, prec) ? c->pmask : nullptr;
    j.gpm16 = edge_capacity(c, trav, trunc);
    j.emax = measured_edges(c, trav, trunc) ? c->d_maxocc + 1 + ATM_NTRAV + trav : nullptr;

    cudaEvent_t ev;
    if (prec != ATM_SURROGATE && !fused) {
        // (the surrogate's descriptor pass computes LJ from the same neighbours)
        ev = ctx_prof_begin(c, PK_LJ);
        CU(enqueue_lj(j));
        ctx_prof_end(c, PK_LJ, ev);
        c->n_launch += 1;
    }

    ev = ctx_prof_begin(c, PK_ATM);
    if (prec == ATM_SURROGATE) {
        atm_status s = sur_enqueue_atm(c);
        if (s != ATM_OK) return s;
        c->n_launch -= 1;  // counted by the surrogate launcher
    } else {
        bool capacity = false;
        cudaError_t e = enqueue_atm(j, &c->smem_set[prec][trav][trunc], &capacity);
        if (capacity)
            return ctx_fail(c, ATM_E_CAPACITY,
                            "a traversal unit of %d molecules does not fit the kernels' shared memory",
                            j.mcap);
        CU(e);
        if (atm_split_active(j)) c->n_launch += j.ncls;  // the class kernel and ncls - 1 more
        if (atm_uses_pair_masks(j)) c->n_launch += 1;      // the pair bitmaps
        if (j.det && (trav == ATM_3C18 || trav == ATM_3C08 || trav == ATM_3C08A) && c->n > 0)
            c->n_launch += 1;  // the fixed-point force conversion
    }
    ctx_prof_end(c, PK_ATM, ev);
    c->n_launch += 1;
    c->n_atm += 1;
    c->forces_valid = true;
    c->f_trav = trav;
    c->f_trunc = trunc;
    c->f_prec = prec;
    c->f_fused = fused;
    return ATM_OK;
}

static atm_status enqueue_reduce(atm_ctx* c)
{
    ReduceArgs r;
    r.b = c->b;
    r.unit_ew = c->unit_ew;
    r.unit_cnt = c->unit_cnt;
    r.unit_ew2 = c->f_fused ? c->unit_ew2 : nullptr;
    r.unit_cnt2 = c->f_fused ? c->unit_cnt2 : nullptr;
    r.mol_ew = c->mol_ew;
    r.mol_cnt = c->mol_cnt;
    r.ke = c->ke;
    r.part = c->d_part;
    r.out = c->d_res;
    cudaEvent_t ev = ctx_prof_begin(c, PK_MD);
    CU(launch_final_reduce(r, c->st));
    ctx_prof_end(c, PK_MD, ev);
    c->n_launch += 2;
    CU(cudaMemcpyAsync(c->h_res, c->d_res, c->R * sizeof(ResultDev), cudaMemcpyDeviceToHost, c->st));
    return ATM_OK;
}

static void copy_result(const ResultDev& r, atm_result* out)
{
    out->e2 = r.e2;
    out->e3 = r.e3;
    out->w2 = r.w2;
    out->w3 = r.w3;
    out->ekin = r.ekin;
    out->n_cand3 = r.n_cand3;
    out->n_int3 = r.n_int3;
    out->n_cand2 = r.n_cand2;
    out->n_int2 = r.n_int2;
}

static bool valid_enums(int trav, int trunc, int prec)
{
    return trav >= 0 && trav <= 4 && trunc >= 0 && trunc <= 1 && prec >= 0 && prec <= 2;
}

extern "C" atm_status atm_compute_forces(atm_ctx* c, atm_traversal trav, atm_truncation trunc,
                                         atm_precision prec, atm_result* out)
{
    if (!c) return ATM_E_INVALID;
    if (!valid_enums(trav, trunc, prec)) return ctx_fail(c, ATM_E_INVALID, "unknown traversal/truncation/precision");
    if (!c->cells_built) return ctx_fail(c, ATM_E_STATE, "cells not built");
    CU(cudaSetDevice(c->device));
    {
        atm_status w = ctx_want_wide(c, trav);
        if (w != ATM_OK) return w;
    }
    atm_status s = ctx_enqueue_forces(c, trav, trunc, prec, c->unit_max[trav]);
    if (s != ATM_OK) return s;
    cudaEvent_t ev = ctx_prof_begin(c, PK_MD);
    CU(launch_kinetic(c->n, c->v, c->ke, c->st));
    ctx_prof_end(c, PK_MD, ev);
    c->n_launch += 1;
    s = enqueue_reduce(c);
    if (s != ATM_OK) return s;
    if (out) {
        s = ctx_sync_and_check(c);
        if (s != ATM_OK) return s;
        copy_result(c->h_res[0], out);
    }
    return ATM_OK;
}

extern "C" atm_status atm_get_results(atm_ctx* c, atm_result* out)
{
    if (!c || !out) return ATM_E_INVALID;
    CU(cudaSetDevice(c->device));
    atm_status s = ctx_sync_and_check(c);
    if (s != ATM_OK) return s;
    for (int r = 0; r < c->R; r++) copy_result(c->h_res[r], out + r);
    return ATM_OK;
}

static atm_status get_forces_impl(atm_ctx* c, double* f, int which, bool host)
{
    if (!c || !f || which < 0 || which > 2) return ATM_E_INVALID;
    if (!c->forces_valid) return ctx_fail(c, ATM_E_STATE, "no force evaluation is current");
    CU(cudaSetDevice(c->device));
    if (c->f_fused && which != 0) {
        // a step kept only LJ + ATM together: evaluate the parts apart for the
        // same state (the cells are those of the current positions)
        atm_status s = ctx_enqueue_forces(c, c->f_trav, c->f_trunc, c->f_prec,
                                          c->unit_max[c->f_trav], false);
        if (s != ATM_OK) return s;
    }
    size_t bytes = 3 * (size_t)c->n * sizeof(double);
    if (!bytes) return ATM_OK;
    CU(launch_gather_forces(c->n, c->perm, c->f_lj, c->f_atm, which, host ? c->f_out : f, c->st));
    c->n_launch += 1;
    if (host) {
        CU(cudaMemcpyAsync(f, c->f_out, bytes, cudaMemcpyDeviceToHost, c->st));
        return ctx_sync_and_check(c);
    }
    return ATM_OK;
}

extern "C" atm_status atm_get_forces(atm_ctx* c, double* f, int which)
{
    return get_forces_impl(c, f, which, true);
}

extern "C" atm_status atm_get_forces_dev(atm_ctx* c, double* f_dev, int which)
{
    return get_forces_impl(c, f_dev, which, false);
}

extern "C" atm_status atm_get_state(atm_ctx* c, double* x, double* v)
{
    if (!c) return ATM_E_INVALID;
    if (!c->have_x) return ctx_fail(c, ATM_E_STATE, "no state set");
    CU(cudaSetDevice(c->device));
    size_t bytes = 3 * (size_t)c->n * sizeof(double);
    if (bytes && x) CU(cudaMemcpyAsync(x, c->x, bytes, cudaMemcpyDeviceToHost, c->st));
    if (bytes && v) CU(cudaMemcpyAsync(v, c->v, bytes, cudaMemcpyDeviceToHost, c->st));
    CU(cudaStreamSynchronize(c->st));
    return ATM_OK;
}

// atm_step_host: once the last step's cell build has wrapped the positions
// (enqueue_cells has just synchronised with it, and nothing later in the step
// writes them) they are copied to the caller beside the force evaluation
static atm_status early_x_out(atm_ctx* c)
{
    if (!c->x_host_out || c->n == 0) return ATM_OK;
    CU(cudaMemcpyAsync(c->x_host_out, c->x, 3 * (size_t)c->n * sizeof(double),
                       cudaMemcpyDeviceToHost, c->io_st));
    c->x_host_out = nullptr;
    c->x_out_issued = true;
    return ATM_OK;
}

// one velocity-Verlet step without host synchronisation: kick + drift, cells,
// forces (capacity mcap), kick
static atm_status enqueue_step(atm_ctx* c, int trav, int trunc, int prec, int mcap)
{
    cudaEvent_t ev = ctx_prof_begin(c, PK_MD);
    CU(launch_kick(c->b, c->perm, c->f_lj, c->f_atm, c->x, c->v, 1, c->ke, c->st));
    ctx_prof_end(c, PK_MD, ev);
    c->n_launch += 1;
    atm_status s = launch_cells(c);
    if (s != ATM_OK) return s;
    s = ctx_enqueue_forces(c, trav, trunc, prec, mcap, true);
    if (s != ATM_OK) return s;
    ev = ctx_prof_begin(c, PK_MD);
    CU(launch_kick(c->b, c->perm, c->f_lj, c->f_atm, c->x, c->v, 0, c->ke, c->st));
    ctx_prof_end(c, PK_MD, ev);
    c->n_launch += 1;
    return ATM_OK;
}

// resident CTAs per SM of the ATM launch sized for mcap staged molecules
static int atm_ctas_per_sm(const atm_ctx* c, int trav, int trunc, int prec, int nwarps, int mcap)
{
    AtmPlan P;
    const int g = edge_capacity(c, trav, trunc);
    if (!atm_choose_plan(trav, trunc, prec, mcap, c->smem_optin, P, c->det, g)) return 0;
    if ((nwarps == 2 || nwarps == 4 || nwarps == 8) && trav != ATM_3C01 && trav != ATM_3CW) {
        AtmPlan Q;
        if (atm_choose_plan_nw(trav, trunc, prec, mcap, c->smem_optin, nwarps, Q, c->det, g)) P = Q;
    }
    return prec == ATM_FP64 ? atm_occupancy_fp64(trav, trunc, P.nwarps, P.smem, c->det)
                            : atm_occupancy_fp32(trav, trunc, P.nwarps, P.smem, c->det);
}

// staged-molecule capacity of a graph: the current largest unit plus headroom
// for molecules moving between cells during the steps the graph replays.  The
// headroom is at most a quarter of the unit (at least 8), and the largest
// capacity in that range that keeps the resident CTAs per SM of the current
// unit size is taken (a bigger unit costs shared memory per CTA); with none,
// 4 molecules.  A unit that outgrows the capacity during the replayed steps
// is detected on the device and the run restarts without the graph.
static int graph_mcap(const atm_ctx* c, int trav, int trunc, int prec, int nwarps)
{
    const int m = c->unit_max[trav];
    const int limit = (trav == ATM_3C01 || trav == ATM_3CW) ? 65535 : ATM_MCAP_LIMIT;
    const int hi = std::min(limit, m + std::max(8, m / 4));
    if (prec == ATM_SURROGATE || m < 1) return hi;
    const int occ = atm_ctas_per_sm(c, trav, trunc, prec, nwarps, m);
    for (int cap = hi; cap > m + 4; cap--)
        if (atm_ctas_per_sm(c, trav, trunc, prec, nwarps, cap) >= occ) return cap;
    return std::min(limit, m + 4);
}

// run nsteps with a CUDA graph of one step (no host synchronisation between
// steps); a capacity overflow surfaces in the status word
static atm_status run_graph_steps(atm_ctx* c, int nsteps, int trav, int trunc, int prec)
{
    int persistent = 0, nwarps = 0, cls[3] = {1, 0, 0};
    if (prec != ATM_SURROGATE)
        launch_choice(c, trav, trunc, prec, c->unit_max[trav], persistent, nwarps, cls);
    const int mcap = graph_mcap(c, trav, trunc, prec, nwarps);
    const int key[9] = {trav, trunc, prec, mcap,
                        persistent + 2 * nwarps + 64 * (use_pair_masks(c, trav, trunc, prec) ? 1 : 0),
                        cls[0], cls[1], cls[2], edge_capacity(c, trav, trunc)};
    if (!c->graph || memcmp(key, c->graph_key, sizeof(key)) != 0) {
        drop_graph(c);
        cudaStream_t keep = c->st;
        const int keep_prof = c->prof;
        const long long nl = c->n_launch, na = c->n_atm;
        c->prof = 0;
        c->st = c->cap_st;
        cudaGraph_t g = nullptr;
        CU(cudaStreamBeginCapture(c->cap_st, cudaStreamCaptureModeThreadLocal));
        atm_status s = enqueue_step(c, trav, trunc, prec, mcap);
        cudaError_t e = cudaStreamEndCapture(c->cap_st, &g);
        c->st = keep;
        c->prof = keep_prof;
        c->n_launch = nl;
        c->n_atm = na;
        if (s != ATM_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        CU(e);
        e = cudaGraphInstantiate(&c->graph, g, 0);
        cudaGraphDestroy(g);
        CU(e);
        memcpy(c->graph_key, key, sizeof(key));
    }
    cudaEvent_t ev = ctx_prof_begin(c, PK_MD);
    for (int k = 0; k < nsteps; k++) CU(cudaGraphLaunch(c->graph, c->st));
    ctx_prof_end(c, PK_MD, ev);
    c->n_launch += (long long)nsteps * kernels_per_step(trav, trunc, prec, cls[0]);
    c->n_atm += nsteps;
    return ATM_OK;
}

extern "C" atm_status atm_step(atm_ctx* c, int nsteps, atm_traversal trav, atm_truncation trunc,
                               atm_precision prec, atm_result* last)
{
    if (!c) return ATM_E_INVALID;
    if (nsteps < 0 || !valid_enums(trav, trunc, prec))
        return ctx_fail(c, ATM_E_INVALID, "bad step arguments");
    if (!c->have_x) return ctx_fail(c, ATM_E_STATE, "no state set");
    CU(cudaSetDevice(c->device));
    atm_status s = ctx_want_wide(c, trav);
    if (s != ATM_OK) return s;
    // forces of the current state from this combination (for the surrogate, the
    // exact FP32C forces of an interleaved step serve as well)
    bool fresh = c->forces_valid && c->f_trav == trav && c->f_trunc == trunc &&
                 (c->f_prec == prec || (prec == ATM_SURROGATE && c->f_prec == ATM_FP32C));
    if (!fresh && nsteps > 0 && c->f_in_valid && c->f_in_key[0] == trav &&
        c->f_in_key[1] == trunc && c->f_in_key[2] == prec) {
        // the caller gave the forces of this state: the first step's half kick
        // and drift use them, then the step continues as usual
        CU(launch_kick_orig(c->b, c->f_in, c->x, c->v, c->ke, c->st));
        c->n_launch += 1;
        c->f_in_valid = false;
        s = enqueue_cells(c);
        if (s != ATM_OK) return s;
        if (nsteps == 1) {
            s = early_x_out(c);
            if (s != ATM_OK) return s;
        }
        s = ctx_enqueue_forces(c, trav, trunc, prec, c->unit_max[trav], true);
        if (s != ATM_OK) return s;
        CU(launch_kick(c->b, c->perm, c->f_lj, c->f_atm, c->x, c->v, 0, c->ke, c->st));
        c->n_launch += 1;
        nsteps -= 1;
        fresh = true;
    }
    if (!fresh) {
        s = enqueue_cells(c);
        if (s != ATM_OK) return s;
        s = ctx_enqueue_forces(c, trav, trunc, prec, c->unit_max[trav], true);
        if (s != ATM_OK) return s;
    }
    bool done = false;
    // surrogate runs that interleave exact steps take the per-step path
    const bool sur_mixed = prec == ATM_SURROGATE && sur_exact_every(c) > 0;
    if (c->opt_graph && nsteps > 0 && !sur_mixed) {
        const size_t bytes = 3 * (size_t)c->n * sizeof(double);
        if (bytes) {
            CU(cudaMemcpyAsync(c->x0, c->x, bytes, cudaMemcpyDeviceToDevice, c->st));
            CU(cudaMemcpyAsync(c->v0, c->v, bytes, cudaMemcpyDeviceToDevice, c->st));
        }
        s = run_graph_steps(c, nsteps, trav, trunc, prec);
        if (s != ATM_OK) return s;
        CU(cudaMemcpyAsync(c->h_maxocc, c->d_maxocc, (1 + 2 * ATM_NTRAV) * sizeof(int),
                           cudaMemcpyDeviceToHost, c->st));
        s = ctx_sync_and_check(c);
        if (s == ATM_OK) {
            done = true;
            take_unit_sizes(c);
        } else if (s == ATM_E_CAPACITY) {
            // a unit outgrew the graph's capacity: restart from the snapshot
            // and step with per-step sizing
            if (bytes) {
                CU(cudaMemcpyAsync(c->x, c->x0, bytes, cudaMemcpyDeviceToDevice, c->st));
                CU(cudaMemcpyAsync(c->v, c->v0, bytes, cudaMemcpyDeviceToDevice, c->st));
            }
            drop_graph(c);
            s = enqueue_cells(c);
            if (s != ATM_OK) return s;
            s = ctx_enqueue_forces(c, trav, trunc, prec, c->unit_max[trav], true);
            if (s != ATM_OK) return s;
        } else {
            return s;
        }
    }
    if (!done) {
        for (int k = 0; k < nsteps; k++) {
            cudaEvent_t ev = ctx_prof_begin(c, PK_MD);
            CU(launch_kick(c->b, c->perm, c->f_lj, c->f_atm, c->x, c->v, 1, c->ke, c->st));
            ctx_prof_end(c, PK_MD, ev);
            c->n_launch += 1;
            s = enqueue_cells(c);
            if (s != ATM_OK) return s;
            if (k == nsteps - 1) {
                s = early_x_out(c);
                if (s != ATM_OK) return s;
            }
            // every exact_every-th surrogate step uses the exact FP32C traversal
            // and compares the surrogate with it
            const bool exact = sur_mixed && sur_exact_due(c);
            s = ctx_enqueue_forces(c, trav, trunc, exact ? (int)ATM_FP32C : (int)prec,
                                   c->unit_max[trav], !exact);
            if (s != ATM_OK) return s;
            if (exact) {
                s = sur_enqueue_monitor(c);
                if (s != ATM_OK) return s;
            }
            if (prec == ATM_SURROGATE) sur_count_step(c);
            ev = ctx_prof_begin(c, PK_MD);
            CU(launch_kick(c->b, c->perm, c->f_lj, c->f_atm, c->x, c->v, 0, c->ke, c->st));
            ctx_prof_end(c, PK_MD, ev);
            c->n_launch += 1;
        }
    }
    if (nsteps == 0) {
        CU(launch_kinetic(c->n, c->v, c->ke, c->st));
        c->n_launch += 1;
    }
    s = enqueue_reduce(c);
    if (s != ATM_OK) return s;
    if (last) {
        s = ctx_sync_and_check(c);
        if (s != ATM_OK) return s;
        copy_result(c->h_res[0], last);
    }
    return ATM_OK;
}

extern "C" atm_status atm_step_host(atm_ctx* c, int nsteps, atm_traversal trav,
                                    atm_truncation trunc, atm_precision prec, double* x,
                                    double* v, double* f, atm_result* last)
{
    if (!c) return ATM_E_INVALID;
    if (nsteps < 0 || !valid_enums(trav, trunc, prec))
        return ctx_fail(c, ATM_E_INVALID, "bad step arguments");
    if ((!x || !v) && c->n > 0) return ctx_fail(c, ATM_E_INVALID, "positions and velocities are required");
    if (f && prec == ATM_SURROGATE)
        return ctx_fail(c, ATM_E_INVALID, "given forces need an exact traversal, truncation, precision");
    CU(cudaSetDevice(c->device));
    const long long m = 3 * c->n;
    const size_t bytes = (size_t)m * sizeof(double);
    // inputs: copies and device-side finite checks; the checks' result travels back
    // with the first synchronisation of the step (its cell build) or the last
    // (each check runs on io_st while the next copy runs on the stream)
    *c->h_chk = 0;
    if (m > 0) {
        auto check_on_io = [&](const double* a) -> cudaError_t {
            cudaError_t e = cudaEventRecord(c->ev_io, c->st);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(c->io_st, c->ev_io, 0);
            if (e == cudaSuccess) e = launch_check_finite(m, a, c->d_chk, c->io_st);
            return e;
        };
        CU(cudaMemsetAsync(c->d_chk, 0, sizeof(int), c->st));
        CU(cudaMemcpyAsync(c->x, x, bytes, cudaMemcpyHostToDevice, c->st));
        CU(check_on_io(c->x));
        CU(cudaMemcpyAsync(c->v, v, bytes, cudaMemcpyHostToDevice, c->st));
        CU(check_on_io(c->v));
        c->n_launch += 2;
        if (f) {
            CU(cudaMemcpyAsync(c->f_in, f, bytes, cudaMemcpyHostToDevice, c->st));
            CU(check_on_io(c->f_in));
            c->n_launch += 1;
        }
        CU(cudaEventRecord(c->ev_io_done, c->io_st));
        CU(cudaStreamWaitEvent(c->st, c->ev_io_done, 0));
        CU(cudaMemcpyAsync(c->h_chk, c->d_chk, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    }
    c->have_x = true;
    invalidate(c);
    if (f) {
        c->f_in_valid = true;
        c->f_in_key[0] = trav;
        c->f_in_key[1] = trunc;
        c->f_in_key[2] = prec;
    }
    auto bad_input = [&]() -> atm_status {
        c->have_x = false;
        invalidate(c);
        return ctx_fail(c, ATM_E_NONFINITE, "non-finite position, velocity or force given");
    };
    // the last step copies its positions to x as soon as its cells are built
    c->x_host_out = m > 0 ? x : nullptr;
    c->x_out_issued = false;
    atm_status s = atm_step(c, nsteps, trav, trunc, prec, nullptr);
    const bool x_early = c->x_out_issued;
    c->x_host_out = nullptr;
    c->x_out_issued = false;
    if (s != ATM_OK) {
        cudaStreamSynchronize(c->st);
        cudaStreamSynchronize(c->io_st);
        return *c->h_chk ? bad_input() : s;
    }
    // outputs: state, total force and scalars, then one synchronisation
    if (m > 0) {
        if (x_early) {
            CU(cudaEventRecord(c->ev_io_done, c->io_st));
            CU(cudaStreamWaitEvent(c->st, c->ev_io_done, 0));
        } else {
            CU(cudaMemcpyAsync(x, c->x, bytes, cudaMemcpyDeviceToHost, c->st));
        }
        CU(cudaMemcpyAsync(v, c->v, bytes, cudaMemcpyDeviceToHost, c->st));
        if (f) {
            CU(launch_gather_forces(c->n, c->perm, c->f_lj, c->f_atm, 0, c->f_out, c->st));
            c->n_launch += 1;
            CU(cudaMemcpyAsync(f, c->f_out, bytes, cudaMemcpyDeviceToHost, c->st));
        }
    }
    s = ctx_sync_and_check(c);
    if (*c->h_chk) return bad_input();
    if (s != ATM_OK) return s;
    if (last) copy_result(c->h_res[0], last);
    return ATM_OK;
}

extern "C" atm_status atm_set_pair_masks(atm_ctx* c, int on)
{
    if (!c) return ATM_E_INVALID;
    if (on < 0 || on > 1) return ctx_fail(c, ATM_E_INVALID, "on is 0 or 1");
    c->opt_pmask = on;
    memset(c->tuned, 0, sizeof(c->tuned));
    memset(c->nw_auto, 0, sizeof(c->nw_auto));
    drop_graph(c);
    return ATM_OK;
}

extern "C" atm_status atm_set_options(atm_ctx* c, int persistent, int nwarps, int graph)
{
    if (!c) return ATM_E_INVALID;
    if (persistent < 0 || persistent > 1 || !(nwarps == 0 || nwarps == 4 || nwarps == 8) ||
        graph < 0 || graph > 1)
        return ctx_fail(c, ATM_E_INVALID, "bad options");
    c->opt_persistent = persistent;
    c->opt_nwarps = nwarps;
    c->opt_graph = graph;
    memset(c->tuned, 0, sizeof(c->tuned));
    memset(c->nw_auto, 0, sizeof(c->nw_auto));
    drop_graph(c);
    return ATM_OK;
}

extern "C" atm_status atm_set_owned_layers(atm_ctx* c, int replica, int z_lo, int z_hi)
{
    if (!c) return ATM_E_INVALID;
    if (replica < 0 || replica >= c->R) return ctx_fail(c, ATM_E_INVALID, "no replica %d", replica);
    Rep& r = c->reps[replica];
    if (z_lo < 0 || z_hi > r.g.nc[2] || z_lo >= z_hi)
        return ctx_fail(c, ATM_E_INVALID, "owned layers must satisfy 0 <= z_lo < z_hi <= %d",
                        r.g.nc[2]);
    CU(cudaSetDevice(c->device));
    r.own_z0 = z_lo;
    r.own_z1 = z_hi;
    CU(cudaMemcpyAsync(c->d_rep + replica, &r, sizeof(Rep), cudaMemcpyHostToDevice, c->st));
    CU(cudaStreamSynchronize(c->st));
    drop_graph(c);
    c->forces_valid = false;
    return ATM_OK;
}

extern "C" atm_status atm_set_deterministic(atm_ctx* c, int on)
{
    if (!c) return ATM_E_INVALID;
    if (on < 0 || on > 1) return ctx_fail(c, ATM_E_INVALID, "on must be 0 or 1");
    c->det = on;
    memset(c->tuned, 0, sizeof(c->tuned));
    memset(c->nw_auto, 0, sizeof(c->nw_auto));
    drop_graph(c);
    c->forces_valid = false;
    return ATM_OK;
}

extern "C" atm_status atm_set_unit_classes(atm_ctx* c, int nclass, const int* cuts)
{
    if (!c) return ATM_E_INVALID;
    if (nclass < 1 || nclass > 3 || (nclass > 1 && !cuts))
        return ctx_fail(c, ATM_E_INVALID, "1 to 3 classes, with nclass - 1 bounds");
    for (int k = 0; k + 1 < nclass; k++)
        if (cuts[k] < 1 || cuts[k] > ATM_MCAP_LIMIT || (k > 0 && cuts[k] <= cuts[k - 1]))
            return ctx_fail(c, ATM_E_INVALID, "bounds must rise within 1..%d", ATM_MCAP_LIMIT);
    c->opt_cls[0] = nclass;
    c->opt_cls[1] = nclass > 1 ? cuts[0] : 0;
    c->opt_cls[2] = nclass > 2 ? cuts[1] : 0;
    memset(c->tuned, 0, sizeof(c->tuned));
    memset(c->nw_auto, 0, sizeof(c->nw_auto));
    drop_graph(c);
    return ATM_OK;
}

extern "C" atm_status atm_autotune(atm_ctx* c, atm_traversal trav, atm_truncation trunc,
                                   atm_precision prec, int reps, atm_tuning* out)
{
    if (!c) return ATM_E_INVALID;
    if (!valid_enums(trav, trunc, prec) || prec == ATM_SURROGATE || reps < 1)
        return ctx_fail(c, ATM_E_INVALID, "bad tuning arguments");
    if (!c->cells_built) return ctx_fail(c, ATM_E_STATE, "cells not built");
    CU(cudaSetDevice(c->device));
    {
        atm_status w = ctx_want_wide(c, trav);
        if (w != ATM_OK) return w;
    }
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    const int keep_prof = c->prof;
    c->prof = 0;
    float best = 1e30f;
    int best_code = 1;
    atm_status s = ATM_OK;
    const bool owner = trav == ATM_3C01 || trav == ATM_3CW;
    const int nw_options = owner ? 1 : 2, split_options = owner ? 1 : N_SPLITS;
    // the evaluation as steps take it (LJ inside the units where steps fuse it)
    const bool fuse = lj_fused(trav, trunc, prec);
    for (int sp = 0; sp < split_options && s == ATM_OK; sp++)
    for (int nwi = 0; nwi < nw_options && s == ATM_OK; nwi++)
        for (int pers = 0; pers < 2 && s == ATM_OK; pers++) {
            const int code = 1 + pers + 2 * nwi + 4 * sp;
            c->tuned[prec][trav][trunc] = code;
            s = ctx_enqueue_forces(c, trav, trunc, prec, c->unit_max[trav], fuse);  // warm-up
            if (s != ATM_OK) break;
            cudaEventRecord(e0, c->st);
            for (int k = 0; k < reps && s == ATM_OK; k++)
                s = ctx_enqueue_forces(c, trav, trunc, prec, c->unit_max[trav], fuse);
            cudaEventRecord(e1, c->st);
            if (s != ATM_OK) break;
            s = ctx_sync_and_check(c);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (s == ATM_OK && ms < best) {
                best = ms;
                best_code = code;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->prof = keep_prof;
    c->tuned[prec][trav][trunc] = best_code;
    drop_graph(c);
    if (s != ATM_OK) return s;
    if (out) {
        const int sp = (best_code - 1) >> 2;
        out->persistent = (best_code - 1) & 1;
        out->nwarps = trav == ATM_3C01 ? 4 : (((best_code - 1) & 2) ? 8 : 4);
        out->ms_per_eval = best / reps;
        out->nclass = SPLITS[sp][0];
        out->cut[0] = SPLITS[sp][1];
        out->cut[1] = SPLITS[sp][2];
    }
    return ATM_OK;
}

extern "C" atm_status atm_density_accumulate(atm_ctx* c, int axis, int nbins)
{
    if (!c) return ATM_E_INVALID;
    if (axis < 0 || axis > 2 || nbins < 1 || nbins > DENS_MAX_BINS)
        return ctx_fail(c, ATM_E_INVALID, "axis in 0..2, 1 <= nbins <= %d", DENS_MAX_BINS);
    if (!c->cells_built) return ctx_fail(c, ATM_E_STATE, "cells not built (positions not wrapped)");
    if (c->dens_samples > 0 && (axis != c->dens_axis || nbins != c->dens_nbins))
        return ctx_fail(c, ATM_E_STATE, "density accumulator holds another axis/bin count; reset it");
    CU(cudaSetDevice(c->device));
    CU(launch_density(c->b, c->x, axis, nbins, c->d_dens, c->st));
    c->n_launch += 1;
    c->dens_axis = axis;
    c->dens_nbins = nbins;
    c->dens_samples++;
    return ATM_OK;
}

extern "C" atm_status atm_density_get(atm_ctx* c, uint64_t* counts, int64_t* samples)
{
    if (!c) return ATM_E_INVALID;
    CU(cudaSetDevice(c->device));
    if (counts && c->dens_nbins > 0)
        CU(cudaMemcpyAsync(counts, c->d_dens, (size_t)c->R * c->dens_nbins * sizeof(uint64_t),
                           cudaMemcpyDeviceToHost, c->st));
    CU(cudaStreamSynchronize(c->st));
    if (samples) *samples = c->dens_samples;
    return ATM_OK;
}

extern "C" atm_status atm_density_reset(atm_ctx* c)
{
    if (!c) return ATM_E_INVALID;
    CU(cudaSetDevice(c->device));
    CU(cudaMemsetAsync(c->d_dens, 0, (size_t)c->R * DENS_MAX_BINS * sizeof(uint64_t), c->st));
    c->dens_samples = 0;
    c->dens_axis = -1;
    c->dens_nbins = 0;
    return ATM_OK;
}

extern "C" atm_status atm_set_forces(atm_ctx* c, const double* f, atm_traversal trav,
                                     atm_truncation trunc, atm_precision prec)
{
    if (!c) return ATM_E_INVALID;
    if (!valid_enums(trav, trunc, prec) || prec == ATM_SURROGATE)
        return ctx_fail(c, ATM_E_INVALID, "set_forces needs an exact traversal, truncation, precision");
    if (!f && c->n > 0) return ctx_fail(c, ATM_E_INVALID, "forces are required");
    if (!c->have_x) return ctx_fail(c, ATM_E_STATE, "set the state before its forces");
    CU(cudaSetDevice(c->device));
    bool bad = false;
    atm_status s = copy_in_checked(c, c->f_in, f, nullptr, nullptr, 3 * c->n, &bad);
    if (s != ATM_OK) return s;
    if (bad) {
        c->f_in_valid = false;
        return ctx_fail(c, ATM_E_NONFINITE, "non-finite force");
    }
    c->f_in_valid = true;
    c->f_in_key[0] = trav;
    c->f_in_key[1] = trunc;
    c->f_in_key[2] = prec;
    return ATM_OK;
}

extern "C" atm_status atm_thermostat(atm_ctx* c, const double* t_target)
{
    if (!c || !t_target) return ATM_E_INVALID;
    for (int r = 0; r < c->R; r++)
        if (!(t_target[r] >= 0.0) || !std::isfinite(t_target[r]))
            return ctx_fail(c, ATM_E_INVALID, "target temperature of replica %d", r);
    if (!c->have_x) return ctx_fail(c, ATM_E_STATE, "no state set");
    CU(cudaSetDevice(c->device));
    CU(cudaMemcpyAsync(c->d_ttarget, t_target, c->R * sizeof(double), cudaMemcpyHostToDevice, c->st));
    CU(launch_kinetic(c->n, c->v, c->ke, c->st));
    c->n_launch += 1;
    atm_status s = enqueue_reduce(c);
    if (s != ATM_OK) return s;
    CU(launch_rescale(c->b, c->v, c->ke, c->d_res, c->d_ttarget, c->st));
    c->n_launch += 1;
    s = enqueue_reduce(c);
    if (s != ATM_OK) return s;
    return ctx_sync_and_check(c);
}

extern "C" atm_status atm_rdf_accumulate(atm_ctx* c, double r_max, int nbins)
{
    if (!c) return ATM_E_INVALID;
    if (nbins < 1 || nbins > DENS_MAX_BINS || !(r_max > 0.0) || !std::isfinite(r_max))
        return ctx_fail(c, ATM_E_INVALID, "r_max > 0, 1 <= nbins <= %d", DENS_MAX_BINS);
    for (const Rep& r : c->reps)
        for (int d = 0; d < 3; d++)
            if (r_max > r.g.w[d])
                return ctx_fail(c, ATM_E_INVALID, "r_max above a cell edge (%g)", r.g.w[d]);
    if (!c->cells_built) return ctx_fail(c, ATM_E_STATE, "cells not built");
    if (c->rdf_samples > 0 && (r_max != c->rdf_rmax || nbins != c->rdf_nbins))
        return ctx_fail(c, ATM_E_STATE, "the RDF accumulator holds another range/bin count; reset it");
    CU(cudaSetDevice(c->device));
    CU(launch_rdf(c->b, c->xl, c->start, c->cell_sorted, r_max, nbins, c->d_rdf, c->st));
    c->n_launch += 1;
    c->rdf_rmax = r_max;
    c->rdf_nbins = nbins;
    c->rdf_samples++;
    return ATM_OK;
}

extern "C" atm_status atm_rdf_get(atm_ctx* c, uint64_t* counts, int64_t* samples)
{
    if (!c) return ATM_E_INVALID;
    CU(cudaSetDevice(c->device));
    if (counts && c->rdf_nbins > 0)
        CU(cudaMemcpyAsync(counts, c->d_rdf, (size_t)c->R * c->rdf_nbins * sizeof(uint64_t),
                           cudaMemcpyDeviceToHost, c->st));
    CU(cudaStreamSynchronize(c->st));
    if (samples) *samples = c->rdf_samples;
    return ATM_OK;
}

extern "C" atm_status atm_rdf_reset(atm_ctx* c)
{
    if (!c) return ATM_E_INVALID;
    CU(cudaSetDevice(c->device));
    CU(cudaMemsetAsync(c->d_rdf, 0, (size_t)c->R * DENS_MAX_BINS * sizeof(uint64_t), c->st));
    c->rdf_samples = 0;
    c->rdf_rmax = 0.0;
    c->rdf_nbins = 0;
    return ATM_OK;
}

extern "C" atm_status atm_lj_tail(const atm_params* p, int64_t n, double* e_tail, double* p_tail)
{
    if (!p || n < 0 || !(p->rc > 0.0) || !(p->lj_sigma > 0.0)) return ATM_E_INVALID;
    const double V = p->box[0] * p->box[1] * p->box[2];
    if (!(V > 0.0)) return ATM_E_INVALID;
    const double rho = (double)n / V, pi = 3.14159265358979323846;
    const double sr3 = std::pow(p->lj_sigma / p->rc, 3.0), sr9 = sr3 * sr3 * sr3;
    const double s3 = p->lj_sigma * p->lj_sigma * p->lj_sigma;
    if (e_tail) *e_tail = 8.0 / 3.0 * pi * (double)n * rho * p->lj_eps * s3 * (sr9 / 3.0 - sr3);
    if (p_tail) *p_tail = 16.0 / 3.0 * pi * rho * rho * p->lj_eps * s3 * (2.0 / 3.0 * sr9 - sr3);
    return ATM_OK;
}

extern "C" atm_status atm_set_profiling(atm_ctx* c, int on)
{
    if (!c) return ATM_E_INVALID;
    CU(cudaSetDevice(c->device));
    CU(cudaStreamSynchronize(c->st));
    prof_drain(c);
    c->prof = on == 2 ? 2 : (on != 0 ? 1 : 0);
    for (double& v : c->prof_ms) v = 0.0;
    c->n_launch = 0;
    c->n_atm = 0;
    return ATM_OK;
}

extern "C" atm_status atm_get_profile(atm_ctx* c, atm_profile* out)
{
    if (!c || !out) return ATM_E_INVALID;
    CU(cudaSetDevice(c->device));
    CU(cudaStreamSynchronize(c->st));
    prof_drain(c);
    out->ms_cells = c->prof_ms[PK_CELLS];
    out->ms_lj = c->prof_ms[PK_LJ];
    out->ms_atm = c->prof_ms[PK_ATM];
    out->ms_md = c->prof_ms[PK_MD];
    out->n_launches = c->n_launch;
    out->n_atm_launches = c->n_atm;
    return ATM_OK;
}
