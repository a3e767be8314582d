// capi.cu -- the C ABI declared in include/atm3.h: context, buffers, call order.
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

using namespace atm3;

namespace {
}  // namespace

struct atm_ctx {
    atm_params p;
    long long n = 0;
    cudaStream_t st = nullptr;
    Grid g;
    double* x = nullptr;   // [3n] positions, original order (wrapped by build_cells)
    double* v = nullptr;   // [3n] velocities, original order
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
    double* lj_ew = nullptr;
    unsigned long long* lj_cnt = nullptr;
    long long n_lj_blocks = 0;
    double* ke_part = nullptr;
    long long n_ke_blocks = 0;
    ResultDev* d_res = nullptr;
    ResultDev* h_res = nullptr;
    int* d_status = nullptr;
    int* h_status = nullptr;
    int* d_maxocc = nullptr;
    int* h_maxocc = nullptr;
    int maxocc = 0;
    int unit_max[3] = {0, 0, 0};  // largest unit (staged molecules) of 3c01, 3c18, 3c08
    bool have_x = false, cells_built = false, forces_valid = false;
    int f_trav = -1, f_trunc = -1, f_prec = -1;
    size_t smem_set[2][3][2] = {};
    int smem_optin = 0;
    // profiling: event pairs around launch groups, summed per kind
    bool prof = false;
    struct EvRec {
        cudaEvent_t a, b;
        int kind;
    };
    std::vector<EvRec> ev_live;
    std::vector<cudaEvent_t> ev_pool;
    double prof_ms[4] = {0, 0, 0, 0};  // cells, lj, atm, md
    long long n_launch = 0, n_atm = 0;
    char err[256] = "no error";
};

enum { PK_CELLS = 0, PK_LJ = 1, PK_ATM = 2, PK_MD = 3 };

static cudaEvent_t prof_begin(atm_ctx* c)
{
    if (!c->prof) return nullptr;
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

static void prof_end(atm_ctx* c, int kind, cudaEvent_t a)
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

static atm_status fail(atm_ctx* c, atm_status s, const char* fmt, ...)
{
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return s;
}

#define CU(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(c, ATM_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_));        \
    } while (0)

static void free_all(atm_ctx* c)
{
    void* dev[] = {c->x, c->v, c->xl, c->xl32, c->cell_of, c->rank, c->count, c->start, c->perm,
                   c->cell_sorted, c->f_lj, c->f_atm, c->f_out, c->unit_ew, c->unit_cnt,
                   c->lj_ew, c->lj_cnt, c->ke_part, c->d_res, c->d_status, c->d_maxocc};
    for (void* p : dev)
        if (p) cudaFree(p);
    if (c->h_res) cudaFreeHost(c->h_res);
    if (c->h_status) cudaFreeHost(c->h_status);
    if (c->h_maxocc) cudaFreeHost(c->h_maxocc);
    for (auto& r : c->ev_live) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    c->ev_live.clear();
    c->ev_pool.clear();
}

// n_d = largest k with L/k >= r_c (decided on the rounded quotient), w = L / n_d
static atm_status make_grid(atm_ctx* c, const atm_params* p, Grid& g)
{
    long long ncell = 1;
    for (int d = 0; d < 3; d++) {
        double L = p->box[d], rc = p->rc;
        if (!(L > 0.0) || !(rc > 0.0) || !std::isfinite(L) || !std::isfinite(rc))
            return fail(c, ATM_E_INVALID, "box and rc must be positive and finite");
        double k = std::floor(L / rc);
        if (k < 1.0) k = 1.0;
        while (L / (k + 1.0) >= rc) k += 1.0;
        while (k > 0.0 && L / k < rc) k -= 1.0;
        if (k < 3.0)
            return fail(c, ATM_E_BOX_TOO_SMALL, "box edge %d (%.6g) holds fewer than 3 cells of rc %.6g",
                        d, L, rc);
        if (k > 1.0e6) return fail(c, ATM_E_INVALID, "too many cells along axis %d", d);
        g.nc[d] = (int)k;
        g.L[d] = L;
        g.w[d] = L / k;
        ncell *= (long long)k;
    }
    if (ncell > (1ll << 30)) return fail(c, ATM_E_INVALID, "too many cells (%lld)", ncell);
    g.ncell = ncell;
    return ATM_OK;
}

static atm_status check_status(atm_ctx* c)
{
    int s = *c->h_status;
    if (s == 0) return ATM_OK;
    *c->h_status = 0;
    cudaMemsetAsync(c->d_status, 0, sizeof(int), c->st);
    if (s & ST_NONFINITE) return fail(c, ATM_E_NONFINITE, "non-finite position or velocity");
    if (s & ST_CAPACITY)
        return fail(c, ATM_E_CAPACITY, "a traversal unit holds more molecules than staged");
    return fail(c, ATM_E_CUDA, "device status %d", s);
}

static atm_status sync_and_check(atm_ctx* c)
{
    CU(cudaMemcpyAsync(c->h_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    CU(cudaStreamSynchronize(c->st));
    prof_drain(c);
    return check_status(c);
}

extern "C" int atm_abi_version(void) { return ATM3_ABI_VERSION; }

extern "C" const char* atm_last_error(const atm_ctx* c)
{
    return c ? c->err : "null context";
}

extern "C" atm_status atm_create(const atm_params* params, int64_t n, atm_ctx** out)
{
    if (!out) return ATM_E_INVALID;
    *out = nullptr;
    if (!params || n < 0 || n > (int64_t)0x7fffffff - 1) return ATM_E_INVALID;
    atm_ctx* c = new (std::nothrow) atm_ctx();
    if (!c) return ATM_E_INVALID;
    c->p = *params;
    c->n = n;
    c->st = (cudaStream_t)params->cuda_stream;
    if (!std::isfinite(params->nu) || !std::isfinite(params->lj_eps) ||
        !(params->lj_sigma > 0.0) || !std::isfinite(params->dt)) {
        delete c;
        return ATM_E_INVALID;
    }
    atm_status s = make_grid(c, params, c->g);
    if (s != ATM_OK) {
        delete c;
        return s;
    }
    auto alloc = [&](void** ptr, size_t bytes) -> bool {
        return cudaMalloc(ptr, bytes > 0 ? bytes : 16) == cudaSuccess;
    };
    bool ok = cudaSetDevice(params->device) == cudaSuccess;
    size_t N = (size_t)(n > 0 ? n : 1), NC = (size_t)c->g.ncell;
    c->n_lj_blocks = (long long)((N + LJ_BLOCK - 1) / LJ_BLOCK);
    c->n_ke_blocks = (long long)((N + MD_BLOCK - 1) / MD_BLOCK);
    ok = ok && alloc((void**)&c->x, 3 * N * sizeof(double));
    ok = ok && alloc((void**)&c->v, 3 * N * sizeof(double));
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
    ok = ok && alloc((void**)&c->unit_ew, 2 * NC * sizeof(double));
    ok = ok && alloc((void**)&c->unit_cnt, 2 * NC * sizeof(unsigned long long));
    ok = ok && alloc((void**)&c->lj_ew, 2 * (size_t)c->n_lj_blocks * sizeof(double));
    ok = ok && alloc((void**)&c->lj_cnt, 2 * (size_t)c->n_lj_blocks * sizeof(unsigned long long));
    ok = ok && alloc((void**)&c->ke_part, (size_t)c->n_ke_blocks * sizeof(double));
    ok = ok && alloc((void**)&c->d_res, sizeof(ResultDev));
    ok = ok && alloc((void**)&c->d_status, sizeof(int));
    ok = ok && alloc((void**)&c->d_maxocc, 4 * sizeof(int));
    ok = ok && cudaMallocHost((void**)&c->h_res, sizeof(ResultDev)) == cudaSuccess;
    ok = ok && cudaMallocHost((void**)&c->h_status, sizeof(int)) == cudaSuccess;
    ok = ok && cudaMallocHost((void**)&c->h_maxocc, 4 * sizeof(int)) == cudaSuccess;
    ok = ok && cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                                      params->device) == cudaSuccess;
    ok = ok && cudaMemsetAsync(c->d_status, 0, sizeof(int), c->st) == cudaSuccess;
    ok = ok && cudaMemsetAsync(c->v, 0, 3 * N * sizeof(double), c->st) == cudaSuccess;
    ok = ok && cudaStreamSynchronize(c->st) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_all(c);
        delete c;
        return ATM_E_CUDA;
    }
    *c->h_status = 0;
    *out = c;
    return ATM_OK;
}

extern "C" atm_status atm_destroy(atm_ctx* c)
{
    if (!c) return ATM_OK;
    cudaSetDevice(c->p.device);
    cudaStreamSynchronize(c->st);
    free_all(c);
    delete c;
    return ATM_OK;
}

extern "C" atm_status atm_set_state(atm_ctx* c, const double* x, const double* v)
{
    if (!c) return ATM_E_INVALID;
    if (!x && c->n > 0) return fail(c, ATM_E_INVALID, "positions are required");
    for (long long q = 0; q < 3 * c->n; q++)
        if (!std::isfinite(x[q]) || (v && !std::isfinite(v[q])))
            return fail(c, ATM_E_NONFINITE, "non-finite input at element %lld", q);
    CU(cudaSetDevice(c->p.device));
    size_t bytes = 3 * (size_t)c->n * sizeof(double);
    if (bytes) {
        CU(cudaMemcpyAsync(c->x, x, bytes, cudaMemcpyHostToDevice, c->st));
        if (v)
            CU(cudaMemcpyAsync(c->v, v, bytes, cudaMemcpyHostToDevice, c->st));
        else
            CU(cudaMemsetAsync(c->v, 0, bytes, c->st));
    }
    c->have_x = true;
    c->cells_built = false;
    c->forces_valid = false;
    return ATM_OK;
}

extern "C" atm_status atm_set_state_dev(atm_ctx* c, const double* x_dev, const double* v_dev)
{
    if (!c) return ATM_E_INVALID;
    if (!x_dev && c->n > 0) return fail(c, ATM_E_INVALID, "positions are required");
    CU(cudaSetDevice(c->p.device));
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
    c->cells_built = false;
    c->forces_valid = false;
    return ATM_OK;
}

static atm_status enqueue_cells(atm_ctx* c)
{
    cudaEvent_t ev = prof_begin(c);
    CU(launch_build_cells(c->g, c->n, c->x, c->cell_of, c->rank, c->count, c->start, c->perm,
                          c->xl, c->xl32, c->cell_sorted, c->d_maxocc, c->d_status, c->st));
    prof_end(c, PK_CELLS, ev);
    c->n_launch += c->n > 0 ? 5 : 1;
    CU(cudaMemcpyAsync(c->h_maxocc, c->d_maxocc, 4 * sizeof(int), cudaMemcpyDeviceToHost, c->st));
    atm_status s = sync_and_check(c);
    if (s != ATM_OK) return s;
    c->maxocc = c->h_maxocc[0];
    for (int t = 0; t < 3; t++) c->unit_max[t] = c->h_maxocc[1 + t];
    c->cells_built = true;
    c->forces_valid = false;
    return ATM_OK;
}

extern "C" atm_status atm_build_cells(atm_ctx* c)
{
    if (!c) return ATM_E_INVALID;
    if (!c->have_x) return fail(c, ATM_E_STATE, "no state set");
    CU(cudaSetDevice(c->p.device));
    return enqueue_cells(c);
}

extern "C" atm_status atm_get_cells(atm_ctx* c, int32_t* cell_of, int32_t* cell_start,
                                    int32_t* perm, int32_t* ncell3)
{
    if (!c) return ATM_E_INVALID;
    if (ncell3)
        for (int d = 0; d < 3; d++) ncell3[d] = c->g.nc[d];
    if (!c->cells_built) return fail(c, ATM_E_STATE, "cells not built");
    CU(cudaSetDevice(c->p.device));
    if (cell_of && c->n)
        CU(cudaMemcpyAsync(cell_of, c->cell_of, c->n * sizeof(int), cudaMemcpyDeviceToHost, c->st));
    if (cell_start)
        CU(cudaMemcpyAsync(cell_start, c->start, (c->g.ncell + 1) * sizeof(int),
                           cudaMemcpyDeviceToHost, c->st));
    if (perm && c->n)
        CU(cudaMemcpyAsync(perm, c->perm, c->n * sizeof(int), cudaMemcpyDeviceToHost, c->st));
    CU(cudaStreamSynchronize(c->st));
    return ATM_OK;
}

// LJ + ATM force kernels for the current cells
static atm_status enqueue_forces(atm_ctx* c, int trav, int trunc, int prec)
{
    ForceJob j;
    j.g = c->g;
    j.n = c->n;
    j.xl = c->xl;
    j.xl32 = c->xl32;
    j.start = c->start;
    j.cell_sorted = c->cell_sorted;
    j.f_lj = c->f_lj;
    j.f_atm = c->f_atm;
    j.lj_ew = c->lj_ew;
    j.lj_cnt = c->lj_cnt;
    j.unit_ew = c->unit_ew;
    j.unit_cnt = c->unit_cnt;
    j.status = c->d_status;
    j.rc = c->p.rc;
    j.nu = c->p.nu;
    j.lj_eps = c->p.lj_eps;
    j.lj_sigma = c->p.lj_sigma;
    j.lj_shift = c->p.lj_shift;
    j.trav = trav;
    j.trunc = trunc;
    j.prec = prec;
    j.mcap = c->unit_max[trav] > 0 ? c->unit_max[trav] : 1;
    j.optin = c->smem_optin;
    j.st = c->st;

    cudaEvent_t ev = prof_begin(c);
    CU(enqueue_lj(j));
    prof_end(c, PK_LJ, ev);
    c->n_launch += 1;

    ev = prof_begin(c);
    bool capacity = false;
    cudaError_t e = enqueue_atm(j, &c->smem_set[prec][trav][trunc], &capacity);
    if (capacity)
        return fail(c, ATM_E_CAPACITY,
                    "a traversal unit of %d molecules does not fit the kernels' shared memory",
                    j.mcap);
    CU(e);
    prof_end(c, PK_ATM, ev);
    c->n_launch += 1;
    c->n_atm += 1;
    c->forces_valid = true;
    c->f_trav = trav;
    c->f_trunc = trunc;
    c->f_prec = prec;
    return ATM_OK;
}

static atm_status enqueue_reduce(atm_ctx* c)
{
    ReduceArgs r;
    r.unit_ew = c->unit_ew;
    r.unit_cnt = c->unit_cnt;
    r.n_units = c->g.ncell;
    r.lj_ew = c->lj_ew;
    r.lj_cnt = c->lj_cnt;
    r.n_lj = c->n_lj_blocks;
    r.ke_part = c->ke_part;
    r.n_ke = c->n_ke_blocks;
    r.out = c->d_res;
    cudaEvent_t ev = prof_begin(c);
    CU(launch_final_reduce(r, c->st));
    prof_end(c, PK_MD, ev);
    c->n_launch += 1;
    CU(cudaMemcpyAsync(c->h_res, c->d_res, sizeof(ResultDev), cudaMemcpyDeviceToHost, c->st));
    return ATM_OK;
}

static void copy_result(const atm_ctx* c, atm_result* out)
{
    const ResultDev* r = c->h_res;
    out->e2 = r->e2;
    out->e3 = r->e3;
    out->w2 = r->w2;
    out->w3 = r->w3;
    out->ekin = r->ekin;
    out->n_cand3 = r->n_cand3;
    out->n_int3 = r->n_int3;
    out->n_cand2 = r->n_cand2;
    out->n_int2 = r->n_int2;
}

static bool valid_enums(int trav, int trunc, int prec)
{
    return trav >= 0 && trav <= 2 && trunc >= 0 && trunc <= 1 && prec >= 0 && prec <= 1;
}

extern "C" atm_status atm_compute_forces(atm_ctx* c, atm_traversal trav, atm_truncation trunc,
                                         atm_precision prec, atm_result* out)
{
    if (!c) return ATM_E_INVALID;
    if (!valid_enums(trav, trunc, prec)) return fail(c, ATM_E_INVALID, "unknown traversal/truncation/precision");
    if (!c->cells_built) return fail(c, ATM_E_STATE, "cells not built");
    CU(cudaSetDevice(c->p.device));
    atm_status s = enqueue_forces(c, trav, trunc, prec);
    if (s != ATM_OK) return s;
    cudaEvent_t ev = prof_begin(c);
    CU(launch_kinetic(c->n, c->v, c->ke_part, c->st));
    prof_end(c, PK_MD, ev);
    c->n_launch += 1;
    s = enqueue_reduce(c);
    if (s != ATM_OK) return s;
    if (out) {
        s = sync_and_check(c);
        if (s != ATM_OK) return s;
        copy_result(c, out);
    }
    return ATM_OK;
}

static atm_status get_forces_impl(atm_ctx* c, double* f, int which, bool host)
{
    if (!c || !f || which < 0 || which > 2) return ATM_E_INVALID;
    if (!c->forces_valid) return fail(c, ATM_E_STATE, "no force evaluation is current");
    CU(cudaSetDevice(c->p.device));
    size_t bytes = 3 * (size_t)c->n * sizeof(double);
    if (!bytes) return ATM_OK;
    CU(launch_gather_forces(c->n, c->perm, c->f_lj, c->f_atm, which, host ? c->f_out : f, c->st));
    c->n_launch += 1;
    if (host) {
        CU(cudaMemcpyAsync(f, c->f_out, bytes, cudaMemcpyDeviceToHost, c->st));
        return sync_and_check(c);
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
    if (!c->have_x) return fail(c, ATM_E_STATE, "no state set");
    CU(cudaSetDevice(c->p.device));
    size_t bytes = 3 * (size_t)c->n * sizeof(double);
    if (bytes && x) CU(cudaMemcpyAsync(x, c->x, bytes, cudaMemcpyDeviceToHost, c->st));
    if (bytes && v) CU(cudaMemcpyAsync(v, c->v, bytes, cudaMemcpyDeviceToHost, c->st));
    CU(cudaStreamSynchronize(c->st));
    return ATM_OK;
}

extern "C" atm_status atm_step(atm_ctx* c, int nsteps, atm_traversal trav, atm_truncation trunc,
                               atm_precision prec, atm_result* last)
{
    if (!c) return ATM_E_INVALID;
    if (nsteps < 0 || !valid_enums(trav, trunc, prec))
        return fail(c, ATM_E_INVALID, "bad step arguments");
    if (!c->have_x) return fail(c, ATM_E_STATE, "no state set");
    CU(cudaSetDevice(c->p.device));
    atm_status s;
    if (!c->forces_valid || c->f_trav != trav || c->f_trunc != trunc || c->f_prec != prec) {
        s = enqueue_cells(c);
        if (s != ATM_OK) return s;
        s = enqueue_forces(c, trav, trunc, prec);
        if (s != ATM_OK) return s;
    }
    const double dt = c->p.dt, half_dt = 0.5 * c->p.dt;
    for (int k = 0; k < nsteps; k++) {
        cudaEvent_t ev = prof_begin(c);
        CU(launch_kick(c->n, c->perm, c->f_lj, c->f_atm, c->x, c->v, half_dt, dt, 1, c->ke_part,
                       c->st));
        prof_end(c, PK_MD, ev);
        c->n_launch += 1;
        s = enqueue_cells(c);
        if (s != ATM_OK) return s;
        s = enqueue_forces(c, trav, trunc, prec);
        if (s != ATM_OK) return s;
        ev = prof_begin(c);
        CU(launch_kick(c->n, c->perm, c->f_lj, c->f_atm, c->x, c->v, half_dt, dt, 0, c->ke_part,
                       c->st));
        prof_end(c, PK_MD, ev);
        c->n_launch += 1;
    }
    if (nsteps == 0) {
        CU(launch_kinetic(c->n, c->v, c->ke_part, c->st));
        c->n_launch += 1;
    }
    s = enqueue_reduce(c);
    if (s != ATM_OK) return s;
    if (last) {
        s = sync_and_check(c);
        if (s != ATM_OK) return s;
        copy_result(c, last);
    }
    return ATM_OK;
}

extern "C" atm_status atm_set_profiling(atm_ctx* c, int on)
{
    if (!c) return ATM_E_INVALID;
    CU(cudaSetDevice(c->p.device));
    CU(cudaStreamSynchronize(c->st));
    prof_drain(c);
    c->prof = on != 0;
    for (double& v : c->prof_ms) v = 0.0;
    c->n_launch = 0;
    c->n_atm = 0;
    return ATM_OK;
}

extern "C" atm_status atm_get_profile(atm_ctx* c, atm_profile* out)
{
    if (!c || !out) return ATM_E_INVALID;
    CU(cudaSetDevice(c->p.device));
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
