// noalloc.cu -- one force evaluation without any device allocation.
//
// For callers that cannot call cudaMalloc: code running where the device
// memory is already budgeted and owned by someone else (a host application
// that forbids allocation after start-up, a plug-in handed only raw device
// pointers, a process whose allocator is locked).  The caller passes the
// positions and the output buffers; every intermediate array (the linked
// cells, the sorted coordinates, the per-unit partial sums) lives in one
// file-scope __device__ array of fixed size below.
//
// The array belongs to every GPU that loads this library and stays reserved
// until the process exits.  In host code its name is only a host-side stand-in
// for the symbol, so the device address is fetched once per device with
// cudaGetSymbolAddress (with that device current) and passed to the kernels.
// Every call uses the same array and leaves its contents behind; everything
// that must start at zero is cleared on each call.  Two calls whose GPU work
// overlaps (different streams, or different host threads) race on the array.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "atm3.h"
#include "atm3_internal.cuh"
#include "forces.cuh"
#include "md_kernels.cuh"

using namespace atm3;

namespace {

constexpr size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }

struct NaLayout {
    size_t rep, rep_of_cell, rep_of_mol, x, cell_of, rank, count, start, perm, cell_sorted, xl,
        xl32, f_lj, f_atm, unit_ew, unit_cnt, mol_ew, mol_cnt, ke, res, status, maxocc, total;
};

constexpr long long NA_N = ATM_NOALLOC_MAX_N;
constexpr long long NA_C = ATM_NOALLOC_MAX_CELLS;

constexpr NaLayout na_layout()
{
    NaLayout L{};
    size_t o = 0;
    L.rep = o;         o = al256(o + sizeof(Rep));
    L.rep_of_cell = o; o = al256(o + NA_C * sizeof(int));
    L.rep_of_mol = o;  o = al256(o + NA_N * sizeof(int));
    L.x = o;           o = al256(o + 3 * NA_N * sizeof(double));
    L.cell_of = o;     o = al256(o + NA_N * sizeof(int));
    L.rank = o;        o = al256(o + NA_N * sizeof(int));
    L.count = o;       o = al256(o + NA_C * sizeof(int));
    L.start = o;       o = al256(o + (NA_C + 1) * sizeof(int));
    L.perm = o;        o = al256(o + NA_N * sizeof(int));
    L.cell_sorted = o; o = al256(o + NA_N * sizeof(int));
    L.xl = o;          o = al256(o + 3 * NA_N * sizeof(double));
    L.xl32 = o;        o = al256(o + 3 * NA_N * sizeof(float));
    L.f_lj = o;        o = al256(o + 3 * NA_N * sizeof(double));
    L.f_atm = o;       o = al256(o + 3 * NA_N * sizeof(double));
    L.unit_ew = o;     o = al256(o + 2 * NA_C * sizeof(double));
    L.unit_cnt = o;    o = al256(o + 2 * NA_C * sizeof(unsigned long long));
    L.mol_ew = o;      o = al256(o + 2 * NA_N * sizeof(double));
    L.mol_cnt = o;     o = al256(o + 2 * NA_N * sizeof(unsigned));
    L.ke = o;          o = al256(o + NA_N * sizeof(double));
    L.res = o;         o = al256(o + (1 + REDUCE_PARTS) * sizeof(ResultDev));
    L.status = o;      o = al256(o + sizeof(int));
    L.maxocc = o;      o = al256(o + (1 + ATM_NTRAV) * sizeof(int));
    L.total = o;
    return L;
}
constexpr NaLayout NA = na_layout();

// the scratch array (about 6.7 MB at the limits above)
__device__ __align__(256) unsigned char g_na_scratch[NA.total];

constexpr int NA_MAX_DEVICES = 64;
unsigned char* g_na_addr[NA_MAX_DEVICES] = {};
std::mutex g_na_mutex;

// device address of g_na_scratch on the current device (set-up on first use)
cudaError_t na_scratch(int device, unsigned char** out)
{
    std::lock_guard<std::mutex> lk(g_na_mutex);
    if (!g_na_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess) return e;
        g_na_addr[device] = static_cast<unsigned char*>(p);
    }
    *out = g_na_addr[device];
    return cudaSuccess;
}

}  // namespace

#define NA_CU(call)                                      \
    do {                                                 \
        if ((call) != cudaSuccess) return ATM_E_CUDA;    \
    } while (0)

namespace {
// makes params.device current for the call and gives the caller's current
// device back on every return path
struct DeviceScope {
    int prev = -1;
    bool ok = false;
    explicit DeviceScope(int device)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) return;
        ok = prev == device || cudaSetDevice(device) == cudaSuccess;
    }
    ~DeviceScope()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};
}  // namespace

static atm_status noalloc_run(const atm_params* p, int64_t n, const double* x_dev,
                              atm_traversal trav, atm_truncation trunc, atm_precision prec,
                              double* f_dev, atm_result* out);

extern "C" atm_status atm_compute_forces_noalloc(const atm_params* p, int64_t n,
                                                 const double* x_dev, atm_traversal trav,
                                                 atm_truncation trunc, atm_precision prec,
                                                 double* f_dev, atm_result* out)
{
    if (!p || n < 0 || (n > 0 && (!x_dev || !f_dev))) return ATM_E_INVALID;
    // 3c01, 3c18, 3c08 and the corner-anchored 3c08; the wide traversal needs
    // its 5^3 unit sizes, which this entry point does not form
    if (trav < 0 || trav > 4 || trav == ATM_3CW || trunc < 0 || trunc > 1 || prec < 0 || prec > 1)
        return ATM_E_INVALID;
    if (p->device < 0 || p->device >= NA_MAX_DEVICES) return ATM_E_INVALID;
    if (n > NA_N) return ATM_E_CAPACITY;
    DeviceScope dev(p->device);
    if (!dev.ok) return ATM_E_CUDA;
    return noalloc_run(p, n, x_dev, trav, trunc, prec, f_dev, out);
}

static atm_status noalloc_run(const atm_params* p, int64_t n, const double* x_dev,
                              atm_traversal trav, atm_truncation trunc, atm_precision prec,
                              double* f_dev, atm_result* out)
{
    // the single system as a batch of one replica
    Rep rp;
    atm_status rs = make_rep(*p, n, 0, 0, rp);
    if (rs != ATM_OK) return rs;
    if (rp.g.ncell > NA_C) return ATM_E_CAPACITY;

    unsigned char* base = nullptr;
    NA_CU(na_scratch(p->device, &base));
    cudaStream_t st = (cudaStream_t)p->cuda_stream;
    Rep* d_rep = reinterpret_cast<Rep*>(base + NA.rep);
    int* rep_of_cell = reinterpret_cast<int*>(base + NA.rep_of_cell);
    int* rep_of_mol = reinterpret_cast<int*>(base + NA.rep_of_mol);
    double* x = reinterpret_cast<double*>(base + NA.x);
    int* cell_of = reinterpret_cast<int*>(base + NA.cell_of);
    int* rank = reinterpret_cast<int*>(base + NA.rank);
    int* count = reinterpret_cast<int*>(base + NA.count);
    int* start = reinterpret_cast<int*>(base + NA.start);
    int* perm = reinterpret_cast<int*>(base + NA.perm);
    int* cell_sorted = reinterpret_cast<int*>(base + NA.cell_sorted);
    double* xl = reinterpret_cast<double*>(base + NA.xl);
    float* xl32 = reinterpret_cast<float*>(base + NA.xl32);
    double* f_lj = reinterpret_cast<double*>(base + NA.f_lj);
    double* f_atm = reinterpret_cast<double*>(base + NA.f_atm);
    double* unit_ew = reinterpret_cast<double*>(base + NA.unit_ew);
    unsigned long long* unit_cnt = reinterpret_cast<unsigned long long*>(base + NA.unit_cnt);
    double* mol_ew = reinterpret_cast<double*>(base + NA.mol_ew);
    unsigned* mol_cnt = reinterpret_cast<unsigned*>(base + NA.mol_cnt);
    double* ke = reinterpret_cast<double*>(base + NA.ke);
    ResultDev* res = reinterpret_cast<ResultDev*>(base + NA.res);
    int* status = reinterpret_cast<int*>(base + NA.status);
    int* maxocc = reinterpret_cast<int*>(base + NA.maxocc);

    Batch b;
    b.rep = d_rep;
    b.rep_of_cell = rep_of_cell;
    b.rep_of_mol = rep_of_mol;
    b.R = 1;
    b.ntot = n;
    b.ncell = rp.g.ncell;

    // replica descriptor and positions in (the cell build wraps positions in
    // place); replica ids, the status word and the kinetic energies start at zero
    const size_t bytes3 = 3 * (size_t)n * sizeof(double);
    NA_CU(cudaMemcpyAsync(d_rep, &rp, sizeof(Rep), cudaMemcpyHostToDevice, st));
    NA_CU(cudaMemsetAsync(rep_of_cell, 0, (size_t)b.ncell * sizeof(int), st));
    if (n > 0) {
        NA_CU(cudaMemsetAsync(rep_of_mol, 0, (size_t)n * sizeof(int), st));
        NA_CU(cudaMemsetAsync(ke, 0, (size_t)n * sizeof(double), st));
        NA_CU(cudaMemcpyAsync(x, x_dev, bytes3, cudaMemcpyDeviceToDevice, st));
    }
    NA_CU(cudaMemsetAsync(status, 0, sizeof(int), st));
    if (n > 0) NA_CU(launch_check_finite(3 * n, x, status, st));
    NA_CU(launch_build_cells(b, x, cell_of, rank, count, start, perm, xl, xl32, cell_sorted,
                             maxocc, status, false, st));
    int hocc[1 + ATM_NTRAV] = {}, hstat = 0;
    NA_CU(cudaMemcpyAsync(hocc, maxocc, sizeof(hocc), cudaMemcpyDeviceToHost, st));
    NA_CU(cudaMemcpyAsync(&hstat, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    NA_CU(cudaStreamSynchronize(st));
    if (hstat & ST_NONFINITE) return ATM_E_NONFINITE;

    // LJ pairs and ATM triplets (staged-molecule capacity = largest unit of the traversal)
    ForceJob j;
    j.b = b;
    j.rep_host = &rp;
    j.xl = xl;
    j.xl32 = xl32;
    j.start = start;
    j.cell_sorted = cell_sorted;
    j.f_lj = f_lj;
    j.f_atm = f_atm;
    j.mol_ew = mol_ew;
    j.mol_cnt = mol_cnt;
    j.unit_ew = unit_ew;
    j.unit_cnt = unit_cnt;
    j.status = status;
    j.work = nullptr;
    j.trav = trav;
    j.trunc = trunc;
    j.prec = prec;
    j.mcap = hocc[1 + trav] > 0 ? hocc[1 + trav] : 1;
    NA_CU(cudaDeviceGetAttribute(&j.optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device));
    j.sms = 0;
    j.persistent = 0;
    j.nwarps = 0;
    j.st = st;
    NA_CU(enqueue_lj(j));
    bool capacity = false;
    cudaError_t e = enqueue_atm(j, nullptr, &capacity);
    if (capacity) return ATM_E_CAPACITY;
    NA_CU(e);

    // scalars, then the total force in the caller's order
    ReduceArgs r;
    r.b = b;
    r.unit_ew = unit_ew;
    r.unit_cnt = unit_cnt;
    r.mol_ew = mol_ew;
    r.mol_cnt = mol_cnt;
    r.ke = ke;
    r.part = res + 1;
    r.out = res;
    NA_CU(launch_final_reduce(r, st));
    if (n > 0) NA_CU(launch_gather_forces(n, perm, f_lj, f_atm, 0, f_dev, st));
    ResultDev hres{};
    NA_CU(cudaMemcpyAsync(&hres, res, sizeof(ResultDev), cudaMemcpyDeviceToHost, st));
    NA_CU(cudaMemcpyAsync(&hstat, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    NA_CU(cudaStreamSynchronize(st));
    if (hstat & ST_NONFINITE) return ATM_E_NONFINITE;
    if (hstat & ST_CAPACITY) return ATM_E_CAPACITY;
    if (out) {
        out->e2 = hres.e2;
        out->e3 = hres.e3;
        out->w2 = hres.w2;
        out->w3 = hres.w3;
        out->ekin = 0.0;
        out->n_cand3 = hres.n_cand3;
        out->n_int3 = hres.n_int3;
        out->n_cand2 = hres.n_cand2;
        out->n_int2 = hres.n_int2;
    }
    return ATM_OK;
}
