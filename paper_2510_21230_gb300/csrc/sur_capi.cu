// sur_capi.cu -- C ABI of the learned ATM force surrogate (include/atm3.h):
// model, data set, training loop, inference inside atm_compute_forces /
// atm_step, and the exact-vs-surrogate comparison of interleaved steps.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "atm3.h"
#include "ctx.cuh"
#include "surrogate.cuh"

using namespace atm3;

static_assert(ATM_SUR_NPARAM == SUR_NP && ATM_SUR_NDESC == SUR_ND && ATM_SUR_NVEC == SUR_NV,
              "public and kernel model sizes agree");

namespace atm3 {

struct SurState {
    // model: FP32 master parameters, Adam moments, normalisation, packed copy
    float* P = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    float* mean = nullptr;
    float* scale = nullptr;
    SurPacked* packed = nullptr;
    bool have_model = false;
    long long adam_t = 0;
    // data set [cap] rows
    float* D = nullptr;
    float* V = nullptr;
    float* T = nullptr;
    long long rows = 0, cap = 0;
    double sigma2 = 0.0;
    bool sigma2_valid = false;
    // training scratch
    long long* idx = nullptr;
    long long idx_cap = 0;
    float* part = nullptr;
    double* part_loss = nullptr;
    int part_cap = 0;
    double* d_loss = nullptr;
    long long loss_cap = 0;
    double* stat_part = nullptr;   // [SUR_STAT_PARTS][33]
    double* stat_center = nullptr; // [32]
    float* grad = nullptr;         // [SUR_NP]
    // staging of host rows
    void* rows_buf = nullptr;
    size_t rows_bytes = 0;
    // interleaved exact steps
    int exact_every = 50;
    long long count = 0;
    double* f_scratch = nullptr;  // [3n] surrogate force at an exact step
    // per-evaluation scratch of the kernels (n rows)
    float4* xl4 = nullptr;
    __nv_bfloat16* xb = nullptr;
    float* vb = nullptr;
    double* d_mon = nullptr;      // [2] sum |diff|^2, sum |exact|^2
    long long checks = 0;
    // gradients on the tensor cores (bfloat16 operands, FP32 accumulators;
    // the default) or in FP32 on the CUDA cores
    int train_tc = 1;
};

}  // namespace atm3

namespace {

SurState* state(atm_ctx* c)
{
    if (!c->sur) c->sur = new (std::nothrow) SurState();
    return c->sur;
}

atm_status model_alloc(atm_ctx* c, SurState* S)
{
    if (S->P) return ATM_OK;
    CU(cudaMalloc(&S->P, SUR_NP * sizeof(float)));
    CU(cudaMalloc(&S->m, SUR_NP * sizeof(float)));
    CU(cudaMalloc(&S->v, SUR_NP * sizeof(float)));
    CU(cudaMalloc(&S->grad, SUR_NP * sizeof(float)));
    CU(cudaMalloc(&S->mean, SUR_ND * sizeof(float)));
    CU(cudaMalloc(&S->scale, SUR_ND * sizeof(float)));
    CU(cudaMalloc(&S->packed, sizeof(SurPacked)));
    return ATM_OK;
}

// upload a model and reset the optimiser
atm_status model_upload(atm_ctx* c, SurState* S, const float* P, const float* mean,
                        const float* scale)
{
    for (int k = 0; k < SUR_NP; k++)
        if (!std::isfinite(P[k])) return ctx_fail(c, ATM_E_INVALID, "non-finite parameter %d", k);
    for (int k = 0; k < SUR_ND; k++)
        if (!std::isfinite(mean[k]) || !(scale[k] > 0.0f) || !std::isfinite(scale[k]))
            return ctx_fail(c, ATM_E_INVALID, "bad normalisation of descriptor %d", k);
    atm_status s = model_alloc(c, S);
    if (s != ATM_OK) return s;
    CU(cudaMemcpyAsync(S->P, P, SUR_NP * sizeof(float), cudaMemcpyHostToDevice, c->st));
    CU(cudaMemcpyAsync(S->mean, mean, SUR_ND * sizeof(float), cudaMemcpyHostToDevice, c->st));
    CU(cudaMemcpyAsync(S->scale, scale, SUR_ND * sizeof(float), cudaMemcpyHostToDevice, c->st));
    CU(cudaMemsetAsync(S->m, 0, SUR_NP * sizeof(float), c->st));
    CU(cudaMemsetAsync(S->v, 0, SUR_NP * sizeof(float), c->st));
    CU(launch_sur_pack(S->P, S->mean, S->scale, S->packed, c->st));
    CU(cudaStreamSynchronize(c->st));
    S->have_model = true;
    S->adam_t = 0;
    return ATM_OK;
}

// device staging area for host rows
atm_status stage(atm_ctx* c, SurState* S, size_t bytes, void** out)
{
    if (bytes > S->rows_bytes) {
        if (S->rows_buf) cudaFree(S->rows_buf);
        S->rows_buf = nullptr;
        S->rows_bytes = 0;
        CU(cudaMalloc(&S->rows_buf, bytes));
        S->rows_bytes = bytes;
    }
    *out = S->rows_buf;
    return ATM_OK;
}

size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }

// mean, scale of the data-set descriptors and sigma2 of its targets
// (two passes, fixed partial sums summed in order on the host)
atm_status dataset_stats(atm_ctx* c, SurState* S, float* mean, float* scale)
{
    if (!S->stat_part) {
        CU(cudaMalloc(&S->stat_part, SUR_STAT_PARTS * (SUR_ND + 1) * sizeof(double)));
        CU(cudaMalloc(&S->stat_center, SUR_ND * sizeof(double)));
    }
    std::vector<double> part(SUR_STAT_PARTS * (SUR_ND + 1));
    auto pass = [&](const double* center, int square) -> atm_status {
        CU(launch_sur_stats(S->D, S->T, S->rows, center, square, S->stat_part, c->st));
        CU(cudaMemcpyAsync(part.data(), S->stat_part, part.size() * sizeof(double),
                           cudaMemcpyDeviceToHost, c->st));
        CU(cudaStreamSynchronize(c->st));
        return ATM_OK;
    };
    const double rows = (double)S->rows;
    atm_status s = pass(nullptr, 0);
    if (s != ATM_OK) return s;
    double mu[SUR_ND], t2 = 0.0;
    for (int k = 0; k < SUR_ND; k++) {
        double a = 0.0;
        for (int p = 0; p < SUR_STAT_PARTS; p++) a += part[p * (SUR_ND + 1) + k];
        mu[k] = a / rows;
    }
    for (int p = 0; p < SUR_STAT_PARTS; p++) t2 += part[p * (SUR_ND + 1) + SUR_ND];
    CU(cudaMemcpyAsync(S->stat_center, mu, sizeof(mu), cudaMemcpyHostToDevice, c->st));
    s = pass(S->stat_center, 1);
    if (s != ATM_OK) return s;
    for (int k = 0; k < SUR_ND; k++) {
        double q = 0.0;
        for (int p = 0; p < SUR_STAT_PARTS; p++) q += part[p * (SUR_ND + 1) + k];
        const double sd = std::sqrt(q / rows);
        if (mean) mean[k] = (float)mu[k];
        if (scale) scale[k] = sd < 1e-12 ? 1.0f : (float)sd;
    }
    S->sigma2 = t2 / (3.0 * rows);
    S->sigma2_valid = true;
    return ATM_OK;
}

// splitmix64 (Steele, Lea & Flood 2014)
uint64_t splitmix64(uint64_t& x)
{
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// kernel arguments for the context's current cells (scratch allocated on first use)
atm_status sur_args(atm_ctx* c, SurState* S, SurForceArgs& a)
{
    if (!S->xl4 && c->n > 0) {
        // the MLP's tiles are read whole: pad to a multiple of the tile rows
        const size_t rows = (size_t)((c->n + SUR_TILE_M - 1) / SUR_TILE_M) * SUR_TILE_M;
        CU(cudaMalloc(&S->xl4, (size_t)c->n * sizeof(float4)));
        CU(cudaMalloc(&S->xb, rows * SUR_ND * sizeof(__nv_bfloat16)));
        CU(cudaMalloc(&S->vb, rows * SUR_NV * sizeof(float)));
        CU(cudaMemsetAsync(S->xb, 0, rows * SUR_ND * sizeof(__nv_bfloat16), c->st));
        CU(cudaMemsetAsync(S->vb, 0, rows * SUR_NV * sizeof(float), c->st));
    }
    a = SurForceArgs{};
    a.b = c->b;
    a.n = c->n;
    a.xl32 = c->xl32;
    a.cell_start = c->start;
    a.cell_sorted = c->cell_sorted;
    a.model = S->packed;
    a.xl4 = S->xl4;
    a.xb = S->xb;
    a.vb = S->vb;
    a.status = c->d_status;
    a.sms = c->sms;
    return ATM_OK;
}

}  // namespace

// ---------------------------------------------------------- library hooks

atm_status atm3::sur_enqueue_atm(atm_ctx* c)
{
    SurState* S = c->sur;
    if (!S || !S->have_model)
        return ctx_fail(c, ATM_E_STATE, "surrogate forces need a model (set, load or init + train)");
    // no triplets: the per-unit energy / virial / count sums are zero
    CU(cudaMemsetAsync(c->unit_ew, 0, 2 * (size_t)c->ncell * sizeof(double), c->st));
    CU(cudaMemsetAsync(c->unit_cnt, 0, 2 * (size_t)c->ncell * sizeof(unsigned long long), c->st));
    SurForceArgs a;
    atm_status s = sur_args(c, S, a);
    if (s != ATM_OK) return s;
    a.f_atm = c->f_atm;
    // LJ from the descriptor kernel's neighbour pass
    a.f_lj = c->f_lj;
    a.mol_ew = c->mol_ew;
    a.mol_cnt = c->mol_cnt;
    a.mode = 0;
    CU(launch_sur_forces(a, c->st));
    c->n_launch += SUR_LAUNCHES;
    return ATM_OK;
}

atm_status atm3::sur_enqueue_monitor(atm_ctx* c)
{
    SurState* S = c->sur;
    if (!S || !S->have_model || c->n == 0) return ATM_OK;
    if (!S->f_scratch) {
        CU(cudaMalloc(&S->f_scratch, 3 * (size_t)c->n * sizeof(double)));
        CU(cudaMalloc(&S->d_mon, 2 * sizeof(double)));
        CU(cudaMemsetAsync(S->d_mon, 0, 2 * sizeof(double), c->st));
    }
    SurForceArgs a;
    atm_status s = sur_args(c, S, a);
    if (s != ATM_OK) return s;
    a.f_atm = S->f_scratch;
    a.mode = 0;
    CU(launch_sur_forces(a, c->st));
    CU(launch_sur_diff(c->n, S->f_scratch, c->f_atm, S->d_mon, c->st));
    c->n_launch += SUR_LAUNCHES + 1;
    S->checks += 1;
    return ATM_OK;
}

bool atm3::sur_exact_due(atm_ctx* c)
{
    SurState* S = c->sur;
    return S && S->exact_every > 0 && S->count % S->exact_every == 0;
}

void atm3::sur_count_step(atm_ctx* c)
{
    if (c->sur) c->sur->count += 1;
}

int atm3::sur_exact_every(const atm_ctx* c) { return c->sur ? c->sur->exact_every : 50; }

void atm3::sur_free(atm_ctx* c)
{
    SurState* S = c->sur;
    if (!S) return;
    void* dev[] = {S->P, S->m, S->v, S->mean, S->scale, S->packed, S->D, S->V, S->T,
                   S->idx, S->part, S->part_loss, S->d_loss, S->stat_part, S->stat_center,
                   S->grad, S->rows_buf, S->f_scratch, S->d_mon, S->xl4, S->xb, S->vb};
    for (void* p : dev)
        if (p) cudaFree(p);
    delete S;
    c->sur = nullptr;
}

// -------------------------------------------------------------- the ABI

extern "C" atm_status atm_surrogate_set_model(atm_ctx* c, const float* params, const float* mean,
                                              const float* scale)
{
    if (!c) return ATM_E_INVALID;
    if (!params || !mean || !scale) return ctx_fail(c, ATM_E_INVALID, "NULL model array");
    SurState* S = state(c);
    if (!S) return ctx_fail(c, ATM_E_CUDA, "out of host memory");
    CU(cudaSetDevice(c->device));
    return model_upload(c, S, params, mean, scale);
}

extern "C" atm_status atm_surrogate_get_model(atm_ctx* c, float* params, float* mean, float* scale)
{
    if (!c) return ATM_E_INVALID;
    SurState* S = c->sur;
    if (!S || !S->have_model) return ctx_fail(c, ATM_E_STATE, "no surrogate model");
    CU(cudaSetDevice(c->device));
    if (params) CU(cudaMemcpyAsync(params, S->P, SUR_NP * sizeof(float), cudaMemcpyDeviceToHost, c->st));
    if (mean) CU(cudaMemcpyAsync(mean, S->mean, SUR_ND * sizeof(float), cudaMemcpyDeviceToHost, c->st));
    if (scale) CU(cudaMemcpyAsync(scale, S->scale, SUR_ND * sizeof(float), cudaMemcpyDeviceToHost, c->st));
    CU(cudaStreamSynchronize(c->st));
    return ATM_OK;
}

extern "C" atm_status atm_surrogate_init(atm_ctx* c, uint64_t seed)
{
    if (!c) return ATM_E_INVALID;
    SurState* S = state(c);
    if (!S) return ctx_fail(c, ATM_E_CUDA, "out of host memory");
    if (S->rows == 0) return ctx_fail(c, ATM_E_STATE, "the surrogate data set is empty");
    CU(cudaSetDevice(c->device));
    float mean[SUR_ND], scale[SUR_ND];
    atm_status s = dataset_stats(c, S, mean, scale);
    if (s != ATM_OK) return s;
    std::vector<float> P(SUR_NP, 0.0f);
    uint64_t x = seed;
    auto uni = [&](double a) {
        const double u = (double)(splitmix64(x) >> 11) * (1.0 / 9007199254740992.0);
        return (float)((2.0 * u - 1.0) * a);
    };
    const double a1 = std::sqrt(6.0 / (SUR_ND + SUR_NH)), a2 = std::sqrt(6.0 / (SUR_NH + SUR_NH));
    const double a3 = 0.1 * std::sqrt(6.0 / (SUR_NH + SUR_NO));
    for (int k = 0; k < SUR_ND * SUR_NH; k++) P[SUR_OFF_W1 + k] = uni(a1);
    for (int k = 0; k < SUR_NH * SUR_NH; k++) P[SUR_OFF_W2 + k] = uni(a2);
    for (int k = 0; k < SUR_NH * SUR_NO; k++) P[SUR_OFF_W3 + k] = uni(a3);
    return model_upload(c, S, P.data(), mean, scale);
}

extern "C" atm_status atm_surrogate_save(atm_ctx* c, const char* path)
{
    if (!c) return ATM_E_INVALID;
    if (!path) return ctx_fail(c, ATM_E_INVALID, "NULL path");
    std::vector<float> P(SUR_NP), mean(SUR_ND), scale(SUR_ND);
    atm_status s = atm_surrogate_get_model(c, P.data(), mean.data(), scale.data());
    if (s != ATM_OK) return s;
    FILE* f = std::fopen(path, "wb");
    if (!f) return ctx_fail(c, ATM_E_INVALID, "cannot open %s for writing", path);
    const int32_t counts[2] = {SUR_NP, SUR_ND};
    bool ok = std::fwrite("ATMSUR01", 1, 8, f) == 8 && std::fwrite(counts, 4, 2, f) == 2 &&
              std::fwrite(P.data(), 4, SUR_NP, f) == (size_t)SUR_NP &&
              std::fwrite(mean.data(), 4, SUR_ND, f) == (size_t)SUR_ND &&
              std::fwrite(scale.data(), 4, SUR_ND, f) == (size_t)SUR_ND;
    ok = (std::fclose(f) == 0) && ok;
    return ok ? ATM_OK : ctx_fail(c, ATM_E_INVALID, "write to %s failed", path);
}

extern "C" atm_status atm_surrogate_load(atm_ctx* c, const char* path)
{
    if (!c) return ATM_E_INVALID;
    if (!path) return ctx_fail(c, ATM_E_INVALID, "NULL path");
    FILE* f = std::fopen(path, "rb");
    if (!f) return ctx_fail(c, ATM_E_INVALID, "cannot open %s", path);
    char tag[8];
    int32_t counts[2];
    std::vector<float> P(SUR_NP), mean(SUR_ND), scale(SUR_ND);
    bool ok = std::fread(tag, 1, 8, f) == 8 && std::memcmp(tag, "ATMSUR01", 8) == 0 &&
              std::fread(counts, 4, 2, f) == 2 && counts[0] == SUR_NP && counts[1] == SUR_ND &&
              std::fread(P.data(), 4, SUR_NP, f) == (size_t)SUR_NP &&
              std::fread(mean.data(), 4, SUR_ND, f) == (size_t)SUR_ND &&
              std::fread(scale.data(), 4, SUR_ND, f) == (size_t)SUR_ND;
    std::fclose(f);
    if (!ok) return ctx_fail(c, ATM_E_INVALID, "%s is not a surrogate model file", path);
    return atm_surrogate_set_model(c, P.data(), mean.data(), scale.data());
}

extern "C" atm_status atm_surrogate_descriptors(atm_ctx* c, float* desc, float* vec)
{
    if (!c) return ATM_E_INVALID;
    if (!desc || !vec) return ctx_fail(c, ATM_E_INVALID, "NULL output");
    if (!c->cells_built) return ctx_fail(c, ATM_E_STATE, "cells not built");
    SurState* S = state(c);
    if (!S) return ctx_fail(c, ATM_E_CUDA, "out of host memory");
    if (c->n == 0) return ATM_OK;
    CU(cudaSetDevice(c->device));
    const size_t n = (size_t)c->n;
    const size_t bd = al256(n * SUR_ND * 4), bv = al256(n * SUR_NV * 4), bt = al256(n * 3 * 4);
    void* buf = nullptr;
    atm_status s = stage(c, S, bd + bv + bt, &buf);
    if (s != ATM_OK) return s;
    char* b = static_cast<char*>(buf);
    SurForceArgs a;
    s = sur_args(c, S, a);
    if (s != ATM_OK) return s;
    a.f_atm = c->f_atm;  // read as the (unused) target rows
    a.d_out = reinterpret_cast<float*>(b);
    a.v_out = reinterpret_cast<float*>(b + bd);
    a.t_out = reinterpret_cast<float*>(b + bd + bv);
    a.row0 = 0;
    a.mode = 1;
    CU(launch_sur_forces(a, c->st));
    c->n_launch += 2;  // packing + descriptors
    std::vector<float> ds(n * SUR_ND), vs(n * SUR_NV);
    std::vector<int32_t> perm(n);
    CU(cudaMemcpyAsync(ds.data(), a.d_out, n * SUR_ND * 4, cudaMemcpyDeviceToHost, c->st));
    CU(cudaMemcpyAsync(vs.data(), a.v_out, n * SUR_NV * 4, cudaMemcpyDeviceToHost, c->st));
    CU(cudaMemcpyAsync(perm.data(), c->perm, n * 4, cudaMemcpyDeviceToHost, c->st));
    s = ctx_sync_and_check(c);
    if (s != ATM_OK) return s;
    // sorted slot s holds molecule perm[s]
    for (size_t k = 0; k < n; k++) {
        std::memcpy(desc + (size_t)perm[k] * SUR_ND, ds.data() + k * SUR_ND, SUR_ND * 4);
        std::memcpy(vec + (size_t)perm[k] * SUR_NV, vs.data() + k * SUR_NV, SUR_NV * 4);
    }
    return ATM_OK;
}

extern "C" atm_status atm_surrogate_mlp(atm_ctx* c, int64_t rows, const float* desc,
                                        const float* vec, float* w, float* force)
{
    if (!c) return ATM_E_INVALID;
    if (rows < 0 || (rows > 0 && (!desc || !vec || !w || !force)))
        return ctx_fail(c, ATM_E_INVALID, "bad surrogate rows");
    SurState* S = c->sur;
    if (!S || !S->have_model) return ctx_fail(c, ATM_E_STATE, "no surrogate model");
    if (rows == 0) return ATM_OK;
    CU(cudaSetDevice(c->device));
    const size_t n = (size_t)rows;
    const size_t bd = al256(n * SUR_ND * 4), bv = al256(n * SUR_NV * 4),
                 bw = al256(n * SUR_NO * 4), bf = al256(n * 3 * 4);
    void* buf = nullptr;
    atm_status s = stage(c, S, bd + bv + bw + bf, &buf);
    if (s != ATM_OK) return s;
    char* b = static_cast<char*>(buf);
    float* dD = reinterpret_cast<float*>(b);
    float* dV = reinterpret_cast<float*>(b + bd);
    float* dW = reinterpret_cast<float*>(b + bd + bv);
    float* dF = reinterpret_cast<float*>(b + bd + bv + bw);
    CU(cudaMemcpyAsync(dD, desc, n * SUR_ND * 4, cudaMemcpyHostToDevice, c->st));
    CU(cudaMemcpyAsync(dV, vec, n * SUR_NV * 4, cudaMemcpyHostToDevice, c->st));
    CU(launch_sur_mlp_rows(rows, dD, dV, S->packed, dW, dF, c->d_status, c->sms, c->st));
    c->n_launch += 1;
    CU(cudaMemcpyAsync(w, dW, n * SUR_NO * 4, cudaMemcpyDeviceToHost, c->st));
    CU(cudaMemcpyAsync(force, dF, n * 3 * 4, cudaMemcpyDeviceToHost, c->st));
    return ctx_sync_and_check(c);
}

namespace {

// gradient of the current master parameters over `batch` rows of (D, V, T)
// (idx = nullptr: rows 0..batch-1); Adam step when update != 0
atm_status grad_step(atm_ctx* c, SurState* S, const float* D, const float* V, const float* T,
                     const long long* idx, long long batch, double sigma2, int update, double lr,
                     double* loss_dev, float* grad_dev)
{
    const int nct = S->train_tc ? sur_grad_tc_tiles(batch) : (int)((batch + SUR_TILE - 1) / SUR_TILE);
    if (nct > S->part_cap) {
        if (S->part) cudaFree(S->part);
        if (S->part_loss) cudaFree(S->part_loss);
        S->part = nullptr;
        S->part_loss = nullptr;
        S->part_cap = 0;
        CU(cudaMalloc(&S->part, (size_t)nct * SUR_NP * sizeof(float)));
        CU(cudaMalloc(&S->part_loss, (size_t)nct * sizeof(double)));
        S->part_cap = nct;
    }
    SurGradArgs g{};
    g.D = D;
    g.V = V;
    g.T = T;
    g.idx = idx;
    g.batch = batch;
    g.P = S->P;
    g.mean = S->mean;
    g.scale = S->scale;
    g.norm = (float)(1.0 / (3.0 * (double)batch * sigma2));
    g.part = S->part;
    g.part_loss = S->part_loss;
    g.packed = S->packed;
    g.status = c->d_status;
    if (S->train_tc)
        CU(launch_sur_grad_tc(g, c->sms, c->st));
    else
        CU(launch_sur_grad(g, nct, c->st));
    SurAdamArgs a{};
    a.part = S->part;
    a.part_loss = S->part_loss;
    a.nct = nct;
    a.P = S->P;
    a.m = S->m;
    a.v = S->v;
    a.mean = S->mean;
    a.scale = S->scale;
    a.packed = S->packed;
    a.grad_out = grad_dev;
    a.loss_out = loss_dev;
    a.update = update;
    if (update) {
        S->adam_t += 1;
        const double b1 = 0.9, b2 = 0.999;
        a.lr = (float)lr;
        a.beta1 = (float)b1;
        a.beta2 = (float)b2;
        a.eps = 1e-8f;
        a.c1 = (float)(1.0 - std::pow(b1, (double)S->adam_t));
        a.c2 = (float)(1.0 - std::pow(b2, (double)S->adam_t));
    }
    CU(launch_sur_adam(a, c->st));
    c->n_launch += 2;
    return ATM_OK;
}

}  // namespace

extern "C" atm_status atm_surrogate_loss_grad(atm_ctx* c, int64_t rows, const float* desc,
                                              const float* vec, const float* target,
                                              double sigma2, double* loss, float* grad)
{
    if (!c) return ATM_E_INVALID;
    if (rows <= 0 || !desc || !vec || !target || !grad || !(sigma2 > 0.0))
        return ctx_fail(c, ATM_E_INVALID, "bad loss_grad arguments");
    SurState* S = c->sur;
    if (!S || !S->have_model) return ctx_fail(c, ATM_E_STATE, "no surrogate model");
    CU(cudaSetDevice(c->device));
    const size_t n = (size_t)rows;
    const size_t bd = al256(n * SUR_ND * 4), bv = al256(n * SUR_NV * 4), bt = al256(n * 3 * 4);
    void* buf = nullptr;
    atm_status s = stage(c, S, bd + bv + bt + 256, &buf);
    if (s != ATM_OK) return s;
    char* b = static_cast<char*>(buf);
    float* dD = reinterpret_cast<float*>(b);
    float* dV = reinterpret_cast<float*>(b + bd);
    float* dT = reinterpret_cast<float*>(b + bd + bv);
    double* dL = reinterpret_cast<double*>(b + bd + bv + bt);
    CU(cudaMemcpyAsync(dD, desc, n * SUR_ND * 4, cudaMemcpyHostToDevice, c->st));
    CU(cudaMemcpyAsync(dV, vec, n * SUR_NV * 4, cudaMemcpyHostToDevice, c->st));
    CU(cudaMemcpyAsync(dT, target, n * 3 * 4, cudaMemcpyHostToDevice, c->st));
    s = grad_step(c, S, dD, dV, dT, nullptr, rows, sigma2, 0, 0.0, dL, S->grad);
    if (s != ATM_OK) return s;
    double hl = 0.0;
    CU(cudaMemcpyAsync(grad, S->grad, SUR_NP * sizeof(float), cudaMemcpyDeviceToHost, c->st));
    CU(cudaMemcpyAsync(&hl, dL, sizeof(double), cudaMemcpyDeviceToHost, c->st));
    s = ctx_sync_and_check(c);
    if (s != ATM_OK) return s;
    if (loss) *loss = hl;
    return ATM_OK;
}

static atm_status reserve_rows(atm_ctx* c, SurState* S, long long need)
{
    if (need <= S->cap) return ATM_OK;
    const long long nc = std::max(need, S->cap * 2);
    float* D = nullptr;
    float* V = nullptr;
    float* T = nullptr;
    CU(cudaMalloc(&D, (size_t)nc * SUR_ND * sizeof(float)));
    cudaError_t e = cudaMalloc(&V, (size_t)nc * SUR_NV * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&T, (size_t)nc * 3 * sizeof(float));
    if (e == cudaSuccess && S->rows > 0) {
        e = cudaMemcpyAsync(D, S->D, (size_t)S->rows * SUR_ND * 4, cudaMemcpyDeviceToDevice, c->st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(V, S->V, (size_t)S->rows * SUR_NV * 4, cudaMemcpyDeviceToDevice, c->st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(T, S->T, (size_t)S->rows * 3 * 4, cudaMemcpyDeviceToDevice, c->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    }
    if (e != cudaSuccess) {
        cudaFree(D);
        if (V) cudaFree(V);
        if (T) cudaFree(T);
        return ctx_fail(c, ATM_E_CUDA, "growing the surrogate data set to %lld rows: %s", nc,
                        cudaGetErrorString(e));
    }
    if (S->D) cudaFree(S->D);
    if (S->V) cudaFree(S->V);
    if (S->T) cudaFree(S->T);
    S->D = D;
    S->V = V;
    S->T = T;
    S->cap = nc;
    return ATM_OK;
}

extern "C" atm_status atm_surrogate_add_frame(atm_ctx* c, atm_traversal trav, atm_truncation trunc,
                                              atm_precision prec)
{
    if (!c) return ATM_E_INVALID;
    if (trav < 0 || trav > 4 || trunc < 0 || trunc > 1 || prec < 0 || prec > 1)
        return ctx_fail(c, ATM_E_INVALID, "add_frame needs an exact traversal, truncation, precision");
    if (!c->cells_built) return ctx_fail(c, ATM_E_STATE, "cells not built");
    SurState* S = state(c);
    if (!S) return ctx_fail(c, ATM_E_CUDA, "out of host memory");
    CU(cudaSetDevice(c->device));
    atm_status s = ctx_want_wide(c, trav);
    if (s != ATM_OK) return s;
    s = reserve_rows(c, S, S->rows + c->n);
    if (s != ATM_OK) return s;
    s = ctx_enqueue_forces(c, trav, trunc, prec, c->unit_max[trav]);
    if (s != ATM_OK) return s;
    SurForceArgs a;
    s = sur_args(c, S, a);
    if (s != ATM_OK) return s;
    a.f_atm = c->f_atm;
    a.d_out = S->D;
    a.v_out = S->V;
    a.t_out = S->T;
    a.row0 = S->rows;
    a.mode = 1;
    CU(launch_sur_forces(a, c->st));
    c->n_launch += 2;  // packing + descriptors
    s = ctx_sync_and_check(c);
    if (s != ATM_OK) return s;
    S->rows += c->n;
    S->sigma2_valid = false;
    return ATM_OK;
}

extern "C" atm_status atm_surrogate_add_rows(atm_ctx* c, int64_t rows, const float* desc,
                                             const float* vec, const float* target)
{
    if (!c) return ATM_E_INVALID;
    if (rows < 0 || (rows > 0 && (!desc || !vec || !target)))
        return ctx_fail(c, ATM_E_INVALID, "bad surrogate rows");
    SurState* S = state(c);
    if (!S) return ctx_fail(c, ATM_E_CUDA, "out of host memory");
    if (rows == 0) return ATM_OK;
    CU(cudaSetDevice(c->device));
    atm_status s = reserve_rows(c, S, S->rows + rows);
    if (s != ATM_OK) return s;
    const size_t r0 = (size_t)S->rows, n = (size_t)rows;
    CU(cudaMemcpyAsync(S->D + r0 * SUR_ND, desc, n * SUR_ND * 4, cudaMemcpyHostToDevice, c->st));
    CU(cudaMemcpyAsync(S->V + r0 * SUR_NV, vec, n * SUR_NV * 4, cudaMemcpyHostToDevice, c->st));
    CU(cudaMemcpyAsync(S->T + r0 * 3, target, n * 3 * 4, cudaMemcpyHostToDevice, c->st));
    CU(cudaStreamSynchronize(c->st));
    S->rows += rows;
    S->sigma2_valid = false;
    return ATM_OK;
}

extern "C" atm_status atm_surrogate_dataset(atm_ctx* c, int64_t* rows, double* sigma2)
{
    if (!c) return ATM_E_INVALID;
    SurState* S = state(c);
    if (!S) return ctx_fail(c, ATM_E_CUDA, "out of host memory");
    if (rows) *rows = S->rows;
    if (sigma2) {
        if (S->rows > 0 && !S->sigma2_valid) {
            CU(cudaSetDevice(c->device));
            atm_status s = dataset_stats(c, S, nullptr, nullptr);
            if (s != ATM_OK) return s;
        }
        *sigma2 = S->rows > 0 ? S->sigma2 : 0.0;
    }
    return ATM_OK;
}

extern "C" atm_status atm_surrogate_clear(atm_ctx* c)
{
    if (!c) return ATM_E_INVALID;
    if (c->sur) {
        c->sur->rows = 0;
        c->sur->sigma2_valid = false;
    }
    return ATM_OK;
}

extern "C" atm_status atm_surrogate_train(atm_ctx* c, int64_t steps, int64_t batch, double lr,
                                          uint64_t seed, double* loss)
{
    if (!c) return ATM_E_INVALID;
    if (steps < 0 || !(lr > 0.0) || !std::isfinite(lr))
        return ctx_fail(c, ATM_E_INVALID, "bad training arguments");
    SurState* S = c->sur;
    if (!S || !S->have_model) return ctx_fail(c, ATM_E_STATE, "no surrogate model");
    if (S->rows == 0) return ctx_fail(c, ATM_E_STATE, "the surrogate data set is empty");
    if (steps == 0) return ATM_OK;
    CU(cudaSetDevice(c->device));
    if (!S->sigma2_valid) {
        atm_status s = dataset_stats(c, S, nullptr, nullptr);
        if (s != ATM_OK) return s;
    }
    if (!(S->sigma2 > 0.0)) return ctx_fail(c, ATM_E_STATE, "all target forces are zero");
    const bool full = batch <= 0 || batch >= S->rows;
    const long long B = full ? S->rows : batch;
    if (!full && B > S->idx_cap) {
        if (S->idx) cudaFree(S->idx);
        S->idx = nullptr;
        S->idx_cap = 0;
        CU(cudaMalloc(&S->idx, (size_t)B * sizeof(long long)));
        S->idx_cap = B;
    }
    if (steps > S->loss_cap) {
        if (S->d_loss) cudaFree(S->d_loss);
        S->d_loss = nullptr;
        S->loss_cap = 0;
        CU(cudaMalloc(&S->d_loss, (size_t)steps * sizeof(double)));
        S->loss_cap = steps;
    }
    for (long long t = 0; t < steps; t++) {
        if (!full) {
            CU(launch_sur_sample(S->idx, B, S->rows, seed, S->adam_t, c->st));
            c->n_launch += 1;
        }
        atm_status s = grad_step(c, S, S->D, S->V, S->T, full ? nullptr : S->idx, B, S->sigma2, 1,
                                 lr, S->d_loss + t, nullptr);
        if (s != ATM_OK) return s;
    }
    if (loss) CU(cudaMemcpyAsync(loss, S->d_loss, (size_t)steps * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    return ctx_sync_and_check(c);
}

extern "C" atm_status atm_surrogate_options(atm_ctx* c, int exact_every)
{
    if (!c) return ATM_E_INVALID;
    if (exact_every < 0) return ctx_fail(c, ATM_E_INVALID, "exact_every < 0");
    SurState* S = state(c);
    if (!S) return ctx_fail(c, ATM_E_CUDA, "out of host memory");
    S->exact_every = exact_every;
    S->count = 0;
    return ATM_OK;
}

extern "C" atm_status atm_surrogate_training_arithmetic(atm_ctx* c, int tensor_cores)
{
    if (!c) return ATM_E_INVALID;
    if (tensor_cores < 0 || tensor_cores > 1) return ctx_fail(c, ATM_E_INVALID, "0 or 1");
    SurState* S = state(c);
    if (!S) return ctx_fail(c, ATM_E_CUDA, "out of host memory");
    S->train_tc = tensor_cores;
    return ATM_OK;
}

extern "C" atm_status atm_surrogate_error(atm_ctx* c, double* rms_diff, double* rms_exact,
                                          int64_t* checks, int reset)
{
    if (!c) return ATM_E_INVALID;
    SurState* S = state(c);
    if (!S) return ctx_fail(c, ATM_E_CUDA, "out of host memory");
    double acc[2] = {0.0, 0.0};
    if (S->d_mon) {
        CU(cudaSetDevice(c->device));
        CU(cudaMemcpyAsync(acc, S->d_mon, sizeof(acc), cudaMemcpyDeviceToHost, c->st));
        atm_status s = ctx_sync_and_check(c);
        if (s != ATM_OK) return s;
    }
    const double cnt = 3.0 * (double)c->n * (double)S->checks;
    if (rms_diff) *rms_diff = cnt > 0 ? std::sqrt(acc[0] / cnt) : 0.0;
    if (rms_exact) *rms_exact = cnt > 0 ? std::sqrt(acc[1] / cnt) : 0.0;
    if (checks) *checks = S->checks;
    if (reset) {
        S->checks = 0;
        if (S->d_mon) {
            CU(cudaMemsetAsync(S->d_mon, 0, 2 * sizeof(double), c->st));
            CU(cudaStreamSynchronize(c->st));
        }
    }
    return ATM_OK;
}
