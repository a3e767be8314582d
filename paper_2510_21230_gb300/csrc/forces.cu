// forces.cu -- replica descriptors, argument set-up and launch of the LJ and
// ATM force kernels, shared by the context API (capi.cu) and the
// allocation-free entry point (noalloc.cu).
#include <algorithm>
#include <cmath>

#include "forces.cuh"

namespace atm3 {

atm_status make_rep(const atm_params& p, long long n, long long mol0, long long cell0, Rep& r)
{
    r = Rep{};
    long long ncell = 1;
    for (int d = 0; d < 3; d++) {
        double L = p.box[d], rc = p.rc;
        if (!(L > 0.0) || !(rc > 0.0) || !std::isfinite(L) || !std::isfinite(rc)) return ATM_E_INVALID;
        double k = std::floor(L / rc);
        if (k < 1.0) k = 1.0;
        while (L / (k + 1.0) >= rc) k += 1.0;
        while (k > 0.0 && L / k < rc) k -= 1.0;
        if (k < 3.0) return ATM_E_BOX_TOO_SMALL;
        if (k > 1.0e6) return ATM_E_INVALID;
        r.g.nc[d] = (int)k;
        r.g.L[d] = L;
        r.g.w[d] = L / k;
        r.g.iw[d] = 1.0 / r.g.w[d];
        r.wf[d] = (float)r.g.w[d];
        ncell *= (long long)k;
    }
    if (ncell > (1ll << 30)) return ATM_E_INVALID;
    if (!std::isfinite(p.nu) || !std::isfinite(p.lj_eps) || !(p.lj_sigma > 0.0) ||
        !std::isfinite(p.dt))
        return ATM_E_INVALID;
    r.g.ncell = ncell;
    r.mol0 = mol0;
    r.n = n;
    r.cell0 = cell0;
    const double rc = p.rc;
    r.rc = rc;
    r.rc2 = rc * rc;
    r.rc6 = r.rc2 * r.rc2 * r.rc2;
    r.nu = p.nu;
    r.dt = p.dt;
    const float rcf = (float)rc;
    r.rcf = rcf;
    r.rc2f = rcf * rcf;
    r.rc6f = r.rc2f * r.rc2f * r.rc2f;
    r.nuf = (float)p.nu;
    const double sig2 = p.lj_sigma * p.lj_sigma;
    const double sc = sig2 / (rc * rc), sc3 = sc * sc * sc;
    r.sig2 = sig2;
    r.eps4 = 4.0 * p.lj_eps;
    r.eps24 = 24.0 * p.lj_eps;
    r.eps48 = 48.0 * p.lj_eps;
    r.ushift = p.lj_shift ? 4.0 * p.lj_eps * (sc3 * sc3 - sc3) : 0.0;
    r.sig2f = (float)r.sig2;
    r.eps4f = (float)r.eps4;
    r.eps24f = (float)r.eps24;
    r.eps48f = (float)r.eps48;
    r.ushiftf = (float)r.ushift;
    const double wmax = std::max(r.g.w[0], std::max(r.g.w[1], r.g.w[2]));
    r.p_lo = (float)(r.rc2 * (1.0 - 1.0 / 4096.0));
    r.p_hi = (float)(r.rc2 * (1.0 + 1.0 / 4096.0));
    r.q_lo = (float)(r.rc6 * (1.0 - 1.0 / 1024.0));
    r.q_hi = (float)(r.rc6 * (1.0 + 1.0 / 1024.0));
    r.dmin = (float)((0.02 * wmax) * (0.02 * wmax));
    const double wmin = std::min(r.g.w[0], std::min(r.g.w[1], r.g.w[2]));
    r.rw2 = (2.0 * wmin) * (2.0 * wmin);
    r.rw2f = (float)r.rw2;
    r.own_z0 = 0;
    r.own_z1 = r.g.nc[2];
    return ATM_OK;
}

cudaError_t enqueue_lj(const ForceJob& j)
{
    LjArgs<double> l64{};
    LjArgs<float> l32{};
    if (j.prec == 0) {
        l64.b = j.b; l64.n = j.b.ntot; l64.xl = j.xl; l64.xl32 = j.xl32; l64.cell_start = j.start;
        l64.cell_sorted = j.cell_sorted; l64.fs = j.f_lj; l64.mol_ew = j.mol_ew;
        l64.mol_cnt = j.mol_cnt;
    } else {
        l32.b = j.b; l32.n = j.b.ntot; l32.xl = j.xl32; l32.xl32 = j.xl32; l32.cell_start = j.start;
        l32.cell_sorted = j.cell_sorted; l32.fs = j.f_lj; l32.mol_ew = j.mol_ew;
        l32.mol_cnt = j.mol_cnt;
    }
    return launch_lj(j.prec, l64, l32, j.st);
}

// one ATM launch over all units, or over the listed units (ulist, ucount)
static cudaError_t launch_atm_one(const ForceJob& j, size_t* smem_set, bool* capacity,
                                  const int* ulist, const int* ucount, int* work)
{
    AtmPlan P;
    // the block kernel packs staged indices in 11 bits, the owner kernels in 16
    const int limit = (j.trav == 0 || j.trav == 3) ? 65535 : ATM_MCAP_LIMIT;
    if (j.mcap > limit || !atm_choose_plan(j.trav, j.trunc, j.prec, j.mcap, j.optin, P, j.det, j.gpm16)) {
        *capacity = true;
        return cudaErrorInvalidValue;
    }
    if ((j.nwarps == 2 || j.nwarps == 4 || j.nwarps == 8) && j.trav != 0 && j.trav != 3) {
        AtmPlan Q;
        if (atm_choose_plan_nw(j.trav, j.trunc, j.prec, j.mcap, j.optin, j.nwarps, Q, j.det, j.gpm16)) P = Q;
    }
    cudaError_t e;
    // the deterministic instantiations are other kernels: their attribute is
    // set on its own (smem_set tracks the floating-point ones)
    if (j.det || !smem_set || P.smem > *smem_set) {
        e = j.prec == 0 ? atm_attr_fp64(j.trav, j.trunc, P.smem, j.det)
                        : atm_attr_fp32(j.trav, j.trunc, P.smem, j.det);
        if (e != cudaSuccess) return e;
        if (smem_set && !j.det) *smem_set = P.smem;
    }
    const int lj = j.lj && (j.trav == 1 || j.trav == 2 || j.trav == 4) && j.trunc == 0;
    int ctas = 0;
    if (j.persistent && work) {
        int per_sm = j.prec == 0 ? atm_occupancy_fp64(j.trav, j.trunc, P.nwarps, P.smem, j.det)
                                 : atm_occupancy_fp32(j.trav, j.trunc, P.nwarps, P.smem, j.det);
        ctas = std::max(1, per_sm) * std::max(1, j.sms);
        e = cudaMemsetAsync(work, 0, sizeof(int), j.st);
        if (e != cudaSuccess) return e;
    }
    if (j.prec == 0) {
        AtmArgs<double> a{};
        a.b = j.b; a.n = j.b.ntot; a.xl = j.xl; a.xl32 = j.xl32; a.cell_start = j.start;
        a.fs = j.f_atm; a.unit_ew = j.unit_ew; a.unit_cnt = j.unit_cnt; a.status = j.status;
        a.work = ctas > 0 ? work : nullptr;
        a.mcap = j.mcap;
        a.gcap = P.gcap;
        a.use_d = P.use_d;
        a.acc_mode = P.acc_mode;
        a.pcap = P.pcap;
        a.lj = lj;
        a.unit_ew2 = j.unit_ew2;
        a.unit_cnt2 = j.unit_cnt2;
        a.ulist = ulist;
        a.ucount = ucount;
        a.det = j.det;
        a.emax = j.emax;
        return launch_atm_fp64(j.trav, j.trunc, a, P.nwarps, P.smem, ctas, j.st);
    }
    AtmArgs<float> a{};
    a.b = j.b; a.n = j.b.ntot; a.xl = j.xl32; a.xl32 = j.xl32; a.cell_start = j.start;
    a.fs = j.f_atm; a.unit_ew = j.unit_ew; a.unit_cnt = j.unit_cnt; a.status = j.status;
    a.work = ctas > 0 ? work : nullptr;
    a.mcap = j.mcap;
    a.gcap = P.gcap;
    a.use_d = P.use_d;
    a.acc_mode = P.acc_mode;
    a.pcap = P.pcap;
    a.lj = lj;
    a.unit_ew2 = j.unit_ew2;
    a.unit_cnt2 = j.unit_cnt2;
    a.ulist = ulist;
    a.ucount = ucount;
    a.det = j.det;
    a.pmask = atm_uses_pair_masks(j) ? j.pmask : nullptr;
    a.emax = j.emax;
    return launch_atm_fp32(j.trav, j.trunc, a, P.nwarps, P.smem, ctas, j.st);
}

bool atm_uses_pair_masks(const ForceJob& j)
{
    return j.pmask && j.prec == 1 && j.trunc == 0 && (j.trav == 1 || j.trav == 2 || j.trav == 4) &&
           j.b.ntot > 0;
}

bool atm_split_active(const ForceJob& j)
{
    return j.ncls > 1 && (j.trav == 1 || j.trav == 2 || j.trav == 4) && j.ulist && j.ucount &&
           j.b.ncell > 0;
}

static cudaError_t enqueue_atm_launches(const ForceJob& j, size_t* smem_set, bool* capacity);

cudaError_t enqueue_atm(const ForceJob& j, size_t* smem_set, bool* capacity)
{
    cudaError_t e = enqueue_atm_launches(j, smem_set, capacity);
    // deterministic block traversals left 64-bit fixed-point sums in f_atm
    if (e == cudaSuccess && j.det && (j.trav == 1 || j.trav == 2 || j.trav == 4) && j.b.ntot > 0)
        e = launch_fix_to_double(j.f_atm, 3 * j.b.ntot, j.prec == 0 ? FixBits<double>::B
                                                                   : FixBits<float>::B, j.st);
    return e;
}

static cudaError_t enqueue_atm_launches(const ForceJob& j, size_t* smem_set, bool* capacity)
{
    *capacity = false;
    {
        // every launch's plan must fit before anything is enqueued
        AtmPlan P;
        const int limit = (j.trav == 0 || j.trav == 3) ? 65535 : ATM_MCAP_LIMIT;
        if (j.mcap > limit || !atm_choose_plan(j.trav, j.trunc, j.prec, j.mcap, j.optin, P, j.det, j.gpm16)) {
            *capacity = true;
            return cudaErrorInvalidValue;
        }
    }
    cudaError_t e;
    if (j.trav != 0 && j.trav != 3 && j.b.ntot > 0) {  // owner traversals write every F_i
        e = cudaMemsetAsync(j.f_atm, 0, 3 * (size_t)j.b.ntot * sizeof(double), j.st);
        if (e != cudaSuccess) return e;
    }
    const int lj = j.lj && (j.trav == 1 || j.trav == 2 || j.trav == 4) && j.trunc == 0;
    if (lj && j.b.ntot > 0) {  // the units write LJ + ATM into f_atm
        e = cudaMemsetAsync(j.f_lj, 0, 3 * (size_t)j.b.ntot * sizeof(double), j.st);
        if (e != cudaSuccess) return e;
    }
    if (atm_uses_pair_masks(j)) {
        e = launch_pair_masks(j.b, j.start, j.xl32, j.cell_sorted, j.pmask, j.status, j.st);
        if (e != cudaSuccess) return e;
    }
    if (!atm_split_active(j)) return launch_atm_one(j, smem_set, capacity, nullptr, nullptr, j.work);
    e = launch_unit_classes(j.b, j.start, j.trav, j.ncls, j.cuts[0], j.cuts[1], j.ulist, j.ucount,
                            j.st);
    if (e != cudaSuccess) return e;
    // the small-unit class on the side stream, beside the others: its CTAs
    // fill the SMs the larger units' launch leaves idle in its tail
    const bool side = j.side_st && j.ev_fork && j.ev_join;
    if (side) {
        e = cudaEventRecord(j.ev_fork, j.st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(j.side_st, j.ev_fork, 0);
        if (e != cudaSuccess) return e;
    }
    for (int k = 0; k < j.ncls && e == cudaSuccess; k++) {
        ForceJob jk = j;
        if (side && k == 0) jk.st = j.side_st;
        if (k < j.ncls - 1) {
            jk.mcap = std::min(j.cuts[k], j.mcap);
            // small units: short phases between the CTA's barriers, so few
            // warps (64-molecule bound: 2 warps measured best on a batch of
            // 64 uneven replicas, against 1 and 4)
            if (j.cuts[k] <= 64) jk.nwarps = 2;
        }
        if (jk.mcap < 1) jk.mcap = 1;
        e = launch_atm_one(jk, smem_set, capacity, j.ulist + (size_t)k * j.b.ncell, j.ucount + k,
                           j.work ? j.work + k : nullptr);
    }
    if (side) {
        // once forked, the side stream is always joined back (a capture
        // must not end with it unjoined, and later work on st must follow
        // what was queued there); the first error is the one returned
        cudaError_t ej = cudaEventRecord(j.ev_join, j.side_st);
        if (ej == cudaSuccess) ej = cudaStreamWaitEvent(j.st, j.ev_join, 0);
        if (e == cudaSuccess) e = ej;
    }
    return e;
}

}  // namespace atm3
