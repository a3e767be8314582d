// forces.cu -- argument set-up and launch of the LJ and ATM force kernels,
// shared by the context API (capi.cu) and the allocation-free entry point.
#include <algorithm>

#include "forces.cuh"

namespace atm3 {

cudaError_t enqueue_lj(const ForceJob& j)
{
    LjArgs<double> l64{};
    LjArgs<float> l32{};
    const double rc = j.rc, sig2 = j.lj_sigma * j.lj_sigma;
    const double sc = sig2 / (rc * rc), sc3 = sc * sc * sc;
    const double ushift = j.lj_shift ? 4.0 * j.lj_eps * (sc3 * sc3 - sc3) : 0.0;
    if (j.prec == 0) {
        l64.g = j.g; l64.n = j.n; l64.xl = j.xl; l64.cell_start = j.start;
        l64.cell_sorted = j.cell_sorted; l64.fs = j.f_lj; l64.part_ew = j.lj_ew;
        l64.part_cnt = j.lj_cnt;
        for (int d = 0; d < 3; d++) {
            l64.w[d] = j.g.w[d];
            l64.wf[d] = (float)j.g.w[d];
        }
        l64.rc2 = rc * rc; l64.sig2 = sig2; l64.eps4 = 4.0 * j.lj_eps;
        l64.eps24 = 24.0 * j.lj_eps; l64.eps48 = 48.0 * j.lj_eps; l64.ushift = ushift;
        l64.xl32 = j.xl32;
        l64.p_lo = (float)(rc * rc * (1.0 - 1.0 / 4096.0));
        l64.p_hi = (float)(rc * rc * (1.0 + 1.0 / 4096.0));
    } else {
        float rcf = (float)rc;
        l32.g = j.g; l32.n = j.n; l32.xl = j.xl32; l32.cell_start = j.start;
        l32.cell_sorted = j.cell_sorted; l32.fs = j.f_lj; l32.part_ew = j.lj_ew;
        l32.part_cnt = j.lj_cnt;
        for (int d = 0; d < 3; d++) {
            l32.w[d] = (float)j.g.w[d];
            l32.wf[d] = (float)j.g.w[d];
        }
        l32.rc2 = rcf * rcf; l32.sig2 = (float)sig2; l32.eps4 = (float)(4.0 * j.lj_eps);
        l32.eps24 = (float)(24.0 * j.lj_eps); l32.eps48 = (float)(48.0 * j.lj_eps);
        l32.ushift = (float)ushift;
        l32.xl32 = j.xl32;
    }
    return launch_lj(j.prec, l64, l32, j.st);
}

cudaError_t enqueue_atm(const ForceJob& j, size_t* smem_set, bool* capacity)
{
    *capacity = false;
    AtmPlan P;
    if (j.mcap > ATM_MCAP_LIMIT || !atm_choose_plan(j.trav, j.trunc, j.prec, j.mcap, j.optin, P)) {
        *capacity = true;
        return cudaErrorInvalidValue;
    }
    cudaError_t e;
    if (!smem_set || P.smem > *smem_set) {
        e = j.prec == 0 ? atm_attr_fp64(j.trav, j.trunc, P.smem) : atm_attr_fp32(j.trav, j.trunc, P.smem);
        if (e != cudaSuccess) return e;
        if (smem_set) *smem_set = P.smem;
    }
    if (j.trav != 0 && j.n > 0) {
        e = cudaMemsetAsync(j.f_atm, 0, 3 * (size_t)j.n * sizeof(double), j.st);
        if (e != cudaSuccess) return e;
    }
    // FP32 prefilter bands of the FP64 decisions (derivation in atm_common.cuh)
    const double rc2d = j.rc * j.rc, rc6d = rc2d * rc2d * rc2d;
    const double wmax = std::max(j.g.w[0], std::max(j.g.w[1], j.g.w[2]));
    if (j.prec == 0) {
        AtmArgs<double> a{};
        a.g = j.g; a.n = j.n; a.xl = j.xl; a.xl32 = j.xl32; a.cell_start = j.start;
        a.fs = j.f_atm; a.unit_ew = j.unit_ew; a.unit_cnt = j.unit_cnt; a.status = j.status;
        for (int d = 0; d < 3; d++) {
            a.w[d] = j.g.w[d];
            a.wf[d] = (float)j.g.w[d];
        }
        a.rc2 = rc2d;
        a.rc6 = rc6d;
        a.nu = j.nu;
        a.p_lo = (float)(rc2d * (1.0 - 1.0 / 4096.0));
        a.p_hi = (float)(rc2d * (1.0 + 1.0 / 4096.0));
        a.q_lo = (float)(rc6d * (1.0 - 1.0 / 1024.0));
        a.q_hi = (float)(rc6d * (1.0 + 1.0 / 1024.0));
        a.dmin = (float)((0.02 * wmax) * (0.02 * wmax));
        a.mcap = j.mcap;
        a.gcap = P.gcap;
        a.use_d = P.use_d;
        a.acc_mode = P.acc_mode;
        return launch_atm_fp64(j.trav, j.trunc, a, P.nwarps, P.smem, j.st);
    }
    AtmArgs<float> a{};
    float rcf = (float)j.rc;
    a.g = j.g; a.n = j.n; a.xl = j.xl32; a.xl32 = j.xl32; a.cell_start = j.start;
    a.fs = j.f_atm; a.unit_ew = j.unit_ew; a.unit_cnt = j.unit_cnt; a.status = j.status;
    for (int d = 0; d < 3; d++) {
        a.w[d] = (float)j.g.w[d];
        a.wf[d] = (float)j.g.w[d];
    }
    a.rc2 = rcf * rcf;
    a.rc6 = a.rc2 * a.rc2 * a.rc2;
    a.nu = (float)j.nu;
    a.mcap = j.mcap;
    a.gcap = P.gcap;
    a.use_d = P.use_d;
    a.acc_mode = P.acc_mode;
    return launch_atm_fp32(j.trav, j.trunc, a, P.nwarps, P.smem, j.st);
}

}  // namespace atm3
