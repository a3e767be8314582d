// md_kernels.cu -- linked-cell build, LJ pair forces, velocity-Verlet update,
// density profile and the per-replica reductions (in a fixed order).
// Every kernel works on a batch of replicas (a single system is a batch of
// one): per-molecule threads look their replica up in rep_of_mol, per-cell
// threads in rep_of_cell.
#include "md_kernels.cuh"

namespace atm3 {

// ---------------------------------------------------------------- linked cells

// periodic wrap into [0, L): t = x - floor(x/L) L, folded once more if the
// rounding lands outside [0, L).  A value already in [0, L) comes back
// unchanged from those steps (x/L rounds to below 1, or to 1 and then
// x - L and (x - L) + L are exact), so it skips the division.
__device__ __forceinline__ double wrap1(double x, double L)
{
    if (x >= 0.0 && x < L) return x;
    double t = __dsub_rn(x, __dmul_rn(floor(__ddiv_rn(x, L)), L));
    if (t < 0.0) t = __dadd_rn(t, L);
    if (t >= L) t = 0.0;
    return t;
}

// cell coordinate floor(t / w) (correctly rounded quotient) and clamped
// cell-local coordinate in [0, w].  q = t * (1/w) is within 3 units of 2^-53
// |t/w| of the rounded quotient, so when no integer lies within 5 units of q
// both have the same floor and the division is skipped.
__device__ __forceinline__ int bin1(double t, double w, double iw, int n, double& loc)
{
    const double q = __dmul_rn(t, iw);
    const double fq = floor(q);
    const double tol = __dmul_rn(fabs(q), 5.551115123125783e-16);  // 5 * 2^-53
    int c;
    if (__dsub_rn(q, fq) > tol && __dsub_rn(__dadd_rn(fq, 1.0), q) > tol)
        c = (int)fq;
    else
        c = (int)floor(__ddiv_rn(t, w));
    c = c > n - 1 ? n - 1 : (c < 0 ? 0 : c);
    double l = __dsub_rn(t, __dmul_rn((double)c, w));
    l = l < 0.0 ? 0.0 : (l > w ? w : l);
    loc = l;
    return c;
}

// K1: wrap positions in place, global cell id per molecule, cell histogram
// with the arrival rank of each molecule
__global__ void k_wrap_bin(Batch B, double* __restrict__ x, int* __restrict__ cell_of,
                           int* __restrict__ rank, int* __restrict__ count, int* __restrict__ status)
{
    const long long n = B.ntot;
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Rep& rp = B.rep[B.rep_of_mol[i]];
    int cc[3];
    for (int d = 0; d < 3; d++) {
        double xv = x[d * n + i];
        if (!isfinite(xv)) {
            atomicOr(status, ST_NONFINITE);
            xv = 0.0;
        }
        double t = wrap1(xv, rp.g.L[d]);
        x[d * n + i] = t;
        double loc;
        cc[d] = bin1(t, rp.g.w[d], rp.g.iw[d], rp.g.nc[d], loc);
    }
    int id = (int)rp.cell0 + (cc[2] * rp.g.nc[1] + cc[1]) * rp.g.nc[0] + cc[0];
    cell_of[i] = id;
    rank[i] = atomicAdd(count + id, 1);
}

// K2: exclusive scan of the cell counts (one CTA of 1024 threads, each warp
// owns a contiguous segment) and the largest occupancy
__global__ void __launch_bounds__(1024) k_scan(long long ncell, const int* __restrict__ count,
                                               int* __restrict__ start, int* __restrict__ maxocc)
{
    // warp w owns the contiguous segment [w seg, (w + 1) seg) of the cells and
    // reads it 32 consecutive counts at a time (coalesced): its total and
    // largest count first, then, after a scan of the 32 totals, the exclusive
    // prefix of every cell with a shuffle scan per 32 and a running carry
    __shared__ int s_tot[32];
    __shared__ int s_max[32];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long seg = ((ncell + 31) / 32 + 31) / 32 * 32;
    const long long lo = warp * seg, hi = lo + seg < ncell ? lo + seg : ncell;
    int tot = 0, mx = 0;
    for (long long c0 = lo; c0 < hi; c0 += 32) {
        const long long c = c0 + lane;
        const int v = c < hi ? count[c] : 0;
        tot += __reduce_add_sync(FULL, v);
        mx = max(mx, (int)__reduce_max_sync(FULL, (unsigned)v));
    }
    if (lane == 0) {
        s_tot[warp] = tot;
        s_max[warp] = mx;
    }
    __syncthreads();
    if (warp == 0) {
        const int t = s_tot[lane];
        int incl = t;
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += u;
        }
        s_tot[lane] = incl - t;  // exclusive: the cells before warp lane's segment
        const int m = (int)__reduce_max_sync(FULL, (unsigned)s_max[lane]);
        if (lane == 0) *maxocc = m;
        if (lane == 31) start[ncell] = incl;
    }
    __syncthreads();
    int carry = s_tot[warp];
    for (long long c0 = lo; c0 < hi; c0 += 32) {
        const long long c = c0 + lane;
        const int v = c < hi ? count[c] : 0;
        int incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += u;
        }
        if (c < hi) start[c] = carry + incl - v;
        carry += __shfl_sync(FULL, incl, 31);
    }
}

// largest staged-molecule count of a traversal unit, per traversal:
// out[0] 3c01 (27 cells), out[1] 3c18 (base + 13 forward), out[2] 3c08 (2x2x2 block)
__global__ void k_unit_max(Batch B, const int* __restrict__ start, int wide, int* __restrict__ out)
{
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    int m01 = 0, m18 = 0, m08 = 0, mw = 0;
    if (c < B.ncell) {
        const Rep& rp = B.rep[B.rep_of_cell[c]];
        const int* st = start + rp.cell0;
        int cx, cy, cz;
        cell_coords(rp.g, c - rp.cell0, cx, cy, cz);
        for (int t = 0; t < 27; t++) {
            int dx, dy, dz;
            offset27(t, dx, dy, dz);
            long long nc = cell_at(rp.g, cx, cy, cz, dx, dy, dz);
            int k = st[nc + 1] - st[nc];
            m01 += k;
            if (t >= 13) m18 += k;
            if (dx >= 0 && dy >= 0 && dz >= 0) m08 += k;
        }
        // the wide traversal's 5^3 neighbourhood (only when that traversal is in use)
        for (int t = 0; t < (wide ? 125 : 0); t++) {
            long long nc = cell_at(rp.g, cx, cy, cz, t % 5 - 2, (t / 5) % 5 - 2, t / 25 - 2);
            mw += st[nc + 1] - st[nc];
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        m01 = max(m01, __shfl_down_sync(0xffffffffu, m01, o));
        m18 = max(m18, __shfl_down_sync(0xffffffffu, m18, o));
        m08 = max(m08, __shfl_down_sync(0xffffffffu, m08, o));
        mw = max(mw, __shfl_down_sync(0xffffffffu, mw, o));
    }
    // block maximum first: one global atomic per value and block
    __shared__ int s_m[4][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) {
        s_m[0][warp] = m01;
        s_m[1][warp] = m18;
        s_m[2][warp] = m08;
        s_m[3][warp] = mw;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        int m = 0;
        for (int w = 0; w < nw; w++) m = max(m, s_m[threadIdx.x][w]);
        atomicMax(out + threadIdx.x, m);
        // the corner-anchored 3c08 stages the same blocks as 3c08
        if (threadIdx.x == 2) atomicMax(out + 4, m);
    }
}

// Unit size classes of the block traversals: unit u (its base cell) holds
// the molecules of its 8 cells (3c08, corner-anchored 3c08) or 14 cells
// (3c18); it goes to the first class whose bound holds them (cut0, then cut1
// when there are three classes; the last class takes the rest).  Class k is
// listed in ulist[k * ncell ..] and counted in counts[k] (zero at launch).
__global__ void k_unit_classes(Batch B, const int* __restrict__ start, int trav, int ncls,
                               int cut0, int cut1, int* __restrict__ ulist,
                               int* __restrict__ counts)
{
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    int cls = -1;
    if (c < B.ncell) {
        const Rep& rp = B.rep[B.rep_of_cell[c]];
        const int* st = start + rp.cell0;
        int cx, cy, cz;
        cell_coords(rp.g, c - rp.cell0, cx, cy, cz);
        int m = 0;
        for (int t = 0; t < 27; t++) {
            int dx, dy, dz;
            offset27(t, dx, dy, dz);
            if (trav == 1 ? t >= 13 : (dx >= 0 && dy >= 0 && dz >= 0)) {
                const long long nc = cell_at(rp.g, cx, cy, cz, dx, dy, dz);
                m += st[nc + 1] - st[nc];
            }
        }
        cls = m <= cut0 ? 0 : ((ncls > 2 && m <= cut1) ? 1 : ncls - 1);
    }
    // one append per class and warp
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    for (int k = 0; k < ncls; k++) {
        const unsigned mk = __ballot_sync(FULL, cls == k);
        if (mk == 0u) continue;
        const int lead = __ffs(mk) - 1;
        int base = 0;
        if (lane == lead) base = atomicAdd(counts + k, __popc(mk));
        base = __shfl_sync(FULL, base, lead);
        if (cls == k) ulist[k * B.ncell + base + __popc(mk & ((1u << lane) - 1u))] = (int)c;
    }
}

// K3a: scatter by arrival rank
__global__ void k_scatter(long long n, const int* __restrict__ cell_of, const int* __restrict__ rank,
                          const int* __restrict__ start, int* __restrict__ perm)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    perm[start[cell_of[i]] + rank[i]] = (int)i;
}

// K3b+c: one warp per cell restores the original index order inside the cell
// (the rank of each entry among the cell's entries; lane 0 insertion-sorts a
// cell of more than 32) and writes, for every sorted slot, the FP64 and FP32
// cell-local coordinates (t - c w clamped to [0, w], the cell's own c: the
// binning's arithmetic without its division) and the slot's global cell
__global__ void __launch_bounds__(128) k_cell_order(Batch B, const double* __restrict__ x,
                                                    const int* __restrict__ start,
                                                    int* __restrict__ perm, double* __restrict__ xl,
                                                    float* __restrict__ xl32,
                                                    int* __restrict__ cell_sorted)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const long long c = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (c >= B.ncell) return;  // whole warps leave together
    const long long n = B.ntot;
    const int lo = start[c], hi = start[c + 1], cnt = hi - lo;
    if (cnt <= 32) {
        const int v = lane < cnt ? perm[lo + lane] : 0x7fffffff;
        int r = 0;
        for (int k = 0; k < cnt; k++) r += __shfl_sync(FULL, v, k) < v ? 1 : 0;
        __syncwarp();  // every entry is read before any is overwritten
        if (lane < cnt) perm[lo + r] = v;
    } else {
        if (lane == 0)
            for (int a = lo + 1; a < hi; a++) {
                const int v = perm[a];
                int b = a - 1;
                while (b >= lo && perm[b] > v) {
                    perm[b + 1] = perm[b];
                    b--;
                }
                perm[b + 1] = v;
            }
    }
    __syncwarp();
    const Rep& rp = B.rep[B.rep_of_cell[c]];
    int cc[3];
    cell_coords(rp.g, c - rp.cell0, cc[0], cc[1], cc[2]);
    for (int s = lo + lane; s < hi; s += 32) {
        const int i = perm[s];
        for (int d = 0; d < 3; d++) {
            const double w = rp.g.w[d];
            double l = __dsub_rn(x[d * n + i], __dmul_rn((double)cc[d], w));
            l = l < 0.0 ? 0.0 : (l > w ? w : l);
            xl[d * n + s] = l;
            xl32[d * n + s] = (float)l;
        }
        cell_sorted[s] = (int)c;
    }
}

// ---------------------------------------------------------------- LJ pairs

template <typename R>
struct LjArith;
template <>
struct LjArith<double> {
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double rcp(double a) { return __drcp_rn(a); }
};
template <>
struct LjArith<float> {
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float rcp(float a) { return __frcp_rn(a); }
};

// LJ (section 5) with owner-computes over the 27-cell neighbourhood: every
// molecule sums its own pair forces (no atomics, deterministic); each pair is
// seen from both ends, so the energy and virial take half per visit.  The
// candidate and interacting counts are those of the half-shell traversal:
// later molecules of the own cell plus the 13 forward cells, so every pair
// is counted once, by one of its molecules (also when the two belong to
// different domains).
template <typename R>
__global__ void __launch_bounds__(128) k_lj_owner(const LjArgs<R> A)
{
    typedef LjArith<R> Q;
    const long long n = A.n;
    long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int cg = A.cell_sorted[s];
    const Rep& rp = A.b.rep[A.b.rep_of_cell[cg]];
    const int* st = A.cell_start + rp.cell0;
    int cx, cy, cz;
    cell_coords(rp.g, cg - rp.cell0, cx, cy, cz);
    if (cz < rp.own_z0 || cz >= rp.own_z1) {
        // another domain's molecule: no pair terms here
        A.fs[s] = 0.0;
        A.fs[n + s] = 0.0;
        A.fs[2 * n + s] = 0.0;
        A.mol_ew[2 * s] = 0.0;
        A.mol_ew[2 * s + 1] = 0.0;
        A.mol_cnt[2 * s] = 0u;
        A.mol_cnt[2 * s + 1] = 0u;
        return;
    }
    const bool f64 = sizeof(R) == 8;
    const R w0 = (R)rp.g.w[0], w1 = (R)rp.g.w[1], w2 = (R)rp.g.w[2];
    const R rc2 = f64 ? (R)rp.rc2 : (R)rp.rc2f;
    const R sig2 = f64 ? (R)rp.sig2 : (R)rp.sig2f;
    const R eps4 = f64 ? (R)rp.eps4 : (R)rp.eps4f;
    const R eps24 = f64 ? (R)rp.eps24 : (R)rp.eps24f;
    const R eps48 = f64 ? (R)rp.eps48 : (R)rp.eps48f;
    const R ushift = f64 ? (R)rp.ushift : (R)rp.ushiftf;
    R xs = A.xl[s], ys = A.xl[n + s], zs = A.xl[2 * n + s];
    R fx = 0, fy = 0, fz = 0;
    R esum = 0, wsum = 0;
    unsigned pairs = 0, cand = 0;
    for (int t = 0; t < 27; t++) {
        int dx, dy, dz;
        offset27(t, dx, dy, dz);
        long long nc = cell_at(rp.g, cx, cy, cz, dx, dy, dz);
        int q0 = st[nc], q1 = st[nc + 1];
        if (t > 13) cand += (unsigned)(q1 - q0);
        if (t == 13) cand += (unsigned)(q1 - 1 - s);
        R sx = Q::mul((R)dx, w0), sy = Q::mul((R)dy, w1), sz = Q::mul((R)dz, w2);
        for (int q = q0; q < q1; q++) {
            if (q == s) continue;
            if (f64) {
                // FP32 prefilter: a value above the band decides the FP64 test
                typedef LjArith<float> F;
                float ex = F::add(F::sub(A.xl32[q], A.xl32[s]), F::mul((float)dx, rp.wf[0]));
                float ey = F::add(F::sub(A.xl32[n + q], A.xl32[n + s]), F::mul((float)dy, rp.wf[1]));
                float ez = F::add(F::sub(A.xl32[2 * n + q], A.xl32[2 * n + s]),
                                  F::mul((float)dz, rp.wf[2]));
                float f2 = F::add(F::add(F::mul(ex, ex), F::mul(ey, ey)), F::mul(ez, ez));
                if (f2 > rp.p_hi) continue;
            }
            R ddx = Q::add(Q::sub(A.xl[q], xs), sx);
            R ddy = Q::add(Q::sub(A.xl[n + q], ys), sy);
            R ddz = Q::add(Q::sub(A.xl[2 * n + q], zs), sz);
            R a = Q::add(Q::add(Q::mul(ddx, ddx), Q::mul(ddy, ddy)), Q::mul(ddz, ddz));
            if (!(a < rc2)) continue;
            if (t > 13 || (t == 13 && q > s)) pairs++;
            R ia = Q::rcp(a);  // correctly rounded: the same value as 1 / a
            R s2 = sig2 * ia;
            R s3 = s2 * s2 * s2;
            R s6 = s3 * s3;
            R fw = (eps48 * s6 - eps24 * s3) * ia;  // F_s = -fw d
            fx -= fw * ddx;
            fy -= fw * ddy;
            fz -= fw * ddz;
            esum += eps4 * (s6 - s3) - ushift;
            wsum += fw * a;
        }
    }
    A.fs[s] = (double)fx;
    A.fs[n + s] = (double)fy;
    A.fs[2 * n + s] = (double)fz;
    A.mol_ew[2 * s] = 0.5 * (double)esum;
    A.mol_ew[2 * s + 1] = 0.5 * (double)wsum;
    A.mol_cnt[2 * s] = cand;
    A.mol_cnt[2 * s + 1] = pairs;
}

// ---------------------------------------------------------------- integrator

// v += (dt/2) F for every molecule (F = LJ + ATM in sorted order), then, if
// drift, x += dt v; kinetic energy per molecule (after the kick)
__global__ void __launch_bounds__(256) k_kick(Batch B, const int* __restrict__ perm,
                                              const double* __restrict__ f_lj,
                                              const double* __restrict__ f_atm,
                                              double* __restrict__ x, double* __restrict__ v,
                                              int drift, double* __restrict__ ke)
{
    const long long n = B.ntot;
    long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= n) return;
    int i = perm[s];
    const Rep& rp = B.rep[B.rep_of_mol[i]];
    const double dt = rp.dt, half_dt = 0.5 * rp.dt;
    double k = 0.0;
    for (int d = 0; d < 3; d++) {
        double f = __dadd_rn(f_lj[d * n + s], f_atm[d * n + s]);
        double vv = __dadd_rn(v[d * n + i], __dmul_rn(half_dt, f));
        v[d * n + i] = vv;
        if (drift) x[d * n + i] = __dadd_rn(x[d * n + i], __dmul_rn(dt, vv));
        k += 0.5 * vv * vv;
    }
    ke[i] = k;
}

// the first half kick and the drift from a total force given in the
// original molecule order (a state restored with its forces)
__global__ void __launch_bounds__(256) k_kick_orig(Batch B, const double* __restrict__ f,
                                                   double* __restrict__ x, double* __restrict__ v,
                                                   double* __restrict__ ke)
{
    const long long n = B.ntot;
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Rep& rp = B.rep[B.rep_of_mol[i]];
    const double dt = rp.dt, half_dt = 0.5 * rp.dt;
    double k = 0.0;
    for (int d = 0; d < 3; d++) {
        double vv = __dadd_rn(v[d * n + i], __dmul_rn(half_dt, f[d * n + i]));
        v[d * n + i] = vv;
        x[d * n + i] = __dadd_rn(x[d * n + i], __dmul_rn(dt, vv));
        k += 0.5 * vv * vv;
    }
    ke[i] = k;
}

// kinetic energy per molecule only (no update)
__global__ void __launch_bounds__(256) k_kinetic(long long n, const double* __restrict__ v,
                                                 double* __restrict__ ke)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double k = 0.0;
    for (int d = 0; d < 3; d++) k += 0.5 * v[d * n + i] * v[d * n + i];
    ke[i] = k;
}

// velocity rescaling thermostat: every velocity of replica r times
// lambda_r = sqrt(T_r (3 N_r - 3) / (2 K_r)) (K_r from the last reduction;
// unchanged when K_r = 0 or N_r < 2), kinetic energies times lambda_r^2
__global__ void __launch_bounds__(256) k_rescale(Batch B, double* __restrict__ v,
                                                 double* __restrict__ ke,
                                                 const ResultDev* __restrict__ res,
                                                 const double* __restrict__ t_target)
{
    const long long n = B.ntot;
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int r = B.rep_of_mol[i];
    const double k = res[r].ekin, dof = 3.0 * (double)B.rep[r].n - 3.0;
    if (!(k > 0.0) || !(dof > 0.0)) return;
    const double l2 = t_target[r] * dof / (2.0 * k), l = sqrt(l2);
    for (int d = 0; d < 3; d++) v[d * n + i] *= l;
    ke[i] *= l2;
}

// finiteness check of a state copied from device memory
__global__ void k_check_finite(long long m, const double* __restrict__ a, int* __restrict__ status)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < m && !isfinite(a[i])) atomicOr(status, ST_NONFINITE);
}

// density profile: histogram of one coordinate of the wrapped positions
__global__ void k_density(Batch B, const double* __restrict__ x, int axis, int nbins,
                          unsigned long long* __restrict__ counts)
{
    const long long n = B.ntot;
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int r = B.rep_of_mol[i];
    const double h = B.rep[r].g.L[axis] / (double)nbins;
    int b = (int)floor(x[axis * n + i] / h);
    b = b < 0 ? 0 : (b >= nbins ? nbins - 1 : b);
    atomicAdd(counts + (long long)r * nbins + b, 1ull);
}

// radial distribution: every pair once (forward half shell of the 27 cells,
// later molecules of the own cell) with r < r_max, binned by floor(r / dr) in
// FP64 on the canonical displacement; per-CTA shared histogram of the CTA's
// first replica (molecules of a second replica go straight to global memory)
__global__ void __launch_bounds__(128) k_rdf(Batch B, const double* __restrict__ xl,
                                             const int* __restrict__ start,
                                             const int* __restrict__ cell_sorted, double rmax,
                                             int nbins, unsigned long long* __restrict__ counts)
{
    extern __shared__ unsigned hist[];
    typedef LjArith<double> Q;
    for (int k = threadIdx.x; k < nbins; k += blockDim.x) hist[k] = 0u;
    __syncthreads();
    const long long n = B.ntot;
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int r0 = B.rep_of_cell[cell_sorted[blockIdx.x * (long long)blockDim.x]];
    if (s < n) {
        const int cg = cell_sorted[s];
        const int rep = B.rep_of_cell[cg];
        const Rep& rp = B.rep[rep];
        const int* st = start + rp.cell0;
        int cx, cy, cz;
        cell_coords(rp.g, cg - rp.cell0, cx, cy, cz);
        const double dr = rmax / (double)nbins, rmax2 = rmax * rmax;
        const double xs = xl[s], ys = xl[n + s], zs = xl[2 * n + s];
        for (int t = 13; t < 27; t++) {
            int dx, dy, dz;
            offset27(t, dx, dy, dz);
            const long long nc = cell_at(rp.g, cx, cy, cz, dx, dy, dz);
            const int q1 = st[nc + 1];
            const int q0 = t == 13 ? (int)s + 1 : st[nc];
            const double sx = Q::mul((double)dx, rp.g.w[0]), sy = Q::mul((double)dy, rp.g.w[1]),
                         sz = Q::mul((double)dz, rp.g.w[2]);
            for (int q = q0; q < q1; q++) {
                const double ex = Q::add(Q::sub(xl[q], xs), sx);
                const double ey = Q::add(Q::sub(xl[n + q], ys), sy);
                const double ez = Q::add(Q::sub(xl[2 * n + q], zs), sz);
                const double r2 = Q::add(Q::add(Q::mul(ex, ex), Q::mul(ey, ey)), Q::mul(ez, ez));
                if (!(r2 < rmax2)) continue;
                int b = (int)(sqrt(r2) / dr);
                b = b >= nbins ? nbins - 1 : b;
                if (rep == r0) atomicAdd(hist + b, 1u);
                else atomicAdd(counts + (long long)rep * nbins + b, 1ull);
            }
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nbins; k += blockDim.x)
        if (hist[k]) atomicAdd(counts + (long long)r0 * nbins + k, (unsigned long long)hist[k]);
}

// ---------------------------------------------------------------- reductions

// Two-level reduction in a fixed order (the same sums for the same partials).  Level 1: CTA
// (r, k) sums the k-th of REDUCE_PARTS equal slices of replica r's units and
// molecules (thread-strided, then a fixed tree).  Level 2: one warp per
// replica adds the REDUCE_PARTS partial sums in a fixed tree.
__global__ void __launch_bounds__(256) k_partial_reduce(ReduceArgs R)
{
    __shared__ double sd[5][256];
    __shared__ unsigned long long su[4][256];
    const int tid = threadIdx.x;
    const int r = blockIdx.x / REDUCE_PARTS, k = blockIdx.x % REDUCE_PARTS;
    const Rep& rp = R.b.rep[r];
    const long long cu = (rp.g.ncell + REDUCE_PARTS - 1) / REDUCE_PARTS;
    const long long cm = (rp.n + REDUCE_PARTS - 1) / REDUCE_PARTS;
    const long long u0 = rp.cell0 + k * cu, u1 = min(rp.cell0 + rp.g.ncell, u0 + cu);
    const long long m0 = rp.mol0 + k * cm, m1 = min(rp.mol0 + rp.n, m0 + cm);
    double e3 = 0, w3 = 0, e2 = 0, w2 = 0, ke = 0;
    unsigned long long c3 = 0, i3 = 0, c2 = 0, v2 = 0;
    for (long long q = u0 + tid; q < u1; q += 256) {
        e3 += R.unit_ew[2 * q];
        w3 += R.unit_ew[2 * q + 1];
        c3 += R.unit_cnt[2 * q];
        i3 += R.unit_cnt[2 * q + 1];
        if (R.unit_ew2) {
            e2 += R.unit_ew2[2 * q];
            w2 += R.unit_ew2[2 * q + 1];
            c2 += R.unit_cnt2[2 * q];
            v2 += R.unit_cnt2[2 * q + 1];
        }
    }
    for (long long q = m0 + tid; q < m1; q += 256) {
        if (!R.unit_ew2) {
            e2 += R.mol_ew[2 * q];
            w2 += R.mol_ew[2 * q + 1];
            c2 += R.mol_cnt[2 * q];
            v2 += R.mol_cnt[2 * q + 1];
        }
        ke += R.ke[q];
    }
    sd[0][tid] = e2; sd[1][tid] = e3; sd[2][tid] = w2; sd[3][tid] = w3; sd[4][tid] = ke;
    su[0][tid] = c3; su[1][tid] = i3; su[2][tid] = c2; su[3][tid] = v2;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (tid < o) {
            for (int k = 0; k < 5; k++) sd[k][tid] += sd[k][tid + o];
            for (int k = 0; k < 4; k++) su[k][tid] += su[k][tid + o];
        }
        __syncthreads();
    }
    if (tid == 0) {
        ResultDev* p = R.part + blockIdx.x;
        p->e2 = sd[0][0];
        p->e3 = sd[1][0];
        p->w2 = sd[2][0];
        p->w3 = sd[3][0];
        p->ekin = sd[4][0];
        p->n_cand3 = su[0][0];
        p->n_int3 = su[1][0];
        p->n_cand2 = su[2][0];
        p->n_int2 = su[3][0];
    }
}

// one warp per replica: lane k holds partials k and k + 32 (added in that
// order), then a fixed shuffle tree; the order is the same for every launch
__global__ void __launch_bounds__(128) k_final_reduce(ReduceArgs R)
{
    static_assert(REDUCE_PARTS == 64, "two partials per lane");
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= R.b.R) return;  // whole warps leave together
    const ResultDev& a = R.part[r * REDUCE_PARTS + lane];
    const ResultDev& b = R.part[r * REDUCE_PARTS + 32 + lane];
    double e2 = a.e2 + b.e2, e3 = a.e3 + b.e3, w2 = a.w2 + b.w2, w3 = a.w3 + b.w3;
    double ek = a.ekin + b.ekin;
    unsigned long long c3 = a.n_cand3 + b.n_cand3, i3 = a.n_int3 + b.n_int3;
    unsigned long long c2 = a.n_cand2 + b.n_cand2, i2 = a.n_int2 + b.n_int2;
    for (int o = 16; o > 0; o >>= 1) {
        e2 += __shfl_down_sync(FULL, e2, o);
        e3 += __shfl_down_sync(FULL, e3, o);
        w2 += __shfl_down_sync(FULL, w2, o);
        w3 += __shfl_down_sync(FULL, w3, o);
        ek += __shfl_down_sync(FULL, ek, o);
        c3 += __shfl_down_sync(FULL, c3, o);
        i3 += __shfl_down_sync(FULL, i3, o);
        c2 += __shfl_down_sync(FULL, c2, o);
        i2 += __shfl_down_sync(FULL, i2, o);
    }
    if (lane == 0) {
        ResultDev t;
        t.e2 = e2;
        t.e3 = e3;
        t.w2 = w2;
        t.w3 = w3;
        t.ekin = ek;
        t.n_cand3 = c3;
        t.n_int3 = i3;
        t.n_cand2 = c2;
        t.n_int2 = i2;
        R.out[r] = t;
    }
}

// gather sorted-order forces to the original order: which 0 total, 1 LJ, 2 ATM
__global__ void k_gather_forces(long long n, const int* __restrict__ perm,
                                const double* __restrict__ f_lj, const double* __restrict__ f_atm,
                                int which, double* __restrict__ out)
{
    long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= n) return;
    int i = perm[s];
    for (int d = 0; d < 3; d++) {
        double a = which == 2 ? 0.0 : f_lj[d * n + s];
        double b = which == 1 ? 0.0 : f_atm[d * n + s];
        out[d * n + i] = which == 0 ? __dadd_rn(a, b) : (which == 1 ? a : b);
    }
}

// the deterministic mode's force sums: 64-bit integers in units of 2^-bits,
// read and rewritten in place as doubles (the value is rounded once)
__global__ void k_fix_to_double(double* __restrict__ f, long long m, double scale)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= m) return;
    const long long v = reinterpret_cast<const long long*>(f)[i];
    f[i] = (double)v * scale;
}

// ---------------------------------------------------------------- launchers

static inline unsigned nblk(long long m, int b) { return (unsigned)((m + b - 1) / b); }

cudaError_t launch_build_cells(const Batch& b, double* x, int* cell_of, int* rank, int* count,
                               int* start, int* perm, double* xl, float* xl32, int* cell_sorted,
                               int* maxocc, int* status, bool wide, cudaStream_t st)
{
    const long long n = b.ntot;
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int) * (size_t)b.ncell, st);
    if (e != cudaSuccess) return e;
    if (n > 0) k_wrap_bin<<<nblk(n, MD_BLOCK), MD_BLOCK, 0, st>>>(b, x, cell_of, rank, count, status);
    k_scan<<<1, 1024, 0, st>>>(b.ncell, count, start, maxocc);
    e = cudaMemsetAsync(maxocc + 1, 0, ATM_NTRAV * sizeof(int), st);
    if (e != cudaSuccess) return e;
    k_unit_max<<<nblk(b.ncell, MD_BLOCK), MD_BLOCK, 0, st>>>(b, start, wide ? 1 : 0, maxocc + 1);
    if (n > 0) {
        k_scatter<<<nblk(n, MD_BLOCK), MD_BLOCK, 0, st>>>(n, cell_of, rank, start, perm);
        k_cell_order<<<(unsigned)((b.ncell + 3) / 4), 128, 0, st>>>(b, x, start, perm, xl, xl32,
                                                                  cell_sorted);
    }
    return cudaGetLastError();
}

cudaError_t launch_unit_classes(const Batch& b, const int* start, int trav, int ncls, int cut0,
                                int cut1, int* ulist, int* counts, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(counts, 0, ncls * sizeof(int), st);
    if (e != cudaSuccess || b.ncell <= 0) return e;
    k_unit_classes<<<nblk(b.ncell, MD_BLOCK), MD_BLOCK, 0, st>>>(b, start, trav, ncls, cut0, cut1,
                                                                  ulist, counts);
    return cudaGetLastError();
}

cudaError_t launch_lj(int prec, const LjArgs<double>& a64, const LjArgs<float>& a32,
                      cudaStream_t st)
{
    long long n = prec == 0 ? a64.n : a32.n;
    if (n <= 0) return cudaSuccess;
    if (prec == 0)
        k_lj_owner<double><<<nblk(n, LJ_BLOCK), LJ_BLOCK, 0, st>>>(a64);
    else
        k_lj_owner<float><<<nblk(n, LJ_BLOCK), LJ_BLOCK, 0, st>>>(a32);
    return cudaGetLastError();
}

cudaError_t launch_kick(const Batch& b, const int* perm, const double* f_lj, const double* f_atm,
                        double* x, double* v, int drift, double* ke, cudaStream_t st)
{
    if (b.ntot <= 0) return cudaSuccess;
    k_kick<<<nblk(b.ntot, MD_BLOCK), MD_BLOCK, 0, st>>>(b, perm, f_lj, f_atm, x, v, drift, ke);
    return cudaGetLastError();
}

cudaError_t launch_kick_orig(const Batch& b, const double* f, double* x, double* v, double* ke,
                             cudaStream_t st)
{
    if (b.ntot <= 0) return cudaSuccess;
    k_kick_orig<<<nblk(b.ntot, MD_BLOCK), MD_BLOCK, 0, st>>>(b, f, x, v, ke);
    return cudaGetLastError();
}

cudaError_t launch_rescale(const Batch& b, double* v, double* ke, const ResultDev* res,
                           const double* t_target, cudaStream_t st)
{
    if (b.ntot <= 0) return cudaSuccess;
    k_rescale<<<nblk(b.ntot, MD_BLOCK), MD_BLOCK, 0, st>>>(b, v, ke, res, t_target);
    return cudaGetLastError();
}

cudaError_t launch_kinetic(long long n, const double* v, double* ke, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_kinetic<<<nblk(n, MD_BLOCK), MD_BLOCK, 0, st>>>(n, v, ke);
    return cudaGetLastError();
}

cudaError_t launch_check_finite(long long m, const double* a, int* status, cudaStream_t st)
{
    if (m <= 0) return cudaSuccess;
    k_check_finite<<<nblk(m, MD_BLOCK), MD_BLOCK, 0, st>>>(m, a, status);
    return cudaGetLastError();
}

cudaError_t launch_final_reduce(const ReduceArgs& r, cudaStream_t st)
{
    k_partial_reduce<<<(unsigned)(r.b.R * REDUCE_PARTS), 256, 0, st>>>(r);
    k_final_reduce<<<(unsigned)((r.b.R + 3) / 4), 128, 0, st>>>(r);
    return cudaGetLastError();
}

cudaError_t launch_gather_forces(long long n, const int* perm, const double* f_lj,
                                 const double* f_atm, int which, double* out, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_gather_forces<<<nblk(n, MD_BLOCK), MD_BLOCK, 0, st>>>(n, perm, f_lj, f_atm, which, out);
    return cudaGetLastError();
}

cudaError_t launch_rdf(const Batch& b, const double* xl, const int* start, const int* cell_sorted,
                       double rmax, int nbins, unsigned long long* counts, cudaStream_t st)
{
    if (b.ntot <= 0) return cudaSuccess;
    k_rdf<<<nblk(b.ntot, 128), 128, (size_t)nbins * sizeof(unsigned), st>>>(b, xl, start, cell_sorted,
                                                                           rmax, nbins, counts);
    return cudaGetLastError();
}

cudaError_t launch_density(const Batch& b, const double* x, int axis, int nbins,
                           unsigned long long* counts, cudaStream_t st)
{
    if (b.ntot <= 0) return cudaSuccess;
    k_density<<<nblk(b.ntot, MD_BLOCK), MD_BLOCK, 0, st>>>(b, x, axis, nbins, counts);
    return cudaGetLastError();
}

cudaError_t launch_fix_to_double(double* f, long long m, int bits, cudaStream_t st)
{
    if (m <= 0) return cudaSuccess;
    k_fix_to_double<<<nblk(m, MD_BLOCK), MD_BLOCK, 0, st>>>(f, m, 1.0 / (double)(1ull << bits));
    return cudaGetLastError();
}

}  // namespace atm3
