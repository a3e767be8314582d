// md_kernels.cu -- linked-cell build, LJ pair forces, velocity-Verlet update
// and the deterministic final reductions.
#include "md_kernels.cuh"

namespace atm3 {

// ---------------------------------------------------------------- linked cells

// periodic wrap into [0, L): t = x - floor(x/L) L, folded once more if the
// rounding lands outside [0, L)
__device__ __forceinline__ double wrap1(double x, double L)
{
    double t = __dsub_rn(x, __dmul_rn(floor(__ddiv_rn(x, L)), L));
    if (t < 0.0) t = __dadd_rn(t, L);
    if (t >= L) t = 0.0;
    return t;
}

// cell coordinate and clamped cell-local coordinate in [0, w]
__device__ __forceinline__ int bin1(double t, double w, int n, double& loc)
{
    int c = (int)floor(__ddiv_rn(t, w));
    c = c > n - 1 ? n - 1 : (c < 0 ? 0 : c);
    double l = __dsub_rn(t, __dmul_rn((double)c, w));
    l = l < 0.0 ? 0.0 : (l > w ? w : l);
    loc = l;
    return c;
}

// K1: wrap positions in place, cell id per molecule, cell histogram with the
// arrival rank of each molecule
__global__ void k_wrap_bin(Grid g, long long n, double* __restrict__ x, int* __restrict__ cell_of,
                           int* __restrict__ rank, int* __restrict__ count, int* __restrict__ status)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int cc[3];
    for (int d = 0; d < 3; d++) {
        double xv = x[d * n + i];
        if (!isfinite(xv)) {
            atomicOr(status, ST_NONFINITE);
            xv = 0.0;
        }
        double t = wrap1(xv, g.L[d]);
        x[d * n + i] = t;
        double loc;
        cc[d] = bin1(t, g.w[d], g.nc[d], loc);
    }
    int id = (cc[2] * g.nc[1] + cc[1]) * g.nc[0] + cc[0];
    cell_of[i] = id;
    rank[i] = atomicAdd(count + id, 1);
}

// K2: exclusive scan of the cell counts (one CTA of 1024 threads, each owns a
// contiguous chunk) and the largest occupancy
__global__ void __launch_bounds__(1024) k_scan(long long ncell, const int* __restrict__ count,
                                               int* __restrict__ start, int* __restrict__ maxocc)
{
    __shared__ int s_part[1024];
    __shared__ int s_max[32];
    const int tid = threadIdx.x;
    long long chunk = (ncell + 1023) / 1024;
    long long lo = tid * chunk, hi = lo + chunk < ncell ? lo + chunk : ncell;
    int sum = 0, mx = 0;
    for (long long c = lo; c < hi; c++) {
        int v = count[c];
        sum += v;
        mx = v > mx ? v : mx;
    }
    s_part[tid] = sum;
    for (int o = 16; o > 0; o >>= 1) {
        int v = __shfl_down_sync(0xffffffffu, mx, o);
        mx = v > mx ? v : mx;
    }
    if ((tid & 31) == 0) s_max[tid >> 5] = mx;
    __syncthreads();
    // Hillis-Steele inclusive scan over the 1024 partial sums
    for (int o = 1; o < 1024; o <<= 1) {
        int v = tid >= o ? s_part[tid - o] : 0;
        __syncthreads();
        s_part[tid] += v;
        __syncthreads();
    }
    int run = tid > 0 ? s_part[tid - 1] : 0;
    for (long long c = lo; c < hi; c++) {
        start[c] = run;
        run += count[c];
    }
    if (tid == 1023) start[ncell] = s_part[1023];
    if (tid == 0) {
        int m = 0;
        for (int q = 0; q < 32; q++) m = s_max[q] > m ? s_max[q] : m;
        *maxocc = m;
    }
}

// largest staged-molecule count of a traversal unit, per traversal:
// out[0] 3c01 (27 cells), out[1] 3c18 (base + 13 forward), out[2] 3c08 (2x2x2 block)
__global__ void k_unit_max(Grid g, const int* __restrict__ start, int* __restrict__ out)
{
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    int m01 = 0, m18 = 0, m08 = 0;
    if (c < g.ncell) {
        int cx, cy, cz;
        cell_coords(g, c, cx, cy, cz);
        for (int t = 0; t < 27; t++) {
            int dx, dy, dz;
            offset27(t, dx, dy, dz);
            long long nc = cell_at(g, cx, cy, cz, dx, dy, dz);
            int k = start[nc + 1] - start[nc];
            m01 += k;
            if (t >= 13) m18 += k;
            if (dx >= 0 && dy >= 0 && dz >= 0) m08 += k;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        m01 = max(m01, __shfl_down_sync(0xffffffffu, m01, o));
        m18 = max(m18, __shfl_down_sync(0xffffffffu, m18, o));
        m08 = max(m08, __shfl_down_sync(0xffffffffu, m08, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(out, m01);
        atomicMax(out + 1, m18);
        atomicMax(out + 2, m08);
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

// K3b: make the order inside every cell the original index order (stable sort)
__global__ void k_cell_sort(long long ncell, const int* __restrict__ start, int* __restrict__ perm)
{
    long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    int lo = start[c], hi = start[c + 1];
    for (int a = lo + 1; a < hi; a++) {
        int v = perm[a];
        int b = a - 1;
        while (b >= lo && perm[b] > v) {
            perm[b + 1] = perm[b];
            b--;
        }
        perm[b + 1] = v;
    }
}

// K3c: sorted FP64 and FP32 cell-local coordinates and the cell of each slot
__global__ void k_local(Grid g, long long n, const double* __restrict__ x,
                        const int* __restrict__ perm, double* __restrict__ xl,
                        float* __restrict__ xl32, int* __restrict__ cell_sorted)
{
    long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= n) return;
    int i = perm[s];
    int cc[3];
    for (int d = 0; d < 3; d++) {
        double loc;
        cc[d] = bin1(x[d * n + i], g.w[d], g.nc[d], loc);
        xl[d * n + s] = loc;
        xl32[d * n + s] = (float)loc;
    }
    cell_sorted[s] = (cc[2] * g.nc[1] + cc[1]) * g.nc[0] + cc[0];
}

// ---------------------------------------------------------------- LJ pairs

template <typename R>
struct LjArith;
template <>
struct LjArith<double> {
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
};
template <>
struct LjArith<float> {
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
};

// LJ (section 5) with owner-computes over the 27-cell neighbourhood: every
// molecule sums its own pair forces (no atomics, deterministic); each pair is
// seen from both ends, so the energy and virial take half per visit and the
// interacting count is visits / 2.  The candidate count is that of the
// half-shell traversal: later molecules of the own cell plus the 13 forward
// cells.
template <typename R>
__global__ void __launch_bounds__(128) k_lj_owner(const LjArgs<R> A)
{
    typedef LjArith<R> Q;
    const long long n = A.n;
    long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double e = 0.0, w = 0.0;
    unsigned long long visits = 0, cand = 0;
    if (s < n) {
        int c = A.cell_sorted[s];
        int cx, cy, cz;
        cell_coords(A.g, c, cx, cy, cz);
        R xs = A.xl[s], ys = A.xl[n + s], zs = A.xl[2 * n + s];
        R fx = 0, fy = 0, fz = 0;
        R esum = 0, wsum = 0;
        for (int t = 0; t < 27; t++) {
            int dx, dy, dz;
            offset27(t, dx, dy, dz);
            long long nc = cell_at(A.g, cx, cy, cz, dx, dy, dz);
            int q0 = A.cell_start[nc], q1 = A.cell_start[nc + 1];
            if (t > 13) cand += (unsigned long long)(q1 - q0);
            if (t == 13) cand += (unsigned long long)(q1 - 1 - s);
            R sx = Q::mul((R)dx, A.w[0]), sy = Q::mul((R)dy, A.w[1]), sz = Q::mul((R)dz, A.w[2]);
            for (int q = q0; q < q1; q++) {
                if (q == s) continue;
                if (sizeof(R) == 8) {
                    // FP32 prefilter: values outside the band decide the FP64 test
                    typedef LjArith<float> F;
                    float ex = F::add(F::sub(A.xl32[q], A.xl32[s]), F::mul((float)dx, A.wf[0]));
                    float ey = F::add(F::sub(A.xl32[n + q], A.xl32[n + s]), F::mul((float)dy, A.wf[1]));
                    float ez = F::add(F::sub(A.xl32[2 * n + q], A.xl32[2 * n + s]),
                                      F::mul((float)dz, A.wf[2]));
                    float f2 = F::add(F::add(F::mul(ex, ex), F::mul(ey, ey)), F::mul(ez, ez));
                    if (f2 > A.p_hi) continue;
                }
                R ddx = Q::add(Q::sub(A.xl[q], xs), sx);
                R ddy = Q::add(Q::sub(A.xl[n + q], ys), sy);
                R ddz = Q::add(Q::sub(A.xl[2 * n + q], zs), sz);
                R a = Q::add(Q::add(Q::mul(ddx, ddx), Q::mul(ddy, ddy)), Q::mul(ddz, ddz));
                if (!(a < A.rc2)) continue;
                visits++;
                R ia = R(1) / a;
                R s2 = A.sig2 * ia;
                R s3 = s2 * s2 * s2;
                R s6 = s3 * s3;
                R fw = (A.eps48 * s6 - A.eps24 * s3) * ia;  // F_s = -fw d
                fx -= fw * ddx;
                fy -= fw * ddy;
                fz -= fw * ddz;
                esum += A.eps4 * (s6 - s3) - A.ushift;
                wsum += fw * a;
            }
        }
        A.fs[s] = (double)fx;
        A.fs[n + s] = (double)fy;
        A.fs[2 * n + s] = (double)fz;
        e = 0.5 * (double)esum;
        w = 0.5 * (double)wsum;
    }
    // block partials
    __shared__ double s_e[4], s_w[4];
    __shared__ unsigned long long s_v[4], s_c[4];
    for (int o = 16; o > 0; o >>= 1) {
        e += __shfl_down_sync(0xffffffffu, e, o);
        w += __shfl_down_sync(0xffffffffu, w, o);
        visits += __shfl_down_sync(0xffffffffu, visits, o);
        cand += __shfl_down_sync(0xffffffffu, cand, o);
    }
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        s_e[warp] = e;
        s_w[warp] = w;
        s_v[warp] = visits;
        s_c[warp] = cand;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double et = 0, wt = 0;
        unsigned long long vt = 0, ct = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); q++) {
            et += s_e[q];
            wt += s_w[q];
            vt += s_v[q];
            ct += s_c[q];
        }
        A.part_ew[2 * blockIdx.x] = et;
        A.part_ew[2 * blockIdx.x + 1] = wt;
        A.part_cnt[2 * blockIdx.x] = ct;
        A.part_cnt[2 * blockIdx.x + 1] = vt;
    }
}


// ---------------------------------------------------------------- integrator

// v += (dt/2) F for every molecule (F = LJ + ATM in sorted order), then, if
// drift, x += dt v.  Kinetic-energy partials per block (after the kick).
__global__ void __launch_bounds__(256) k_kick(long long n, const int* __restrict__ perm,
                                              const double* __restrict__ f_lj,
                                              const double* __restrict__ f_atm,
                                              double* __restrict__ x, double* __restrict__ v,
                                              double half_dt, double dt, int drift,
                                              double* __restrict__ ke_part)
{
    long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double ke = 0.0;
    if (s < n) {
        int i = perm[s];
        for (int d = 0; d < 3; d++) {
            double f = __dadd_rn(f_lj[d * n + s], f_atm[d * n + s]);
            double vv = __dadd_rn(v[d * n + i], __dmul_rn(half_dt, f));
            v[d * n + i] = vv;
            if (drift) x[d * n + i] = __dadd_rn(x[d * n + i], __dmul_rn(dt, vv));
            ke += 0.5 * vv * vv;
        }
    }
    __shared__ double s_k[8];
    for (int o = 16; o > 0; o >>= 1) ke += __shfl_down_sync(0xffffffffu, ke, o);
    if ((threadIdx.x & 31) == 0) s_k[threadIdx.x >> 5] = ke;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); q++) t += s_k[q];
        ke_part[blockIdx.x] = t;
    }
}

// kinetic energy only (no update)
__global__ void __launch_bounds__(256) k_kinetic(long long n, const double* __restrict__ v,
                                                 double* __restrict__ ke_part)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double ke = 0.0;
    if (i < n)
        for (int d = 0; d < 3; d++) ke += 0.5 * v[d * n + i] * v[d * n + i];
    __shared__ double s_k[8];
    for (int o = 16; o > 0; o >>= 1) ke += __shfl_down_sync(0xffffffffu, ke, o);
    if ((threadIdx.x & 31) == 0) s_k[threadIdx.x >> 5] = ke;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); q++) t += s_k[q];
        ke_part[blockIdx.x] = t;
    }
}

// finiteness check of a state copied from device memory
__global__ void k_check_finite(long long m, const double* __restrict__ a, int* __restrict__ status)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < m && !isfinite(a[i])) atomicOr(status, ST_NONFINITE);
}

// ---------------------------------------------------------------- reductions

// One CTA sums every partial in a fixed order (thread-strided then a fixed
// tree), so the scalars are reproducible run to run.
__global__ void __launch_bounds__(256) k_final_reduce(ReduceArgs R)
{
    __shared__ double sd[5][256];
    __shared__ unsigned long long su[4][256];
    const int tid = threadIdx.x;
    double e3 = 0, w3 = 0, e2 = 0, w2 = 0, ke = 0;
    unsigned long long c3 = 0, i3 = 0, c2 = 0, v2 = 0;
    for (long long q = tid; q < R.n_units; q += 256) {
        e3 += R.unit_ew[2 * q];
        w3 += R.unit_ew[2 * q + 1];
        c3 += R.unit_cnt[2 * q];
        i3 += R.unit_cnt[2 * q + 1];
    }
    for (long long q = tid; q < R.n_lj; q += 256) {
        e2 += R.lj_ew[2 * q];
        w2 += R.lj_ew[2 * q + 1];
        c2 += R.lj_cnt[2 * q];
        v2 += R.lj_cnt[2 * q + 1];
    }
    for (long long q = tid; q < R.n_ke; q += 256) ke += R.ke_part[q];
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
        ResultDev* r = R.out;
        r->e2 = sd[0][0];
        r->e3 = sd[1][0];
        r->w2 = sd[2][0];
        r->w3 = sd[3][0];
        r->ekin = sd[4][0];
        r->n_cand3 = su[0][0];
        r->n_int3 = su[1][0];
        r->n_cand2 = su[2][0];
        r->n_int2 = su[3][0] / 2;
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

// ---------------------------------------------------------------- launchers

static inline unsigned nblk(long long m, int b) { return (unsigned)((m + b - 1) / b); }

cudaError_t launch_build_cells(const Grid& g, long long n, double* x, int* cell_of, int* rank,
                               int* count, int* start, int* perm, double* xl, float* xl32,
                               int* cell_sorted, int* maxocc, int* status, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int) * (size_t)g.ncell, st);
    if (e != cudaSuccess) return e;
    if (n > 0) k_wrap_bin<<<nblk(n, MD_BLOCK), MD_BLOCK, 0, st>>>(g, n, x, cell_of, rank, count, status);
    k_scan<<<1, 1024, 0, st>>>(g.ncell, count, start, maxocc);
    e = cudaMemsetAsync(maxocc + 1, 0, 3 * sizeof(int), st);
    if (e != cudaSuccess) return e;
    k_unit_max<<<nblk(g.ncell, MD_BLOCK), MD_BLOCK, 0, st>>>(g, start, maxocc + 1);
    if (n > 0) {
        k_scatter<<<nblk(n, MD_BLOCK), MD_BLOCK, 0, st>>>(n, cell_of, rank, start, perm);
        k_cell_sort<<<nblk(g.ncell, MD_BLOCK), MD_BLOCK, 0, st>>>(g.ncell, start, perm);
        k_local<<<nblk(n, MD_BLOCK), MD_BLOCK, 0, st>>>(g, n, x, perm, xl, xl32, cell_sorted);
    }
    return cudaGetLastError();
}

cudaError_t launch_lj(int prec, const LjArgs<double>& a64, const LjArgs<float>& a32,
                      cudaStream_t st)
{
    long long n = prec == 0 ? a64.n : a32.n;
    unsigned b = nblk(n > 0 ? n : 1, LJ_BLOCK);
    if (prec == 0)
        k_lj_owner<double><<<b, LJ_BLOCK, 0, st>>>(a64);
    else
        k_lj_owner<float><<<b, LJ_BLOCK, 0, st>>>(a32);
    return cudaGetLastError();
}

cudaError_t launch_kick(long long n, const int* perm, const double* f_lj, const double* f_atm,
                        double* x, double* v, double half_dt, double dt, int drift,
                        double* ke_part, cudaStream_t st)
{
    k_kick<<<nblk(n > 0 ? n : 1, MD_BLOCK), MD_BLOCK, 0, st>>>(n, perm, f_lj, f_atm, x, v, half_dt,
                                                              dt, drift, ke_part);
    return cudaGetLastError();
}

cudaError_t launch_kinetic(long long n, const double* v, double* ke_part, cudaStream_t st)
{
    k_kinetic<<<nblk(n > 0 ? n : 1, MD_BLOCK), MD_BLOCK, 0, st>>>(n, v, ke_part);
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
    k_final_reduce<<<1, 256, 0, st>>>(r);
    return cudaGetLastError();
}

cudaError_t launch_gather_forces(long long n, const int* perm, const double* f_lj,
                                 const double* f_atm, int which, double* out, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    k_gather_forces<<<nblk(n, MD_BLOCK), MD_BLOCK, 0, st>>>(n, perm, f_lj, f_atm, which, out);
    return cudaGetLastError();
}

}  // namespace atm3
