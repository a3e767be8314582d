// atm_common.cuh -- arithmetic shared by the ATM triplet kernels.
//
// Distances follow one canonical formula for every traversal (base-frame
// cell shifts, section 4): for staged molecules p, q with cell offsets o_p, o_q
// relative to the unit's base cell,
//     d = (xl_q - xl_p) + (o_q - o_p) w,     |d|^2 = (dx*dx + dy*dy) + dz*dz,
// rounded operation by operation (no contraction), so truncation decisions
// are reproducible bit for bit.
//
// FP64 decisions through an FP32 prefilter.  A squared distance computed in
// FP32 on FP32-rounded cell-local coordinates differs from the FP64 one by at
// most  2 delta (|dx|+|dy|+|dz|) + 3 delta^2 + 4 u D  with u = 2^-24 and
// delta = 8 u w_max (two input roundings, the rounded shift, the subtraction
// and the addition).  Near the cutoff (D ~ r_c^2, w <= 4/3 r_c) that is below
// 2.5e-6 D, so an FP32 value outside [r_c^2 (1 - 2^-12), r_c^2 (1 + 2^-12)]
// already decides the FP64 comparison; only values inside the band are
// recomputed in FP64.  For the product rule each factor D >= (0.02 w_max)^2
// has relative error below 8.3e-5, the product below 2.5e-4 < 2^-10, so an
// FP32 product outside r_c^6 (1 -+ 2^-10) decides; smaller sides or values in
// the band are recomputed in FP64.
#pragma once
#include "atm3_internal.cuh"

namespace atm3 {

template <typename R>
struct Ar;
template <>
struct Ar<double> {
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double rsq(double a) { return ::rsqrt(a); }
    static __device__ __forceinline__ double rcp(double a) { return __drcp_rn(a); }
};
template <>
struct Ar<float> {
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float rsq(float a) { return rsqrtf(a); }
    static __device__ __forceinline__ float rcp(float a) { return __frcp_rn(a); }
};

// canonical displacement p -> q (offset difference m in cells) and its square
template <typename R>
__device__ __forceinline__ R canon_disp(R xp, R yp, R zp, R xq, R yq, R zq, int mx, int my, int mz,
                                        R w0, R w1, R w2, R& dx, R& dy, R& dz)
{
    typedef Ar<R> Q;
    dx = Q::add(Q::sub(xq, xp), Q::mul((R)mx, w0));
    dy = Q::add(Q::sub(yq, yp), Q::mul((R)my, w1));
    dz = Q::add(Q::sub(zq, zp), Q::mul((R)mz, w2));
    return Q::add(Q::add(Q::mul(dx, dx), Q::mul(dy, dy)), Q::mul(dz, dz));
}

// sorted product (lo * mid) * hi of three squared sides
template <typename R>
__device__ __forceinline__ R sorted_product(R a, R b, R c)
{
    R lo = fmin(a, b), hi = fmax(a, b);
    R mid;
    if (c < lo) {
        mid = lo;
        lo = c;
    } else if (c < hi) {
        mid = c;
    } else {
        mid = hi;
        hi = c;
    }
    return Ar<R>::mul(Ar<R>::mul(lo, mid), hi);
}

// truncation test (section 2): pair = every side < r_c; product = the sorted
// squared sides satisfy (p*q)*s < r_c^6
template <int TRUNC, typename R>
__device__ __forceinline__ bool keep_triplet(R a, R b, R c, R rc2, R rc6)
{
    if (TRUNC == 0) return a < rc2 && b < rc2 && c < rc2;
    return sorted_product<R>(a, b, c) < rc6;
}

// ATM energy and its derivatives with respect to the squared sides, from
// Eq. atm in r^2 form: with s = abc, q = s^(-1/2), A = -a+b+c, B = a-b+c,
// C = a+b-c, P = ABC:
//   u     = nu q^3 (1 + 3/8 P q^2)
//   du/da = nu q^5 (3/8 (2aA - BC) - bc (3/2 + 15/16 P q^2))   (and cyclic)
// One reciprocal square root, no division.
template <typename R>
__device__ __forceinline__ void atm_terms(R a, R b, R c, R nu, R& u, R& ua, R& ub, R& uc)
{
    R s = a * b * c;
    R q = Ar<R>::rsq(s);
    R q2 = q * q;
    R q3 = q2 * q;
    R q5 = q3 * q2;
    R A = (b + c) - a;
    R B = (a + c) - b;
    R C = (a + b) - c;
    R P = A * B * C;
    R Pq2 = P * q2;
    u = nu * q3 * (R(1) + R(0.375) * Pq2);
    R K = R(1.5) + R(0.9375) * Pq2;
    R nq5 = nu * q5;
    ua = nq5 * (R(0.375) * (R(2) * a * A - B * C) - K * (b * c));
    ub = nq5 * (R(0.375) * (R(2) * b * B - A * C) - K * (a * c));
    uc = nq5 * (R(0.375) * (R(2) * c * C - A * B) - K * (a * b));
}

// Deterministic mode: v as a term in units of 2^-B (B = FixBits<R>::B),
// rounded to nearest; a term of size 2^(FIX_LIMIT - B) or more, or not
// finite, sets ST_RANGE and counts as zero.  The scaling by a power of two
// is exact, so a term is rounded once.
template <typename R>
__device__ __forceinline__ unsigned long long to_fix(double v, int* status)
{
    const double x = v * (double)(1ull << FixBits<R>::B);
    if (!(fabs(x) < (double)(1ull << FIX_LIMIT))) {
        atomicOr(status, ST_RANGE);
        return 0ull;
    }
    return (unsigned long long)__double2ll_rn(x);
}

// to_fix of a term in working precision: the FP32 path stays in FP32 (the
// scaling by 2^32 is exact there too, so the integer is the same) and keeps
// the hot loops off the slow FP64 pipe
template <typename R>
__device__ __forceinline__ unsigned long long to_fix_w(R v, int* status)
{
    if constexpr (sizeof(R) == 8) {
        return to_fix<R>(v, status);
    } else {
        const float x = v * (float)(1ull << FixBits<R>::B);
        if (!(fabsf(x) < (float)(1ull << FIX_LIMIT))) {
            atomicOr(status, ST_RANGE);
            return 0ull;
        }
        return (unsigned long long)__float2ll_rn(x);
    }
}

// a fixed-point sum back in working precision (FP32: the integer rounded to
// FP32 once, then scaled exactly)
template <typename R>
__device__ __forceinline__ R from_fix(long long v)
{
    if constexpr (sizeof(R) == 8)
        return (R)((double)v * (1.0 / (double)(1ull << FixBits<R>::B)));
    else
        return (float)v * (1.0f / (float)(1ull << FixBits<R>::B));
}

// running sum: plain for FP64, Kahan-compensated for FP32
template <typename R>
struct Sum;
template <>
struct Sum<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double v) { s += v; }
    __device__ __forceinline__ double get() const { return s; }
};
template <>
struct Sum<float> {
    // Kahan: c carries the rounding error of the last addition, the sum is s - c
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v)
    {
        float y = __fsub_rn(v, c);
        float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ double get() const { return (double)s - (double)c; }
};

// Candidate triplets of one unit's cell tasks (Eqs. celltriplet,
// twoonetriplets, carttriplets) from the staged slot occupancies N[0..S).
template <int TRAV, int S>
__device__ inline unsigned long long unit_candidates(const int* beg)
{
    unsigned long long N[S];
    for (int s = 0; s < S; s++) N[s] = (unsigned long long)(beg[s + 1] - beg[s]);
    auto C2 = [](unsigned long long m) { return m < 2 ? 0ull : m * (m - 1) / 2; };
    auto C3 = [](unsigned long long m) { return m < 3 ? 0ull : m * (m - 1) * (m - 2) / 6; };
    unsigned long long cand = 0;
    if (TRAV == 0) {
        unsigned long long M = (unsigned long long)beg[S];
        cand = M > 0 ? N[0] * C2(M - 1) : 0ull;
    } else if (TRAV == 1 || TRAV == 4) {
        // every task holds the base cell (slot 0): <b>, <b, s>, <b, s, t>
        unsigned long long sum1 = 0, sum2 = 0;
        cand = C3(N[0]);
        for (int s = 1; s < S; s++) {
            cand += N[s] * C2(N[0]) + N[0] * C2(N[s]);
            sum2 += N[s] * sum1;
            sum1 += N[s];
        }
        cand += N[0] * sum2;
    } else {
        cand = C3(N[0]);
        for (int s = 0; s < S; s++)
            for (int t = s + 1; t < S; t++) {
                if ((s & t) == 0) cand += N[t] * C2(N[s]) + N[s] * C2(N[t]);
                for (int v = t + 1; v < S; v++)
                    if ((s & t & v) == 0) cand += N[s] * N[t] * N[v];
            }
    }
    return cand;
}

// The same count for the block traversals (3c18, 3c08, corner-anchored 3c08),
// spread over the lanes of one warp (every lane calls; lane 0 gets the total).
template <int TRAV, int S>
__device__ inline unsigned long long unit_candidates_warp(const int* beg)
{
    static_assert(S <= 32, "one slot per lane");
    const int lane = threadIdx.x & 31;
    auto Nn = [&](int s) { return (unsigned long long)(beg[s + 1] - beg[s]); };
    auto C2 = [](unsigned long long m) { return m < 2 ? 0ull : m * (m - 1) / 2; };
    auto C3 = [](unsigned long long m) { return m < 3 ? 0ull : m * (m - 1) * (m - 2) / 6; };
    unsigned long long cand = 0;
    if (lane < S) {
        const int s = lane;
        const unsigned long long Ns = Nn(s);
        if (TRAV == 2) {
            // lane s: the tasks whose first slot is s
            if (s == 0) cand += C3(Ns);
            for (int t = s + 1; t < S; t++) {
                const unsigned long long Nt = Nn(t);
                if ((s & t) == 0) cand += Nt * C2(Ns) + Ns * C2(Nt);
                for (int v = t + 1; v < S; v++)
                    if ((s & t & v) == 0) cand += Ns * Nt * Nn(v);
            }
        } else {
            // every task holds slot 0: lane s > 0 takes <0, s> and <0, s, t > s>
            const unsigned long long N0 = Nn(0);
            if (s == 0) {
                cand = C3(N0);
            } else {
                unsigned long long later = 0;
                for (int t = s + 1; t < S; t++) later += Nn(t);
                cand = Ns * C2(N0) + N0 * C2(Ns) + N0 * Ns * later;
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) cand += __shfl_down_sync(0xffffffffu, cand, o);
    return cand;
}

// Candidate pairs of a unit's own 2-body share: 3c08 / corner-anchored 3c08,
// the c08 traversal in one 2x2x2 block -- the anchor cell's own pairs and the
// pairs of every two slots whose bounding box starts at the anchor (13 slot
// pairs); 3c18, the base cell's half-shell -- its own pairs and its pairs
// with the 13 forward cells.  Summed over all units either is the half-shell
// count.  Lane 0 of the calling warp gets the total.
template <int TRAV, int S>
__device__ inline unsigned long long unit_pair_candidates_warp(const int* beg)
{
    const int lane = threadIdx.x & 31;
    unsigned long long c = 0;
    if (lane < S) {
        const unsigned long long Ns = (unsigned long long)(beg[lane + 1] - beg[lane]);
        if (lane == 0) c = Ns < 2 ? 0ull : Ns * (Ns - 1) / 2;
        for (int t = lane + 1; t < S; t++)
            if (TRAV == 1 ? lane == 0 : (lane & t) == 0)
                c += Ns * (unsigned long long)(beg[t + 1] - beg[t]);
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    return c;
}

// unit geometry: per-slot cell start, occupancy prefix and offsets (warp 0)
template <int TRAV, int S>
__device__ __forceinline__ void unit_slots(const Grid& g, const int* cell_start, long long u,
                                          int* s_beg, int* s_cell0, signed char (*s_off)[3])
{
    const unsigned FULL = 0xffffffffu;
    int lane = threadIdx.x & 31;
    int cx, cy, cz;
    cell_coords(g, u, cx, cy, cz);
    int run = 0;  // staged molecules of the slots before this chunk of 32
    for (int s0 = 0; s0 < S; s0 += 32) {
        const int s = s0 + lane;
        int cnt = 0;
        if (s < S) {
            int dx, dy, dz;
            slot_offset<TRAV>(s, dx, dy, dz);
            long long c = cell_at(g, cx, cy, cz, dx, dy, dz);
            int c0 = cell_start[c];
            cnt = cell_start[c + 1] - c0;
            s_cell0[s] = c0;
            s_off[s][0] = (signed char)dx;
            s_off[s][1] = (signed char)dy;
            s_off[s][2] = (signed char)dz;
        }
        int incl = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            int v = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += v;
        }
        if (s < S) s_beg[s + 1] = run + incl;
        run += __shfl_sync(FULL, incl, 31);
    }
    if (lane == 0) s_beg[0] = 0;
}

// block-wide reduction of the unit partials and their store (thread 0 writes)
// the fused LJ sums of a unit (E2, W2 doubles, pair count) to unit_ew2 /
// unit_cnt2; every thread calls, thread 0 writes
template <int NWMAX>
__device__ __forceinline__ void unit_reduce_store2(double e, double w, unsigned long long np,
                                                   unsigned long long cand, double* unit_ew2,
                                                   unsigned long long* unit_cnt2, long long u,
                                                   double (*s_red)[NWMAX],
                                                   unsigned long long* s_redn)
{
    const unsigned FULL = 0xffffffffu;
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        e += __shfl_down_sync(FULL, e, o);
        w += __shfl_down_sync(FULL, w, o);
        np += __shfl_down_sync(FULL, np, o);
    }
    __syncthreads();  // the slots are free (a previous reduction may still read them)
    if (lane == 0) {
        s_red[0][warp] = e;
        s_red[1][warp] = w;
        s_redn[warp] = np;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double et = 0.0, wt = 0.0;
        unsigned long long nt = 0;
        for (int q = 0; q < nw; q++) {
            et += s_red[0][q];
            wt += s_red[1][q];
            nt += s_redn[q];
        }
        unit_ew2[2 * u] = et;
        unit_ew2[2 * u + 1] = wt;
        unit_cnt2[2 * u] = cand;
        unit_cnt2[2 * u + 1] = nt;
    }
}

template <int NWMAX>
__device__ __forceinline__ void unit_reduce_store(double e, double w, unsigned long long ni,
                                                  double scale, unsigned long long cand,
                                                  double* unit_ew, unsigned long long* unit_cnt,
                                                  long long u, double (*s_red)[NWMAX],
                                                  unsigned long long* s_redn)
{
    const unsigned FULL = 0xffffffffu;
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        e += __shfl_down_sync(FULL, e, o);
        w += __shfl_down_sync(FULL, w, o);
        ni += __shfl_down_sync(FULL, ni, o);
    }
    if (lane == 0) {
        s_red[0][warp] = e;
        s_red[1][warp] = w;
        s_redn[warp] = ni;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double et = 0.0, wt = 0.0;
        unsigned long long nt = 0;
        for (int q = 0; q < nw; q++) {
            et += s_red[0][q];
            wt += s_red[1][q];
            nt += s_redn[q];
        }
        unit_ew[2 * u] = et * scale;
        unit_ew[2 * u + 1] = wt * scale;
        unit_cnt[2 * u] = cand;
        unit_cnt[2 * u + 1] = nt;
    }
}

}  // namespace atm3
