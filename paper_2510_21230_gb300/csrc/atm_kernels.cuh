// atm_kernels.cuh -- the ATM three-body unit kernel (the hot loop).
//
// One CTA processes one traversal unit (a base cell for 3c01/3c18, the 2x2x2
// block anchored at a base cell for 3c08).  The unit's cells are staged in
// shared memory; warps take "first" molecules i in turn, build i's partner
// list (pair rule: partners within r_c), enumerate the pairs {j, k} of that
// list, apply the truncation test, and push interacting triplets into a
// warp-private queue.  A full queue (32 entries) is evaluated by the whole
// warp at once, so the ATM arithmetic runs without lane divergence.
//
// Distances follow one canonical formula for every traversal (base-frame
// cell shifts, section 4): for staged molecules p, q with cell offsets o_p, o_q
// relative to the unit's base cell,
//     d = (xl_q - xl_p) + (o_q - o_p) w,     |d|^2 = (dx*dx + dy*dy) + dz*dz,
// rounded operation by operation (no contraction), so truncation decisions
// are reproducible bit for bit.
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
};
template <>
struct Ar<float> {
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float rsq(float a) { return rsqrtf(a); }
};

// truncation test (section 2): pair = every side < r_c; product = the sorted
// squared sides satisfy (p*q)*s < r_c^6
template <int TRUNC, typename R>
__device__ __forceinline__ bool keep_triplet(R a, R b, R c, R rc2, R rc6)
{
    if (TRUNC == 0) return a < rc2 && b < rc2 && c < rc2;
    R lo = a < b ? a : b, hi = a < b ? b : a;
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
    return Ar<R>::mul(Ar<R>::mul(lo, mid), hi) < rc6;
}

// ATM energy and its derivatives with respect to the squared sides, from
// Eq. atm in r^2 form: with s = abc, q = s^(-1/2), A = -a+b+c, B = a-b+c,
// C = a+b-c, P = ABC:
//   u    = nu q^3 (1 + 3/8 P q^2)
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

// running sum: plain for FP64, Neumaier-compensated for FP32
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
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v)
    {
        float t = __fadd_rn(s, v);
        if (fabsf(s) >= fabsf(v))
            c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, t), v));
        else
            c = __fadd_rn(c, __fadd_rn(__fsub_rn(v, t), s));
        s = t;
    }
    __device__ __forceinline__ double get() const { return (double)s + (double)c; }
};

// shared-memory force accumulator of one staged molecule component
template <typename R>
struct Acc;
template <>
struct Acc<double> {
    static __device__ __forceinline__ void add(unsigned char* base, int mcap, int idx, double v)
    {
        atomicAdd(reinterpret_cast<double*>(base) + idx, v);
    }
    static __device__ __forceinline__ double get(const unsigned char* base, int mcap, int idx)
    {
        return reinterpret_cast<const double*>(base)[idx];
    }
    static __device__ __forceinline__ void zero(unsigned char* base, int mcap, int idx)
    {
        reinterpret_cast<double*>(base)[idx] = 0.0;
    }
};
// FP32: hi accumulates the rounded sum, lo the exact rounding error of every
// atomic addition (two-sum of the value the atomic returned and the addend),
// i.e. compensated summation that stays correct under concurrent updates.
template <>
struct Acc<float> {
    static __device__ __forceinline__ void add(unsigned char* base, int mcap, int idx, float v)
    {
        float* hi = reinterpret_cast<float*>(base);
        float* lo = hi + 3 * mcap;
        float old = atomicAdd(hi + idx, v);
        float s = __fadd_rn(old, v);
        float bp = __fsub_rn(s, old);
        float ap = __fsub_rn(s, bp);
        float e = __fadd_rn(__fsub_rn(old, ap), __fsub_rn(v, bp));
        if (e != 0.f) atomicAdd(lo + idx, e);
    }
    static __device__ __forceinline__ double get(const unsigned char* base, int mcap, int idx)
    {
        const float* hi = reinterpret_cast<const float*>(base);
        return (double)hi[idx] + (double)hi[3 * mcap + idx];
    }
    static __device__ __forceinline__ void zero(unsigned char* base, int mcap, int idx)
    {
        float* hi = reinterpret_cast<float*>(base);
        hi[idx] = 0.f;
        hi[3 * mcap + idx] = 0.f;
    }
};

__device__ __forceinline__ unsigned long long pack3(int i, int j, int k)
{
    return (unsigned long long)i | ((unsigned long long)j << 21) | ((unsigned long long)k << 42);
}

template <int TRAV, int TRUNC, typename R>
__global__ void __launch_bounds__(256) atm_unit_kernel(const AtmArgs<R> A)
{
    constexpr int S = Trav<TRAV>::S;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_beg[S + 1];
    __shared__ int s_cell0[S];
    __shared__ signed char s_off[S][3];
    __shared__ int s_next;
    __shared__ double s_red[2][8];
    __shared__ unsigned long long s_redn[8];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = blockDim.x >> 5;
    const long long u = blockIdx.x;
    const int mcap = A.mcap;
    const AtmSmem plan = atm_smem_plan<R>(mcap, nwarps);
    R* px = reinterpret_cast<R*>(smem + plan.off_pos);
    R* py = px + mcap;
    R* pz = py + mcap;
    int* sidx = reinterpret_cast<int*>(smem + plan.off_idx);
    unsigned char* sslot = smem + plan.off_slot;
    unsigned char* acc = smem + plan.off_acc;
    unsigned short* plq = reinterpret_cast<unsigned short*>(smem + plan.off_pl_q) + warp * mcap;
    R* pla = reinterpret_cast<R*>(smem + plan.off_pl_a) + (size_t)warp * mcap;
    unsigned long long* queue =
        reinterpret_cast<unsigned long long*>(smem + plan.off_queue) + warp * plan.qcap;

    // ---- unit geometry: staged cells, their offsets and occupancies
    int cx, cy, cz;
    cell_coords(A.g, u, cx, cy, cz);
    if (warp == 0) {
        int cnt = 0;
        if (lane < S) {
            int dx, dy, dz;
            slot_offset<TRAV>(lane, dx, dy, dz);
            long long c = cell_at(A.g, cx, cy, cz, dx, dy, dz);
            int c0 = A.cell_start[c];
            cnt = A.cell_start[c + 1] - c0;
            s_cell0[lane] = c0;
            s_off[lane][0] = (signed char)dx;
            s_off[lane][1] = (signed char)dy;
            s_off[lane][2] = (signed char)dz;
        }
        int incl = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            int v = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane < S) s_beg[lane + 1] = incl;
        if (lane == 0) {
            s_beg[0] = 0;
            s_next = 0;
        }
    }
    __syncthreads();
    const int M = s_beg[S];
    const int Mfirst = (TRAV == 2) ? M : s_beg[1];
    if (M > mcap) {
        if (tid == 0) {
            atomicOr(A.status, ST_CAPACITY);
            A.unit_ew[2 * u] = 0.0;
            A.unit_ew[2 * u + 1] = 0.0;
            A.unit_cnt[2 * u] = 0ull;
            A.unit_cnt[2 * u + 1] = 0ull;
        }
        return;
    }

    // ---- stage positions (coalesced per cell) and clear the accumulators
    const long long n = A.n;
    for (int t = tid; t < M; t += blockDim.x) {
        int s = 0;
        while (s_beg[s + 1] <= t) s++;
        int g = s_cell0[s] + (t - s_beg[s]);
        px[t] = A.xl[g];
        py[t] = A.xl[n + g];
        pz[t] = A.xl[2 * n + g];
        sidx[t] = g;
        sslot[t] = (unsigned char)s;
    }
    for (int t = tid; t < M; t += blockDim.x) {
        Acc<R>::zero(acc, mcap, t);
        Acc<R>::zero(acc, mcap, mcap + t);
        Acc<R>::zero(acc, mcap, 2 * mcap + t);
    }
    __syncthreads();

    const R w0 = A.w[0], w1 = A.w[1], w2 = A.w[2];
    const R rc2 = A.rc2, rc6 = A.rc6, nu = A.nu;

    // canonical displacement p -> q and its square
    auto disp = [&](int p, int q, R& dx, R& dy, R& dz) -> R {
        int sp = sslot[p], sq = sslot[q];
        R sx = Ar<R>::mul((R)(s_off[sq][0] - s_off[sp][0]), w0);
        R sy = Ar<R>::mul((R)(s_off[sq][1] - s_off[sp][1]), w1);
        R sz = Ar<R>::mul((R)(s_off[sq][2] - s_off[sp][2]), w2);
        dx = Ar<R>::add(Ar<R>::sub(px[q], px[p]), sx);
        dy = Ar<R>::add(Ar<R>::sub(py[q], py[p]), sy);
        dz = Ar<R>::add(Ar<R>::sub(pz[q], pz[p]), sz);
        return Ar<R>::add(Ar<R>::add(Ar<R>::mul(dx, dx), Ar<R>::mul(dy, dy)), Ar<R>::mul(dz, dz));
    };

    Sum<R> esum, wsum;
    unsigned int nint = 0;
    int qn = 0;  // warp-uniform queue length
    const unsigned lt_mask = (1u << lane) - 1u;

    // evaluate one queued triplet: forces by Eq. forcepairs, W by Eq. P_3
    auto evaluate = [&](unsigned long long e) {
        int i = (int)(e & 0x1fffff), j = (int)((e >> 21) & 0x1fffff), k = (int)(e >> 42);
        R dijx, dijy, dijz, dikx, diky, dikz, djkx, djky, djkz;
        R a = disp(i, j, dijx, dijy, dijz);
        R b = disp(i, k, dikx, diky, dikz);
        R c = disp(j, k, djkx, djky, djkz);
        R uu, ua, ub, uc;
        atm_terms<R>(a, b, c, nu, uu, ua, ub, uc);
        R gij = R(2) * ua, gik = R(2) * ub, gjk = R(2) * uc;
        esum.add(uu);
        wsum.add(-(gij * a + gik * b + gjk * c));
        Acc<R>::add(acc, mcap, i, gij * dijx + gik * dikx);
        Acc<R>::add(acc, mcap, mcap + i, gij * dijy + gik * diky);
        Acc<R>::add(acc, mcap, 2 * mcap + i, gij * dijz + gik * dikz);
        if (TRAV != 0) {
            Acc<R>::add(acc, mcap, j, gjk * djkx - gij * dijx);
            Acc<R>::add(acc, mcap, mcap + j, gjk * djky - gij * dijy);
            Acc<R>::add(acc, mcap, 2 * mcap + j, gjk * djkz - gij * dijz);
            Acc<R>::add(acc, mcap, k, -(gik * dikx + gjk * djkx));
            Acc<R>::add(acc, mcap, mcap + k, -(gik * diky + gjk * djky));
            Acc<R>::add(acc, mcap, 2 * mcap + k, -(gik * dikz + gjk * djkz));
        }
    };

    auto push = [&](bool keep, int i, int j, int k) {
        unsigned m = __ballot_sync(FULL, keep);
        if (keep) queue[qn + __popc(m & lt_mask)] = pack3(i, j, k);
        qn += __popc(m);
        nint += keep ? 1u : 0u;
        __syncwarp();
        if (qn >= 32) {
            evaluate(queue[lane]);
            __syncwarp();
            if (lane < qn - 32) queue[lane] = queue[32 + lane];
            qn -= 32;
            __syncwarp();
        }
    };

    // ---- warps take first molecules i dynamically
    for (;;) {
        int i = 0;
        if (lane == 0) i = atomicAdd(&s_next, 1);
        i = __shfl_sync(FULL, i, 0);
        if (i >= Mfirst) break;
        if (TRAV == 2 && sslot[i] == 7) continue;  // no later slot completes an anchored set

        // partner list of i: later staged molecules (3c18/3c08) or all others (3c01)
        int np = 0;
        const int qlo = (TRAV == 0) ? 0 : i + 1;
        for (int q0 = qlo; q0 < M; q0 += 32) {
            int q = q0 + lane;
            bool keep = false;
            R a = R(0);
            if (q < M && (TRAV != 0 || q != i)) {
                R dx, dy, dz;
                a = disp(i, q, dx, dy, dz);
                keep = (TRUNC == 0) ? (a < rc2) : true;
            }
            unsigned m = __ballot_sync(FULL, keep);
            if (keep) {
                int pos = np + __popc(m & lt_mask);
                plq[pos] = (unsigned short)q;
                pla[pos] = a;
            }
            np += __popc(m);
        }
        __syncwarp();

        // pairs (jj < kk) of the partner list, t = kk (kk - 1) / 2 + jj
        const int T = np * (np - 1) / 2;
        const int si = sslot[i];
        for (int t0 = 0; t0 < T; t0 += 32) {
            int t = t0 + lane;
            bool keep = false;
            int j = 0, k = 0;
            if (t < T) {
                int kk = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)t)) * 0.5f);
                while (kk * (kk - 1) / 2 > t) kk--;
                while ((kk + 1) * kk / 2 <= t) kk++;
                int jj = t - kk * (kk - 1) / 2;
                j = plq[jj];
                k = plq[kk];
                bool member = (TRAV != 2) || ((si & sslot[j] & sslot[k]) == 0);
                if (member) {
                    R dx, dy, dz;
                    R c = disp(j, k, dx, dy, dz);
                    keep = keep_triplet<TRUNC, R>(pla[jj], pla[kk], c, rc2, rc6);
                }
            }
            push(keep, i, j, k);
        }
        __syncwarp();
    }
    // flush the queue
    if (lane < qn) evaluate(queue[lane]);
    __syncthreads();

    // ---- forces back to global memory (sorted order)
    if (TRAV == 0) {
        // 3c01: the base cell's molecules are owned by this unit alone
        for (int t = tid; t < Mfirst; t += blockDim.x) {
            int g = sidx[t];
            A.fs[g] = Acc<R>::get(acc, mcap, t);
            A.fs[n + g] = Acc<R>::get(acc, mcap, mcap + t);
            A.fs[2 * n + g] = Acc<R>::get(acc, mcap, 2 * mcap + t);
        }
    } else {
        for (int t = tid; t < M; t += blockDim.x) {
            int g = sidx[t];
            double fx = Acc<R>::get(acc, mcap, t);
            double fy = Acc<R>::get(acc, mcap, mcap + t);
            double fz = Acc<R>::get(acc, mcap, 2 * mcap + t);
            if (fx != 0.0) atomicAdd(A.fs + g, fx);
            if (fy != 0.0) atomicAdd(A.fs + n + g, fy);
            if (fz != 0.0) atomicAdd(A.fs + 2 * n + g, fz);
        }
    }

    // ---- unit partials: E3, W3 (FP64), interacting and candidate counts
    double e = esum.get(), w = wsum.get();
    unsigned long long ni = nint;
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
    if (tid == 0) {
        double et = 0.0, wt = 0.0;
        unsigned long long nt = 0;
        for (int q = 0; q < nwarps; q++) {
            et += s_red[0][q];
            wt += s_red[1][q];
            nt += s_redn[q];
        }
        if (TRAV == 0) {
            et /= 3.0;
            wt /= 3.0;
        }
        // candidate triplets of the unit's tasks (Eqs. celltriplet,
        // twoonetriplets, carttriplets)
        unsigned long long N[S];
        for (int s = 0; s < S; s++) N[s] = (unsigned long long)(s_beg[s + 1] - s_beg[s]);
        auto C2 = [](unsigned long long m) { return m < 2 ? 0ull : m * (m - 1) / 2; };
        auto C3 = [](unsigned long long m) { return m < 3 ? 0ull : m * (m - 1) * (m - 2) / 6; };
        unsigned long long cand = 0;
        if (TRAV == 0) {
            cand = M > 0 ? N[0] * C2((unsigned long long)M - 1) : 0ull;
        } else if (TRAV == 1) {
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
            for (int s = 0; s < 8; s++)
                for (int t = s + 1; t < 8; t++) {
                    if ((s & t) == 0) cand += N[t] * C2(N[s]) + N[s] * C2(N[t]);
                    for (int v = t + 1; v < 8; v++)
                        if ((s & t & v) == 0) cand += N[s] * N[t] * N[v];
                }
        }
        A.unit_ew[2 * u] = et;
        A.unit_ew[2 * u + 1] = wt;
        A.unit_cnt[2 * u] = cand;
        A.unit_cnt[2 * u + 1] = nt;
    }
}

template <typename R>
cudaError_t launch_atm_t(int trav, int trunc, const AtmArgs<R>& a, int nwarps, size_t smem,
                         cudaStream_t s)
{
    dim3 grid((unsigned)a.g.ncell), block(32 * nwarps);
#define ATM_LAUNCH(TV, TR)                                                        \
    if (trav == TV && trunc == TR) {                                              \
        atm_unit_kernel<TV, TR, R><<<grid, block, smem, s>>>(a);                  \
        return cudaGetLastError();                                                \
    }
    ATM_LAUNCH(0, 0)
    ATM_LAUNCH(0, 1)
    ATM_LAUNCH(1, 0)
    ATM_LAUNCH(1, 1)
    ATM_LAUNCH(2, 0)
    ATM_LAUNCH(2, 1)
#undef ATM_LAUNCH
    return cudaErrorInvalidValue;
}

template <typename R>
cudaError_t atm_attr_t(int trav, int trunc, size_t smem)
{
#define ATM_ATTR(TV, TR)                                                                 \
    if (trav == TV && trunc == TR)                                                       \
        return cudaFuncSetAttribute(atm_unit_kernel<TV, TR, R>,                          \
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    ATM_ATTR(0, 0)
    ATM_ATTR(0, 1)
    ATM_ATTR(1, 0)
    ATM_ATTR(1, 1)
    ATM_ATTR(2, 0)
    ATM_ATTR(2, 1)
#undef ATM_ATTR
    return cudaErrorInvalidValue;
}

}  // namespace atm3
