// atm_block.cuh -- Newton-3 traversals 3c18 and 3c08 (section 4).
//
// One CTA per unit: the base cell with its 13 forward neighbours (3c18) or
// the 2x2x2 block anchored at the base cell (3c08, and TRAV 4, the
// corner-anchored 3c08 whose tasks all hold the base cell: the 3c18 procedure
// over the block's 7 other cells).  The unit's M molecules
// are staged in shared memory in slot order, so a triplet p < q < r of staged
// indices lists its cells in the order the traversal's tasks do.  Each staged
// molecule carries its exact base-frame shift o*w, so the canonical
// displacement (xl_q - xl_p) + (o_q - o_p) w needs no slot lookups.  FP32
// pair rule: once the pairs are decided, the shift rows are replaced by the
// rounded unit-frame positions xl + o w, so the triplet evaluation and the
// gather take one difference per component (the decisions stay canonical).
//
// Pair rule
//  1. Upper-triangular bitmask adjacency adj[p] = {q > p : |d(p,q)| < r_c}
//     (one ballot per 32 pairs) and its transpose.
//  2. Edges are numbered row by row (row offsets and per-word prefix
//     popcounts) and listed as (p, q); FP64 also tabulates their vectors.
//  3. A warp takes 32 edges (p, q) at a time.  The triangles of an edge are
//     the set bits r > q of adj[p] & adj[q] & (slots allowed as third member):
//     counted per lane (3c18: per word, packed in bytes), prefix-summed over
//     the warp and expanded 32 per round, so every pair test is shared by all
//     the triplets that contain the pair and every lane of a round evaluates
//     one triangle.
// Product rule
//  1. Dense FP32 squared distances (or on-the-fly when they do not fit).
//  3. Every candidate p < q < r of the unit's tasks, enumerated q-major, is
//     tested on the sorted product of its squared sides; interacting triplets
//     are queued per warp and evaluated 32 at a time.
// Both rules
//  4. Evaluation: one reciprocal square root, no division.  By Eq. forcepairs
//     a triplet's forces are three pair terms g_e d_e along its sides, so it
//     adds three scalars to per-pair accumulators G_e (product rule: runs of
//     equal pairs in a batch are first summed with a segmented warp reduction).
//  5. Every molecule sums F_m = sum_e G_e d(m -> other end) over its pairs in
//     one thread and adds the unit's share to the global FP64 force with one
//     atomic per component.
// When a unit has more edges than the edge table holds, or the dense pair
// table does not fit, the unit falls back to per-molecule shared-memory force
// accumulators (compensated atomics in FP32).
#pragma once
#include <type_traits>

#include "atm_common.cuh"

namespace atm3 {

__device__ __forceinline__ int tri_index(int x, int y) { return y * (y - 1) / 2 + x; }  // x < y

// position of the set bit of K with nth set bits below it (0 <= nth < popc(K)),
// by halving the word: the same five steps for every lane
__device__ __forceinline__ int nth_bit(unsigned K, int nth)
{
    int pos = 0, c;
    c = __popc(K & 0xffffu); if (nth >= c) { nth -= c; K >>= 16; pos += 16; }
    c = __popc(K & 0xffu);   if (nth >= c) { nth -= c; K >>= 8;  pos += 8; }
    c = __popc(K & 0xfu);    if (nth >= c) { nth -= c; K >>= 4;  pos += 4; }
    c = __popc(K & 0x3u);    if (nth >= c) { nth -= c; K >>= 2;  pos += 2; }
    if (nth >= (int)(K & 1u)) pos += 1;
    return pos;
}

// per-molecule force accumulators in shared memory (fallback mode)
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
// FP32: hi holds the rounded sum, lo the exact rounding error of every atomic
// addition (two-sum of the value the atomic returned and the addend)
template <>
struct Acc<float> {
    static __device__ __forceinline__ void add(unsigned char* base, int mcap, int idx, float v)
    {
        float* hi = reinterpret_cast<float*>(base);
        float old = atomicAdd(hi + idx, v);
        float s = __fadd_rn(old, v);
        float bp = __fsub_rn(s, old);
        float ap = __fsub_rn(s, bp);
        float e = __fadd_rn(__fsub_rn(old, ap), __fsub_rn(v, bp));
        if (e != 0.f) atomicAdd(hi + 3 * mcap + idx, e);
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

// sum of v over the contiguous run of lanes that share key, delivered to the
// run's first lane (the return value is meaningful there only)
template <typename R>
__device__ __forceinline__ R seg_sum(R v, int key, int lane)
{
    const unsigned FULL = 0xffffffffu;
    for (int o = 1; o < 32; o <<= 1) {
        R t = __shfl_down_sync(FULL, v, o);
        int tk = __shfl_down_sync(FULL, key, o);
        if (lane + o < 32 && tk == key) v += t;
    }
    return v;
}

template <int TRAV, int TRUNC, typename R, bool DET>
__device__ __forceinline__ void atm_block_unit(const AtmArgs<R>& A, const long long u)
{
    constexpr int S = Trav<TRAV>::S;
    constexpr bool F64 = sizeof(R) == 8;
    constexpr bool PAIR = TRUNC == 0;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_beg[S + 1];
    __shared__ int s_cell0[S];
    __shared__ signed char s_off[S][3];
    __shared__ int s_next, s_edges;
    constexpr int NWB = TRUNC == 1 && TRAV == 1 ? 16 : 8;  // most warps of a CTA
    __shared__ double s_red[2][NWB];
    __shared__ unsigned long long s_redn[NWB];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = blockDim.x >> 5;
    const int mcap = A.mcap;
    const BlockSmem plan =
        block_smem_plan<R>(TRUNC, mcap, nwarps, A.gcap, A.use_d, A.acc_mode, DET ? 1 : 0);
    // the replica this unit belongs to and the unit's index inside it
    const Rep& rp = A.b.rep[A.b.rep_of_cell[u]];
    const long long lu = u - rp.cell0;
    const int W = plan.W;
    R* px = reinterpret_cast<R*>(smem + plan.off_pos);
    R* py = px + mcap;
    R* pz = py + mcap;
    R* shx = reinterpret_cast<R*>(smem + plan.off_sh);
    R* shy = shx + mcap;
    R* shz = shy + mcap;
    // FP64 path: FP32 copies for the prefilter (SoA); FP32 path: float4 rows
    float* fx32 = reinterpret_cast<float*>(smem + plan.off_pos32);
    float* fy32 = fx32 + mcap;
    float* fz32 = fy32 + mcap;
    float* sx32 = reinterpret_cast<float*>(smem + plan.off_sh32);
    float* sy32 = sx32 + mcap;
    float* sz32 = sy32 + mcap;
    float4* P4 = reinterpret_cast<float4*>(smem + plan.off_pos);
    float4* S4 = reinterpret_cast<float4*>(smem + plan.off_sh);  // FP32 pair rule: the shifted rows after the decisions
    int* sidx = reinterpret_cast<int*>(smem + plan.off_idx);  // FP64; FP32: P4[t].w
    unsigned char* sslot = smem + plan.off_slot;
    unsigned* adj = reinterpret_cast<unsigned*>(smem + plan.off_adj);
    unsigned* adjT = reinterpret_cast<unsigned*>(smem + plan.off_adjT);
    unsigned short* rowpre = reinterpret_cast<unsigned short*>(smem + plan.off_rowpre);
    int* rowoff = reinterpret_cast<int*>(smem + plan.off_rowoff);
    unsigned* memb = reinterpret_cast<unsigned*>(smem + plan.off_memb);
    R* ED = reinterpret_cast<R*>(smem + plan.off_ed);                // FP64: edge vectors
    unsigned* el = reinterpret_cast<unsigned*>(smem + plan.off_el);  // edge list p | q << 16
    // pair scalars: R, or (deterministic mode) 64-bit fixed point
    using GT = std::conditional_t<DET, long long, R>;
    GT* G = reinterpret_cast<GT*>(smem + plan.off_G);
    float* D = reinterpret_cast<float*>(smem + plan.off_D);
    unsigned char* acc = smem + plan.off_acc;
    unsigned long long* queue =
        reinterpret_cast<unsigned long long*>(smem + plan.off_queue) + warp * 64;

    if (!unit_owned(rp, lu)) {
        // another domain's unit: no forces, zero sums
        if (tid == 0) {
            A.unit_ew[2 * u] = 0.0;
            A.unit_ew[2 * u + 1] = 0.0;
            A.unit_cnt[2 * u] = 0ull;
            A.unit_cnt[2 * u + 1] = 0ull;
            if (PAIR && (TRAV == 1 || TRAV == 2 || TRAV == 4) && A.lj) {
                A.unit_ew2[2 * u] = 0.0;
                A.unit_ew2[2 * u + 1] = 0.0;
                A.unit_cnt2[2 * u] = 0ull;
                A.unit_cnt2[2 * u + 1] = 0ull;
            }
        }
        return;
    }
    if (warp == 0) unit_slots<TRAV, S>(rp.g, A.cell_start + rp.cell0, lu, s_beg, s_cell0, s_off);
    if (tid == 0) s_next = 0;
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
            if (PAIR && (TRAV == 1 || TRAV == 2 || TRAV == 4) && A.lj) {
                A.unit_ew2[2 * u] = 0.0;
                A.unit_ew2[2 * u + 1] = 0.0;
                A.unit_cnt2[2 * u] = 0ull;
                A.unit_cnt2[2 * u + 1] = 0ull;
            }
        }
        return;
    }
    const int Wm = (M + 31) >> 5;
    const long long n = A.n;
    const R w0 = (R)rp.g.w[0], w1 = (R)rp.g.w[1], w2 = (R)rp.g.w[2];
    const float wf0 = rp.wf[0], wf1 = rp.wf[1], wf2 = rp.wf[2];
    const R rc2 = F64 ? (R)rp.rc2 : (R)rp.rc2f;
    const R rc6 = F64 ? (R)rp.rc6 : (R)rp.rc6f;
    const R nu = F64 ? (R)rp.nu : (R)rp.nuf;
    const unsigned lt_mask = (1u << lane) - 1u;
    // LJ of the unit's own cell pairs (pair rule in a step): 3c08 and the
    // corner-anchored 3c08 the c08 cell pairs (the pair's cells anchored at
    // the unit), 3c18 the pairs with a molecule in the base cell (the
    // half-shell of the base cell); the LJ kernel's arithmetic on the same
    // canonical displacement
    const bool LJ = PAIR && (TRAV == 1 || TRAV == 2 || TRAV == 4) && A.lj != 0;
    // p < q in staging order, so a pair with a base-cell molecule has it at p
    auto lj_own = [&](int p, int q) -> bool {
        return TRAV == 1 ? sslot[p] == 0 : (sslot[p] & sslot[q]) == 0;
    };
    const R sig2 = F64 ? (R)rp.sig2 : (R)rp.sig2f;
    const R eps4 = F64 ? (R)rp.eps4 : (R)rp.eps4f;
    const R eps24 = F64 ? (R)rp.eps24 : (R)rp.eps24f;
    const R eps48 = F64 ? (R)rp.eps48 : (R)rp.eps48f;
    const R ushift = F64 ? (R)rp.ushift : (R)rp.ushiftf;
    Sum<R> e2sum, w2sum;
    unsigned n2 = 0;
    // LJ pair scalar of squared distance a (F_p = G d(p -> q)); adds E2, W2
    auto lj_pair = [&](R a) -> R {
        const R ia = Ar<R>::rcp(a);
        const R s2 = sig2 * ia;
        const R s3 = s2 * s2 * s2;
        const R s6 = s3 * s3;
        const R fw = (eps48 * s6 - eps24 * s3) * ia;
        e2sum.add(eps4 * (s6 - s3) - ushift);
        w2sum.add(fw * a);
        n2++;
        return -fw;
    };

    // pair-scalar and per-molecule accumulation: floating-point atomics, or
    // (deterministic mode) integer atomics on fixed-point terms, whose sums
    // do not depend on the order of the additions
    auto gadd = [&](int idx, R v) {
        if constexpr (DET)
            atomicAdd(reinterpret_cast<unsigned long long*>(G + idx), to_fix_w<R>(v, A.status));
        else
            atomicAdd(G + idx, v);
    };
    auto gset = [&](int idx, R v) {
        if constexpr (DET)
            G[idx] = (GT)to_fix_w<R>(v, A.status);
        else
            G[idx] = v;
    };
    auto gget = [&](int idx) -> R {
        if constexpr (DET)
            return from_fix<R>(G[idx]);
        else
            return G[idx];
    };
    auto acc_add = [&](int idx, R v) {
        if constexpr (DET)
            atomicAdd(reinterpret_cast<unsigned long long*>(acc) + idx, to_fix_w<R>(v, A.status));
        else
            Acc<R>::add(acc, mcap, idx, v);
    };
    auto acc_get = [&](int idx) -> double {
        if constexpr (DET)
            return (double)from_fix<R>(reinterpret_cast<const long long*>(acc)[idx]);
        else
            return Acc<R>::get(acc, mcap, idx);
    };
    auto acc_zero = [&](int idx) {
        if constexpr (DET)
            reinterpret_cast<long long*>(acc)[idx] = 0ll;
        else
            Acc<R>::zero(acc, mcap, idx);
    };

    // ---- stage the unit: positions and exact shifts o * w
    for (int t = tid; t < M; t += blockDim.x) {
        int s = 0;
        while (s_beg[s + 1] <= t) s++;
        int g = s_cell0[s] + (t - s_beg[s]);
        if (!F64) {
            // (w: the molecule's sorted index)
            P4[t] = make_float4((float)A.xl[g], (float)A.xl[n + g], (float)A.xl[2 * n + g],
                                __int_as_float(g));
            S4[t] = make_float4((float)s_off[s][0] * wf0, (float)s_off[s][1] * wf1,
                                (float)s_off[s][2] * wf2, 0.0f);
        } else {
            px[t] = A.xl[g];
            py[t] = A.xl[n + g];
            pz[t] = A.xl[2 * n + g];
            shx[t] = (R)s_off[s][0] * w0;
            shy[t] = (R)s_off[s][1] * w1;
            shz[t] = (R)s_off[s][2] * w2;
            fx32[t] = A.xl32[g];
            fy32[t] = A.xl32[n + g];
            fz32[t] = A.xl32[2 * n + g];
            sx32[t] = (float)s_off[s][0] * wf0;
            sy32[t] = (float)s_off[s][1] * wf1;
            sz32[t] = (float)s_off[s][2] * wf2;
        }
        if (F64) sidx[t] = g;
        sslot[t] = (unsigned char)s;
    }
    const bool dense_g = !PAIR && A.acc_mode == 0;
    if (dense_g)
        for (int t = tid; t < M * (M - 1) / 2; t += blockDim.x) G[t] = GT(0);
    if (!PAIR && A.acc_mode == 1)
        for (int t = tid; t < M; t += blockDim.x) {
            acc_zero(t);
            acc_zero(mcap + t);
            acc_zero(2 * mcap + t);
        }
    if (PAIR)
        for (int t = tid; t < M * W; t += blockDim.x) {
            adjT[t] = 0u;
            adj[t] = 0u;
            rowpre[t] = 0;
        }
    __syncthreads();

    // canonical displacement p -> q, working precision and FP32
    auto disp = [&](int p, int q, R& dx, R& dy, R& dz) -> R {
        typedef Ar<R> Q;
        if constexpr (!F64) {
            const float4 a = P4[q], b = P4[p], sa = S4[q], sb = S4[p];
            dx = Q::add(Q::sub(a.x, b.x), Q::sub(sa.x, sb.x));
            dy = Q::add(Q::sub(a.y, b.y), Q::sub(sa.y, sb.y));
            dz = Q::add(Q::sub(a.z, b.z), Q::sub(sa.z, sb.z));
        } else {
            dx = Q::add(Q::sub(px[q], px[p]), Q::sub(shx[q], shx[p]));
            dy = Q::add(Q::sub(py[q], py[p]), Q::sub(shy[q], shy[p]));
            dz = Q::add(Q::sub(pz[q], pz[p]), Q::sub(shz[q], shz[p]));
        }
        return Q::add(Q::add(Q::mul(dx, dx), Q::mul(dy, dy)), Q::mul(dz, dz));
    };
    auto disp32 = [&](int p, int q) -> float {
        typedef Ar<float> Q;
        if constexpr (!F64) {
            R dx, dy, dz;
            return disp(p, q, dx, dy, dz);
        } else {
            float dx = Q::add(Q::sub(fx32[q], fx32[p]), Q::sub(sx32[q], sx32[p]));
            float dy = Q::add(Q::sub(fy32[q], fy32[p]), Q::sub(sy32[q], sy32[p]));
            float dz = Q::add(Q::sub(fz32[q], fz32[p]), Q::sub(sz32[q], sz32[p]));
            return Q::add(Q::add(Q::mul(dx, dx), Q::mul(dy, dy)), Q::mul(dz, dz));
        }
    };
    // pair-rule decision |d(p,q)| < r_c (FP64 through the FP32 prefilter)
    auto close = [&](int p, int q) -> bool {
        R dx, dy, dz;
        if (!F64) return disp(p, q, dx, dy, dz) < rc2;
        float f2 = disp32(p, q);
        if (f2 < rp.p_lo) return true;
        if (f2 > rp.p_hi) return false;
        return disp(p, q, dx, dy, dz) < rc2;
    };
    // product rule: D[dsel(x) + y] is the FP32 squared distance of x < y (the
    // upper triangle packed row by row; row x starts at x M - x (x + 1) / 2)
    auto dsel = [&](int x) -> int { return x * M - ((x * (x + 1)) >> 1) - x - 1; };
    // rank of y among the set bits of row x = edge number of (x, y) within row x
    auto rank = [&](int x, int y) -> int {
        int wy = y >> 5;
        return rowpre[x * W + wy] + __popc(adj[x * W + wy] & ((1u << (y & 31)) - 1u));
    };

    // ends (p, q) of edge e from the row offsets and the adjacency: p = the
    // last row with rowoff[p] <= e, q = the (e - rowoff[p])-th set bit of row
    // p (the word by a scan, then its bit once)
    auto locate_edge = [&](int e, int& p, int& q) {
        int lo = 0, hi = M - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (rowoff[mid] <= e) lo = mid; else hi = mid - 1;
        }
        p = lo;
        int j = e - rowoff[p];
        int wsel = p >> 5;
        unsigned Ksel = 0u;
        for (int w = p >> 5; w < Wm; w++) {
            const unsigned word = adj[p * W + w];
            const int c = __popc(word);
            if (j < c) {
                wsel = w;
                Ksel = word;
                break;
            }
            j -= c;
        }
        q = (wsel << 5) + nth_bit(Ksel, j);
    };

    // ---- 1. pair decisions
    if (PAIR) {
        // row p of the adjacency, its per-word prefix popcounts and its edge
        // count (kept in rowoff[p + 1] until the row offsets are formed).
        // FP32: one thread per row builds the row's words in a register while
        // the warp walks the columns together (the column's staged row is a
        // broadcast load).  FP64: one warp per row, one ballot per 32 pairs
        // (the rare FP64 recomputations of the prefilter band stay spread
        // over the lanes).
        if (!F64 && A.pmask) {
            // from the evaluation's pair bitmaps (k_pair_masks): word k - 13 of
            // a molecule covers the molecules of the cell at offset27(k), k =
            // 13 (its own cell, the later molecules) .. 26 (the forward
            // cells), in cell order, which is the staging order.  Slot s2
            // lies at offset o(s2) - o(sp) from p's slot, and a later slot is
            // a forward cell in both unit kinds (3c08: s = ox + 2 oy + 4 oz;
            // 3c18: forward neighbours in lexicographic order), so row p of
            // adj comes from p's own words.  Cells two apart (a 3c18 unit's
            // outer slots) hold no pair within r_c: the host hands over
            // bitmaps only when fl(w^2) >= the FP32 r_c^2 on every axis.
            for (int p = tid; p < M; p += blockDim.x) {
                const int sp = sslot[p];
                const long long gp = __float_as_int(P4[p].w);
                unsigned* rowa = adj + p * W;
                unsigned wd[S];  // the row's words first: independent loads in flight
#pragma unroll
                for (int s2 = 0; s2 < S; s2++) {
                    const int ox = s_off[s2][0] - s_off[sp][0];
                    const int oy = s_off[s2][1] - s_off[sp][1];
                    const int oz = s_off[s2][2] - s_off[sp][2];
                    const bool use = s2 >= sp && ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1 &&
                                     oz >= -1 && oz <= 1;
                    const int k = (oz + 1) * 9 + (oy + 1) * 3 + (ox + 1);
                    wd[s2] = use ? __ldg(A.pmask + (long long)(k - 13) * n + gp) : 0u;
                }
#pragma unroll
                for (int s2 = 0; s2 < S; s2++) {
                    const int b = s_beg[s2], nb = s_beg[s2 + 1] - b;
                    // bits beyond the slot's molecules cannot be set by an
                    // evaluation with every cell within 32; a graph replay
                    // whose cells outgrew that (flagged, and discarded) must
                    // not place them outside the slot either
                    const unsigned word = wd[s2] & (nb >= 32 ? ~0u : (1u << nb) - 1u);
                    if (!word) continue;
                    const int w0 = b >> 5, sh = b & 31;
                    rowa[w0] |= word << sh;
                    if (sh && (word >> (32 - sh))) rowa[w0 + 1] |= word >> (32 - sh);
                }
            }
            __syncthreads();
            // adjT by transposing 32 x 32 blocks of adj (row block rb, column
            // word cb >= rb): lane i holds row rb * 32 + i's word cb and ends
            // with column cb * 32 + i's word rb
            const int nblk = Wm * (Wm + 1) / 2;
            for (int it = warp; it < nblk; it += nwarps) {
                int rb = 0, cb = it;
                while (cb >= Wm - rb) {
                    cb -= Wm - rb;
                    rb++;
                }
                cb += rb;
                const int p = (rb << 5) + lane;
                unsigned col = p < M ? adj[p * W + cb] : 0u;
                const int jn = min(32, M - (cb << 5));
                // recursive block transpose: at size sz = 16, 8, .., 1 lanes i and
                // i ^ sz swap the off-diagonal sz x sz sub-blocks of their
                // 2sz x 2sz block (msk: the bits of the left sub-block columns)
                unsigned msk = 0x0000ffffu;
#pragma unroll
                for (int sz = 16; sz >= 1; sz >>= 1, msk ^= msk << sz) {
                    const unsigned o = __shfl_xor_sync(FULL, col, sz);
                    col = (lane & sz) ? (col & ~msk) | ((o >> sz) & msk) : (col & msk) | ((o << sz) & ~msk);
                }
                if (lane < jn) adjT[((cb << 5) + lane) * W + rb] = col;
            }
            __syncthreads();
            // per-word prefix popcounts and the row's edge count
            for (int p = tid; p < M; p += blockDim.x) {
                int run = 0;
                for (int w = p >> 5; w < Wm; w++) {
                    rowpre[p * W + w] = (unsigned short)run;
                    run += __popc(adj[p * W + w]);
                }
                rowoff[p + 1] = run;
            }
        } else if (!F64) {
            for (int p = tid; p < M; p += blockDim.x) {
                int run = 0;
                const unsigned pbit = 1u << (p & 31);
                const int pw = p >> 5;
                for (int w = p >> 5; w < Wm; w++) {  // words below the diagonal stay zero
                    unsigned word = 0u;
                    const int qa = max(p + 1, w << 5), qb = min(M, (w << 5) + 32);
                    for (int q = qa; q < qb; q++)
                        if (close(p, q)) {
                            word |= 1u << (q & 31);
                            atomicOr(&adjT[q * W + pw], pbit);
                        }
                    adj[p * W + w] = word;
                    rowpre[p * W + w] = (unsigned short)run;
                    run += __popc(word);
                }
                rowoff[p + 1] = run;
            }
        } else {
            for (int p = warp; p < M; p += nwarps) {
                int run = 0;
                for (int w = p >> 5; w < Wm; w++) {  // words below the diagonal stay zero
                    int q = (w << 5) + lane;
                    bool keep = q > p && q < M && close(p, q);
                    unsigned word = __ballot_sync(FULL, keep);
                    if (lane == 0) {
                        adj[p * W + w] = word;
                        rowpre[p * W + w] = (unsigned short)run;
                    }
                    run += __popc(word);
                    if (keep) atomicOr(&adjT[q * W + (p >> 5)], 1u << (p & 31));
                }
                if (lane == 0) rowoff[p + 1] = run;
            }
        }
    } else if (A.use_d) {
        // row x of the upper triangle holds y = x+1 .. M-1 contiguously:
        // D[dsel(x) + y]; one warp per row
        for (int x = warp; x < M - 1; x += nwarps) {
            const int dx = dsel(x);
            for (int y = x + 1 + lane; y < M; y += 32) D[dx + y] = disp32(x, y);
        }
    }
    __syncthreads();

    // ---- 2. edge numbering, third-member slot masks, edge vectors
    bool edge_mode = false;
    if (PAIR) {
        if (warp == 0) {
            // row offsets: exclusive prefix sum of the row edge counts
            int run = 0;
            for (int p0 = 0; p0 < M; p0 += 32) {
                int p = p0 + lane;
                int c = p < M ? rowoff[p + 1] : 0;
                int incl = c;
                for (int o = 1; o < 32; o <<= 1) {
                    int v = __shfl_up_sync(FULL, incl, o);
                    if (lane >= o) incl += v;
                }
                __syncwarp();  // every count of this chunk is read before it is overwritten
                if (p < M) rowoff[p] = run + incl - c;
                run += __shfl_sync(FULL, incl, 31);
                __syncwarp();
            }
            if (lane == 0) {
                rowoff[M] = run;
                s_edges = run;
            }
        }
        if (TRAV == 2) {
            // allowed third members r given v = slot(p) & slot(q): (v & slot(r)) == 0
            const int w0w = nwarps > 1 ? 1 : 0, nw = nwarps > 1 ? nwarps - 1 : 1;
            for (int idx = warp - w0w; idx >= 0 && idx < 8 * Wm; idx += nw) {
                int v = idx / Wm, w = idx - v * Wm;
                int r = (w << 5) + lane;
                unsigned word = __ballot_sync(FULL, r < M && (v & sslot[r]) == 0);
                if (lane == 0) memb[v * W + w] = word;
            }
        }
        __syncthreads();
        edge_mode = s_edges <= A.gcap;
        if (tid == 0 && A.emax) atomicMax(A.emax, (16 * s_edges + mcap - 1) / mcap);
        if (edge_mode) {
            // edge list (p, q) in edge order, one thread per row; FP64 then
            // tabulates d(p -> q) and |d|^2 one thread per edge (every lane
            // does FP64 work)
            for (int p = tid; p < M; p += blockDim.x) {
                int e = rowoff[p];
                for (int w = p >> 5; w < Wm; w++) {
                    unsigned word = adj[p * W + w];
                    while (word) {
                        const int q = (w << 5) + __ffs(word) - 1;
                        word &= word - 1u;
                        el[e] = (unsigned)p | ((unsigned)q << 16);
                        G[e] = GT(0);
                        e++;
                    }
                }
            }
            if (F64 && A.use_d) {
                __syncthreads();
                for (int e = tid; e < s_edges; e += blockDim.x) {
                    const unsigned x = el[e];
                    R dx, dy, dz;
                    const R a = disp((int)(x & 0xffffu), (int)(x >> 16), dx, dy, dz);
                    ED[4 * e] = dx;
                    ED[4 * e + 1] = dy;
                    ED[4 * e + 2] = dz;
                    ED[4 * e + 3] = a;
                }
            }
        } else {
            for (int t = tid; t < M; t += blockDim.x) {
                acc_zero(t);
                acc_zero(mcap + t);
                acc_zero(2 * mcap + t);
            }
            if (LJ) {
                __syncthreads();
                // LJ of the c08 pairs straight into the per-molecule accumulators
                for (int p = warp; p < M; p += nwarps)
                    for (int w = p >> 5; w < Wm; w++) {
                        const int q = (w << 5) + lane;
                        if (((adj[p * W + w] >> lane) & 1u) && lj_own(p, q)) {
                            R dx, dy, dz;
                            const R g = lj_pair(disp(p, q, dx, dy, dz));
                            acc_add(p, g * dx);
                            acc_add(mcap + p, g * dy);
                            acc_add(2 * mcap + p, g * dz);
                            acc_add(q, -(g * dx));
                            acc_add(mcap + q, -(g * dy));
                            acc_add(2 * mcap + q, -(g * dz));
                        }
                    }
            }
        }
        __syncthreads();
    }
    if (LJ && edge_mode) {
        // pair scalars of the c08 pairs start at their LJ term (thread per edge)
        for (int e = tid; e < s_edges; e += blockDim.x) {
            const unsigned x = el[e];
            const int p = (int)(x & 0xffffu), q = (int)(x >> 16);
            if (lj_own(p, q)) {
                R a;
                if (F64 && A.use_d) {
                    a = ED[4 * e + 3];
                } else {
                    R dx, dy, dz;
                    a = disp(p, q, dx, dy, dz);
                }
                gset(e, lj_pair(a));
            }
        }
    }
    if (LJ) {
        // the unit's LJ sums are complete: store them now (nothing stays live
        // through the triplet phase; the reduction's barriers also order the
        // pair-scalar writes above before the triplet phase)
        unsigned long long cand2 = 0;
        if (warp == 0) cand2 = unit_pair_candidates_warp<TRAV, S>(s_beg);
        unit_reduce_store2<NWB>(e2sum.get(), w2sum.get(), (unsigned long long)n2, cand2, A.unit_ew2,
                              A.unit_cnt2, u, s_red, s_redn);
    }
    const bool use_acc = PAIR ? !edge_mode : (A.acc_mode == 1);
    // FP32: once every decision is taken with the canonical displacement (the
    // pair rule's adjacency and LJ; the product rule's dense distance table),
    // the triplet phase and the gather take the FP32 shifted rows xl + o w
    // (one rounding per coordinate), so a displacement is one difference per
    // component and the third side of a triangle costs no load.  (The product
    // rule without the table decides from the rows and keeps them.)
    bool shifted = false;
    if constexpr (!F64) shifted = PAIR || A.use_d;
    else shifted = PAIR && !A.use_d;  // FP64 pair rule without the edge-vector table
    if (shifted) {
        __syncthreads();
        for (int t = tid; t < M; t += blockDim.x) {
            if constexpr (!F64) {
                const float4 a = P4[t], sh = S4[t];
                S4[t] = make_float4(a.x + sh.x, a.y + sh.y, a.z + sh.z, 0.0f);
            } else {
                px[t] += shx[t];
                py[t] += shy[t];
                pz[t] += shz[t];
            }
        }
        __syncthreads();
    }

    // ---- 3 + 4. triangles, evaluation, pair scalars
    Sum<R> esum, wsum;
    unsigned int nint = 0;
    int qn = 0;

    // pair rule: evaluate triangle (p, q, r) whose edge (p, q) is edge epq (all
    // lanes call; invalid lanes carry a valid stand-in and discard the result).
    // Adds the (p, r) and (q, r) pair scalars and returns the (p, q) one (0 for
    // invalid lanes and in accumulator mode), which the edge's owner lane sums.
    auto eval_tri = [&](int p, int q, int r, int epq, int epr, int eqr, bool valid) -> R {
        R dpqx, dpqy, dpqz, dprx, dpry, dprz, dqrx, dqry, dqrz, a, b, c;
        if (F64 && shifted) {
            const R Px = px[p], Py = py[p], Pz = pz[p], Qx = px[q], Qy = py[q], Qz = pz[q];
            const R Rx = px[r], Ry = py[r], Rz = pz[r];
            dpqx = Qx - Px; dpqy = Qy - Py; dpqz = Qz - Pz;
            dprx = Rx - Px; dpry = Ry - Py; dprz = Rz - Pz;
            dqrx = Rx - Qx; dqry = Ry - Qy; dqrz = Rz - Qz;
            a = dpqx * dpqx + dpqy * dpqy + dpqz * dpqz;
            b = dprx * dprx + dpry * dpry + dprz * dprz;
            c = dqrx * dqrx + dqry * dqry + dqrz * dqrz;
        } else if (F64 && !use_acc) {
            dpqx = ED[4 * epq]; dpqy = ED[4 * epq + 1]; dpqz = ED[4 * epq + 2]; a = ED[4 * epq + 3];
            dprx = ED[4 * epr]; dpry = ED[4 * epr + 1]; dprz = ED[4 * epr + 2]; b = ED[4 * epr + 3];
            dqrx = ED[4 * eqr]; dqry = ED[4 * eqr + 1]; dqrz = ED[4 * eqr + 2]; c = ED[4 * eqr + 3];
        } else if constexpr (!F64) {
            const float4 P = S4[p], Qv = S4[q], Rv = S4[r];  // shifted rows
            dpqx = Qv.x - P.x; dpqy = Qv.y - P.y; dpqz = Qv.z - P.z;
            dprx = Rv.x - P.x; dpry = Rv.y - P.y; dprz = Rv.z - P.z;
            dqrx = Rv.x - Qv.x; dqry = Rv.y - Qv.y; dqrz = Rv.z - Qv.z;
            a = dpqx * dpqx + dpqy * dpqy + dpqz * dpqz;
            b = dprx * dprx + dpry * dpry + dprz * dprz;
            c = dqrx * dqrx + dqry * dqry + dqrz * dqrz;
        } else {
            a = disp(p, q, dpqx, dpqy, dpqz);
            b = disp(p, r, dprx, dpry, dprz);
            c = disp(q, r, dqrx, dqry, dqrz);
        }
        R uu, ua, ub, uc;
        atm_terms<R>(a, b, c, nu, uu, ua, ub, uc);
        R gpq = R(2) * ua, gpr = R(2) * ub, gqr = R(2) * uc;
        if (!valid) return R(0);
        esum.add(uu);
        wsum.add(-(gpq * a + gpr * b + gqr * c));
        if (!use_acc) {
            gadd(epr, gpr);
            gadd(eqr, gqr);
            return gpq;
        } else {
            acc_add(p, gpq * dpqx + gpr * dprx);
            acc_add(mcap + p, gpq * dpqy + gpr * dpry);
            acc_add(2 * mcap + p, gpq * dpqz + gpr * dprz);
            acc_add(q, gqr * dqrx - gpq * dpqx);
            acc_add(mcap + q, gqr * dqry - gpq * dpqy);
            acc_add(2 * mcap + q, gqr * dqrz - gpq * dpqz);
            acc_add(r, -(gpr * dprx + gqr * dqrx));
            acc_add(mcap + r, -(gpr * dpry + gqr * dqry));
            acc_add(2 * mcap + r, -(gpr * dprz + gqr * dqrz));
        }
        return R(0);
    };

    // product rule: evaluate one queued triplet per lane (all lanes call;
    // invalid lanes take part in the warp reduction only)
    auto evaluate = [&](unsigned long long ent, bool valid) {
        int p = (int)(ent & 0x7ff), q = (int)((ent >> 11) & 0x7ff), r = (int)((ent >> 22) & 0x7ff);
        R dpqx, dpqy, dpqz, dprx, dpry, dprz, dqrx, dqry, dqrz, a, b, c;
        int epq = 0, epr = 0, eqr = 0;
        {
            if constexpr (!F64) {
                if (shifted) {
                    const float4 P = S4[p], Qv = S4[q], Rv = S4[r];  // shifted rows
                    dpqx = Qv.x - P.x; dpqy = Qv.y - P.y; dpqz = Qv.z - P.z;
                    dprx = Rv.x - P.x; dpry = Rv.y - P.y; dprz = Rv.z - P.z;
                    dqrx = Rv.x - Qv.x; dqry = Rv.y - Qv.y; dqrz = Rv.z - Qv.z;
                    a = dpqx * dpqx + dpqy * dpqy + dpqz * dpqz;
                    b = dprx * dprx + dpry * dpry + dprz * dprz;
                    c = dqrx * dqrx + dqry * dqry + dqrz * dqrz;
                } else {
                    a = disp(p, q, dpqx, dpqy, dpqz);
                    b = disp(p, r, dprx, dpry, dprz);
                    c = disp(q, r, dqrx, dqry, dqrz);
                }
            } else {
                a = disp(p, q, dpqx, dpqy, dpqz);
                b = disp(p, r, dprx, dpry, dprz);
                c = disp(q, r, dqrx, dqry, dqrz);
            }
            if (!PAIR) {
                epq = tri_index(p, q);
                epr = tri_index(p, r);
                eqr = tri_index(q, r);
            }
        }
        R uu, ua, ub, uc;
        atm_terms<R>(a, b, c, nu, uu, ua, ub, uc);
        R gpq = R(2) * ua, gpr = R(2) * ub, gqr = R(2) * uc;
        if (!valid) {
            uu = R(0);
            gpq = gpr = gqr = R(0);
        }
        esum.add(uu);
        wsum.add(-(gpq * a + gpr * b + gqr * c));
        if (DET && !use_acc) {
            // every term on its own: integer sums, the same for any batching
            if (valid) {
                gadd(epq, gpq);
                gadd(epr, gpr);
                gadd(eqr, gqr);
            }
        } else if (!use_acc) {
            // runs of equal e(p,q) are contiguous in a batch (q-major order)
            int key = epq;
            if (!valid) key = -1 - lane;
            R run = seg_sum<R>(gpq, key, lane);
            int prev = __shfl_up_sync(FULL, key, 1);
            bool head = lane == 0 || prev != key;
            if (valid) {
                if (head) gadd(key, run);
                gadd(epr, gpr);
                gadd(eqr, gqr);
            }
        } else if (valid) {
            acc_add(p, gpq * dpqx + gpr * dprx);
            acc_add(mcap + p, gpq * dpqy + gpr * dpry);
            acc_add(2 * mcap + p, gpq * dpqz + gpr * dprz);
            acc_add(q, gqr * dqrx - gpq * dpqx);
            acc_add(mcap + q, gqr * dqry - gpq * dpqy);
            acc_add(2 * mcap + q, gqr * dqrz - gpq * dpqz);
            acc_add(r, -(gpr * dprx + gqr * dqrx));
            acc_add(mcap + r, -(gpr * dpry + gqr * dqry));
            acc_add(2 * mcap + r, -(gpr * dprz + gqr * dqrz));
        }
    };
    auto push = [&](bool keep, unsigned long long entry) {
        unsigned m = __ballot_sync(FULL, keep);
        if (m == 0u) return;
        if (keep) queue[qn + __popc(m & lt_mask)] = entry;
        qn += __popc(m);
        nint += keep ? 1u : 0u;
        __syncwarp();
        if (qn >= 32) {
            evaluate(queue[lane], true);
            __syncwarp();
            if (lane < qn - 32) queue[lane] = queue[32 + lane];
            qn -= 32;
            __syncwarp();
        }
    };
    auto pack = [](int p, int q, int r, int jj) -> unsigned long long {
        return (unsigned long long)p | ((unsigned long long)q << 11) |
               ((unsigned long long)r << 22) | ((unsigned long long)jj << 33);
    };
    auto kword = [&](int p, int q, int v, int w) -> unsigned {
        return adj[p * W + w] & adj[q * W + w] & (TRAV == 2 ? memb[v * W + w] : FULL);
    };

    // ends (p, q) of edge e: from the edge list, or (no list) p = the last row
    // with rowoff[p] <= e and q = the (e - rowoff[p])-th set bit of row p
    auto edge_ends = [&](int e, int& p, int& q) {
        if (edge_mode) {
            const unsigned x = el[e];
            p = (int)(x & 0xffffu);
            q = (int)(x >> 16);
            return;
        }
        locate_edge(e, p, q);
    };

    if (PAIR) {
        // warps take 32 edges (p, q) at a time; the triangles of edge (p, q) are
        // the set bits r > q of adj[p] & adj[q] (& the slots allowed as third
        // member); they are counted per lane, prefix-summed and expanded 32 per
        // round, so every lane of a round evaluates one triangle
        const int Ework = rowoff[Mfirst];  // edges whose first molecule can open a triangle
        // 3c18 units (up to 14 cells, more adjacency words per row) locate a
        // third member's word from per-word counts packed in bytes, pass an
        // edge's (p, q, slot mask) in one shuffle and sum runs from a head
        // mask; the 2x2x2 units scan the words (measured faster there in
        // steps with LJ inside the units: 1.19 against 1.25 ms at 256k)
        constexpr bool PACK = TRAV == 1;
        for (int it = 0;; it++) {
            // deterministic mode: warp w takes the groups w, w + nwarps, ...
            int e0 = (it * nwarps + warp) * 32;
            if (!DET) {
                if (lane == 0) e0 = atomicAdd(&s_next, 32);
                e0 = __shfl_sync(FULL, e0, 0);
            }
            if (e0 >= Ework) break;
            const int e = e0 + lane;
            int p = 0, q = 0, v = 0, cnt = 0;
            unsigned long long cw = 0ull;  // third members per word, byte j = word (q >> 5) + j
            if (e < Ework) {
                edge_ends(e, p, q);
                v = sslot[p] & sslot[q];
                if (!(TRAV == 2 && sslot[p] == 7)) {  // no later slot completes an anchored set
                    const int wq = q >> 5;
                    for (int w = wq; w < Wm; w++) {
                        const unsigned c = __popc(kword(p, q, v, w));
                        cnt += (int)c;
                        if (PACK && Wm <= 8) cw |= (unsigned long long)c << ((w - wq) << 3);
                    }
                }
            }
            // inclusive byte sums of the per-word counts (no carry between
            // bytes while every count of the group is below 128)
            const bool packed = PACK && Wm <= 8 && __all_sync(FULL, cnt < 128);
            const unsigned c0 = (unsigned)cw * 0x01010101u;
            const unsigned c1 = Wm > 4 ? (unsigned)(cw >> 32) * 0x01010101u + (c0 >> 24) * 0x01010101u
                                       : 0x7f7f7f7fu;
            int incl = cnt;
            for (int o = 1; o < 32; o <<= 1) {
                int t = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += t;
            }
            const int total = __shfl_sync(FULL, incl, 31);
            const int excl = incl - cnt;
            // the edge's ends and slot mask in one word (staged indices < 2048)
            const unsigned pqv = (unsigned)p | ((unsigned)q << 11) | ((unsigned)v << 22);
            R gown = R(0);  // (p, q) scalar of this lane's edge, summed over its triangles
            for (int t0 = 0; t0 < total; t0 += 32) {
                const bool valid = t0 + lane < total;
                const int t = valid ? t0 + lane : t0;  // invalid lanes repeat the round's first
                // lane owning triangle t: the last lane whose exclusive prefix is <= t
                int l = 0;
                for (int s = 16; s >= 1; s >>= 1) {
                    int ec = __shfl_sync(FULL, excl, l + s);
                    if (ec <= t) l += s;
                }
                int pl, ql, vl;
                if constexpr (PACK) {
                    const unsigned pk = __shfl_sync(FULL, pqv, l);
                    pl = (int)(pk & 0x7ffu);
                    ql = (int)((pk >> 11) & 0x7ffu);
                    vl = (int)(pk >> 22);
                } else {
                    pl = __shfl_sync(FULL, p, l);
                    ql = __shfl_sync(FULL, q, l);
                    vl = __shfl_sync(FULL, v, l);
                }
                int nth = t - __shfl_sync(FULL, excl, l);
                // the word holding the nth third member -- from the owner's
                // packed counts (the number of words whose inclusive count is
                // <= nth), else by a scan -- then its bit, and the edge
                // numbers of (p, r) and (q, r)
                int r, epr = 0, eqr = 0;
                if (packed) {
                    const unsigned k0 = __shfl_sync(FULL, c0, l);
                    const unsigned k1 = Wm > 4 ? __shfl_sync(FULL, c1, l) : 0x7f7f7f7fu;
                    const unsigned n4 = ((unsigned)nth * 0x01010101u) | 0x80808080u;
                    const int js = __popc((n4 - k0) & 0x80808080u) + __popc((n4 - k1) & 0x80808080u);
                    if (js > 0) nth -= (int)(((js <= 4 ? k0 : k1) >> (((js - 1) & 3) << 3)) & 0xffu);
                    const int wsel = (ql >> 5) + js;
                    const unsigned Ap = adj[pl * W + wsel], Aq = adj[ql * W + wsel];
                    const unsigned Ksel = Ap & Aq & (TRAV == 2 ? memb[vl * W + wsel] : FULL);
                    r = (wsel << 5) + nth_bit(Ksel, nth);
                    if (!use_acc) {
                        const unsigned below = (1u << (r & 31)) - 1u;
                        epr = rowoff[pl] + rowpre[pl * W + wsel] + __popc(Ap & below);
                        eqr = rowoff[ql] + rowpre[ql * W + wsel] + __popc(Aq & below);
                    }
                } else {
                    int wsel = ql >> 5;
                    unsigned Ksel = 0u;
                    for (int w = ql >> 5; w < Wm; w++) {
                        const unsigned K = kword(pl, ql, vl, w);
                        const int c = __popc(K);
                        if (nth < c) {
                            wsel = w;
                            Ksel = K;
                            break;
                        }
                        nth -= c;
                    }
                    r = (wsel << 5) + nth_bit(Ksel, nth);
                    if (!use_acc) {
                        epr = rowoff[pl] + rank(pl, r);
                        eqr = rowoff[ql] + rank(ql, r);
                    }
                }
                // (invalid lanes repeat a valid triangle, so the selected word
                // has a set bit)
                nint += valid ? 1u : 0u;
                const R gpq = eval_tri(pl, ql, r, e0 + l, epr, eqr, valid);
                if (!use_acc) {
                    // a round holds each edge's triangles as one run of lanes:
                    // the run's sum goes to the edge's owner lane
                    R run;
                    if constexpr (PACK) {
                        // runs start at lane 0 and where the owner changes (the
                        // invalid lanes' zeros may join the last run)
                        const int lprev = __shfl_up_sync(FULL, l, 1);
                        const unsigned heads = __ballot_sync(FULL, lane == 0 || lprev != l);
                        const unsigned above = heads & ~((2u << lane) - 1u);
                        const int rend = above ? __ffs(above) - 1 : 32;
                        run = gpq;
#pragma unroll
                        for (int o = 1; o < 32; o <<= 1) {
                            const R tt = __shfl_down_sync(FULL, run, o);
                            if (lane + o < rend) run += tt;
                        }
                    } else {
                        run = seg_sum<R>(gpq, valid ? l : -1 - lane, lane);
                    }
                    const bool mine = cnt > 0 && excl < t0 + 32 && excl + cnt > t0;
                    const int head = (excl > t0 ? excl : t0) - t0;
                    const R got = __shfl_sync(FULL, run, mine ? head : 0);
                    if (mine) gown += got;
                }
            }
            if (!use_acc && e < Ework && gown != R(0)) gadd(e, gown);
        }
    } else {
        // the candidates p < q < r of each p run q-major (q, then r) and are cut
        // into tasks of CH, numbered row by row; warps take tasks from the
        // unit's counter (a warp's tasks only move forward, and so does its row
        // cursor).  A task runs 32 candidates per round: every lane walks from
        // the warp's cursor (qc, rc) to its own pair across the rows it
        // crosses, so a round's lanes read consecutive words of the distance
        // rows of p and q.
        constexpr int CH = 2048;
        const float t_lo = (float)rc6 * (1.0f - 0x1p-18f), t_hi = (float)rc6 * (1.0f + 0x1p-18f);
        int pc = 0, kbase = 0;  // row cursor; tasks of the rows before it
        for (int it = 0;; it++) {
            // deterministic mode: warp w takes the tasks w, w + nwarps, ...
            int k = it * nwarps + warp;
            if (!DET) {
                if (lane == 0) k = atomicAdd(&s_next, 1);
                k = __shfl_sync(FULL, k, 0);
            }
            for (; pc < Mfirst; pc++) {
                const int Lc = M - 1 - pc;
                // no later slot completes an anchored set: no tasks
                const int nch = (TRAV == 2 && sslot[pc] == 7) ? 0 : (Lc * (Lc - 1) / 2 + CH - 1) / CH;
                if (k < kbase + nch) break;
                kbase += nch;
            }
            if (pc >= Mfirst) break;
            const int p = pc;
            const int sp = sslot[p];
            const int dp = dsel(p);
            // candidates t0 .. t1-1 of p; row i (q = p + 1 + i) starts at
            // off(i) = i (L - 1) - i (i - 1) / 2
            const int L = M - 1 - p;
            const int t0 = (k - kbase) * CH, t1 = min(L * (L - 1) / 2, t0 + CH);
            auto off = [&](int i) -> int { return i * (L - 1) - i * (i - 1) / 2; };
            const float b2 = (float)(2 * L - 1);
            int i = (int)((b2 - sqrtf(fmaxf(b2 * b2 - 8.0f * (float)t0, 0.0f))) * 0.5f);
            i = max(i, 0);
            while (i > 0 && off(i) > t0) i--;
            while (off(i + 1) <= t0) i++;
            int qc = p + 1 + i, rc = qc + 1 + (t0 - off(i)), dqc = dsel(qc);
            for (int left = t1 - t0; left > 0; left -= 32) {
                int q = qc, r = rc + lane, dq = dqc;
                while (r >= M) {  // into the next row: it starts at r = q + 2
                    if (q >= M - 2) {
                        q = M;  // past the last pair
                        break;
                    }
                    r += q + 2 - M;
                    dq += M - q - 2;
                    q++;
                }
                bool keep = false;
                if (lane < left && q <= M - 2 && (TRAV != 2 || (sp & sslot[q] & sslot[r]) == 0)) {
                    float a32, b32, c32;
                    if (A.use_d) {
                        a32 = D[dp + q];
                        b32 = D[dp + r];
                        c32 = D[dq + r];
                    } else {
                        a32 = disp32(p, q);
                        b32 = disp32(p, r);
                        c32 = disp32(q, r);
                    }
                    // the product in this order is within 2^-22 (relative) of the
                    // sorted product that decides: only products in the band
                    // [t_lo, t_hi) around r_c^6 need the sorted form
                    const float pr = (a32 * b32) * c32;
                    if (!F64) {
                        keep = pr < t_lo;
                        if (!keep && pr < t_hi) keep = sorted_product<float>(a32, b32, c32) < (float)rc6;
                    } else {
                        float lo = fminf(a32, fminf(b32, c32));
                        if (lo >= rp.dmin && pr < rp.q_lo) {
                            keep = true;
                        } else if (lo >= rp.dmin && pr > rp.q_hi) {
                            keep = false;
                        } else {
                            R dx, dy, dz;
                            R a = disp(p, q, dx, dy, dz);
                            R b = disp(p, r, dx, dy, dz);
                            R c = disp(q, r, dx, dy, dz);
                            keep = sorted_product<R>(a, b, c) < rc6;
                        }
                    }
                }
                push(keep, pack(p, q, r, 0));
                // the next cursor: one past lane 31's pair
                qc = __shfl_sync(FULL, q, 31);
                rc = __shfl_sync(FULL, r, 31) + 1;
                dqc = __shfl_sync(FULL, dq, 31);
                if (rc >= M && qc <= M - 2) {
                    dqc += M - qc - 2;
                    qc++;
                    rc = qc + 1;
                }
            }
        }
    }
    if (!PAIR && qn > 0) evaluate(queue[lane < qn ? lane : 0], lane < qn);
    __syncthreads();

    // ---- 5. gather: F_m = sum over m's pairs of G_e d(m -> other end)
    // plain sums: a unit adds about 28 pair terms per molecule, and against
    // the oracle's FP32-decision forces the compensated form changed neither
    // the largest error (0.40 of the parity tolerance) nor the RMS error
    // (2.1e-6 of the RMS force) on the 32,000-molecule liquid
    struct PlainSum {
        R s = R(0);
        __device__ __forceinline__ void add(R v) { s += v; }
        __device__ __forceinline__ double get() const { return (double)s; }
    };
    for (int m = tid; m < M; m += blockDim.x) {
        PlainSum fxs, fys, fzs;
        if (use_acc) {
            fxs.add((R)acc_get(m));
            fys.add((R)acc_get(mcap + m));
            fzs.add((R)acc_get(2 * mcap + m));
        } else if (PAIR && !F64) {
            // FP32 edge vectors from the shifted rows; two pairs per iteration
            // (their loads in flight together), added in pair order
            int e = rowoff[m];
            const float4 Pm = S4[m];
            for (int w = 0; w < Wm; w++) {
                unsigned up = adj[m * W + w];
                while (up) {
                    const int y0 = (w << 5) + __ffs(up) - 1;
                    up &= up - 1u;
                    const bool two = up != 0u;
                    const int y1 = two ? (w << 5) + __ffs(up) - 1 : y0;
                    up &= up - 1u;
                    const int ee0 = e;
                    e += two ? 2 : 1;
                    const R g0 = gget(ee0);
                    const R g1 = two ? gget(ee0 + 1) : R(0);
                    const float4 Y0 = S4[y0], Y1 = S4[y1];
                    if (g0 != R(0)) {
                        fxs.add(g0 * (Y0.x - Pm.x));
                        fys.add(g0 * (Y0.y - Pm.y));
                        fzs.add(g0 * (Y0.z - Pm.z));
                    }
                    if (g1 != R(0)) {
                        fxs.add(g1 * (Y1.x - Pm.x));
                        fys.add(g1 * (Y1.y - Pm.y));
                        fzs.add(g1 * (Y1.z - Pm.z));
                    }
                }
                unsigned dn = adjT[m * W + w];
                while (dn) {
                    const int x0 = (w << 5) + __ffs(dn) - 1;
                    dn &= dn - 1u;
                    const bool two = dn != 0u;
                    const int x1 = two ? (w << 5) + __ffs(dn) - 1 : x0;
                    dn &= dn - 1u;
                    const R g0 = gget(rowoff[x0] + rank(x0, m));
                    const R g1 = two ? gget(rowoff[x1] + rank(x1, m)) : R(0);
                    const float4 X0 = S4[x0], X1 = S4[x1];
                    if (g0 != R(0)) {
                        fxs.add(g0 * (X0.x - Pm.x));
                        fys.add(g0 * (X0.y - Pm.y));
                        fzs.add(g0 * (X0.z - Pm.z));
                    }
                    if (g1 != R(0)) {
                        fxs.add(g1 * (X1.x - Pm.x));
                        fys.add(g1 * (X1.y - Pm.y));
                        fzs.add(g1 * (X1.z - Pm.z));
                    }
                }
            }
        } else if (PAIR) {
            // FP64 edge vectors: from the shifted rows, or from the table
            // (d(lo -> hi), so the sign flips for edges where m is the upper end)
            int e = rowoff[m];
            for (int w = 0; w < Wm; w++) {
                unsigned up = adj[m * W + w];
                while (up) {
                    int y = (w << 5) + __ffs(up) - 1;
                    up &= up - 1u;
                    const int ee = e++;
                    R g = gget(ee);
                    if (g != R(0)) {
                        R dx, dy, dz;
                        if (shifted) {
                            dx = px[y] - px[m]; dy = py[y] - py[m]; dz = pz[y] - pz[m];
                        } else {
                            dx = ED[4 * ee]; dy = ED[4 * ee + 1]; dz = ED[4 * ee + 2];
                        }
                        fxs.add(g * dx);
                        fys.add(g * dy);
                        fzs.add(g * dz);
                    }
                }
                unsigned dn = adjT[m * W + w];
                while (dn) {
                    int x = (w << 5) + __ffs(dn) - 1;
                    dn &= dn - 1u;
                    const int ee = rowoff[x] + rank(x, m);
                    R g = gget(ee);
                    if (g != R(0)) {
                        R dx, dy, dz;
                        if (shifted) {
                            dx = px[x] - px[m]; dy = py[x] - py[m]; dz = pz[x] - pz[m];
                        } else {
                            dx = -ED[4 * ee]; dy = -ED[4 * ee + 1]; dz = -ED[4 * ee + 2];
                        }
                        fxs.add(g * dx);
                        fys.add(g * dy);
                        fzs.add(g * dz);
                    }
                }
            }
        } else {
            for (int y = 0; y < M; y++) {
                if (y == m) continue;
                R g = gget(y > m ? tri_index(m, y) : tri_index(y, m));
                if (g != R(0)) {
                    R dx, dy, dz;
                    if (shifted) {
                        const float4 Pm4 = S4[m], Y = S4[y];
                        dx = Y.x - Pm4.x; dy = Y.y - Pm4.y; dz = Y.z - Pm4.z;
                    } else {
                        disp(m, y, dx, dy, dz);
                    }
                    fxs.add(g * dx);
                    fys.add(g * dy);
                    fzs.add(g * dz);
                }
            }
        }
        double f0 = use_acc ? acc_get(m) : fxs.get();
        double f1 = use_acc ? acc_get(mcap + m) : fys.get();
        double f2 = use_acc ? acc_get(2 * mcap + m) : fzs.get();
        const int g = F64 ? sidx[m] : __float_as_int(P4[m].w);
        if constexpr (DET) {
            // 64-bit fixed-point sums across units (converted after the launch)
            unsigned long long* fsx = reinterpret_cast<unsigned long long*>(A.fs);
            if (f0 != 0.0) atomicAdd(fsx + g, to_fix<R>(f0, A.status));
            if (f1 != 0.0) atomicAdd(fsx + n + g, to_fix<R>(f1, A.status));
            if (f2 != 0.0) atomicAdd(fsx + 2 * n + g, to_fix<R>(f2, A.status));
        } else {
            if (f0 != 0.0) atomicAdd(A.fs + g, f0);
            if (f1 != 0.0) atomicAdd(A.fs + n + g, f1);
            if (f2 != 0.0) atomicAdd(A.fs + 2 * n + g, f2);
        }
    }

    unsigned long long cand = 0;
    if (warp == 0) cand = unit_candidates_warp<TRAV, S>(s_beg);
    unit_reduce_store<NWB>(esum.get(), wsum.get(), (unsigned long long)nint, 1.0, cand, A.unit_ew,
                         A.unit_cnt, u, s_red, s_redn);
}

// One CTA per unit, or (A.work set) a persistent grid whose CTAs take units
// from a global counter until all units of the batch are done; with a unit
// list (size classes) the same over the listed units.
// FP32: at most 56 registers, so that 9 CTAs of 4 warps fit an SM (with the
// 16-edge-per-molecule pair-scalar table, 9 also fit its shared memory at the
// rho* = 0.8 cell occupancy); FP64: 2 CTAs of 8 warps.  The 3c18 product
// rule takes up to 16 warps (one CTA per SM when its tables fill shared
// memory); the bound of 512 threads costs the other kernels registers.
template <int TRAV, int TRUNC, typename R, bool DET = false>
__global__ void __launch_bounds__(TRUNC == 1 && TRAV == 1 ? 512 : 256)
    __maxnreg__(sizeof(R) == 8 ? 128 : 56)
    atm_block_kernel(const AtmArgs<R> A)
{
    // units 0 .. ncell, or (size classes) the units ulist[0 .. *ucount)
    const long long nu = A.ulist ? (long long)*A.ucount : A.b.ncell;
    if (A.work == nullptr) {
        if ((long long)blockIdx.x >= nu) return;
        atm_block_unit<TRAV, TRUNC, R, DET>(A, A.ulist ? A.ulist[blockIdx.x] : (long long)blockIdx.x);
        return;
    }
    __shared__ int s_u;
    for (;;) {
        __syncthreads();  // the previous unit is done with shared memory
        if (threadIdx.x == 0) s_u = atomicAdd(A.work, 1);
        __syncthreads();
        const int k = s_u;
        if (k >= nu) break;
        atm_block_unit<TRAV, TRUNC, R, DET>(A, A.ulist ? A.ulist[k] : (long long)k);
    }
}

}  // namespace atm3
