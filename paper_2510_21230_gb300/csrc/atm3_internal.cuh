// atm3_internal.cuh -- device-side types shared by the CUDA translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace atm3 {

constexpr int ATM_NTRAV = 5;  // 3c01, 3c18, 3c08, 3cw, corner-anchored 3c08
constexpr int ATM_MAX_DEVICES = 64;  // per-device kernel attribute bookkeeping

// device status word bits (set by kernels, read back by the host)
enum : int {
    ST_CAPACITY = 1,   // a unit stages more molecules than its shared memory holds
    ST_NONFINITE = 2,  // a non-finite position or velocity was seen
    ST_TIMEOUT = 4,    // a bounded device-side wait gave up
    ST_RANGE = 8,      // deterministic mode: a term beyond the fixed-point range
};

// Deterministic mode: force terms are summed as signed 64-bit integers in
// units of 2^-FIX_BITS (integer addition does not depend on the order of
// the additions).  FP32C keeps 2^-32 (terms up to 2^30 in size), FP64 2^-44
// (terms up to 2^18 = 262,144, below the resolution of a 1e-10 relative
// force error for forces of order one).
template <typename R>
struct FixBits {
    static constexpr int B = sizeof(R) == 8 ? 44 : 32;
};
// a term may not exceed 2^(FIX_LIMIT - B) in size, so that sums of up to
// 2^(63 - FIX_LIMIT) = 32 such terms still fit
constexpr int FIX_LIMIT = 58;

// Linked-cell grid (section 3): n_d cells of edge w_d = L_d / n_d per axis.
struct Grid {
    int nc[3];
    double L[3];
    double w[3];
    double iw[3];  // 1 / w rounded to nearest (the binning's fast path)
    long long ncell;
};

// One replica (an independent periodic system) of a batch.  Its molecules
// are [mol0, mol0 + n) in both the original and the sorted order, its cells
// [cell0, cell0 + g.ncell) in the global cell numbering, so every per-molecule
// and per-cell array of the batch is the replicas' arrays back to back.
// A single system is a batch of one replica.
struct Rep {
    Grid g;
    long long mol0, n, cell0;
    double rc, rc2, rc6, nu, dt;
    double sig2, eps4, eps24, eps48, ushift;  // LJ
    float rcf, rc2f, rc6f, nuf, sig2f, eps4f, eps24f, eps48f, ushiftf;
    float wf[3];
    float p_lo, p_hi;          // FP64 prefilter band of a squared distance
    float q_lo, q_hi, dmin;    // FP64 prefilter band of the FP32 product of the squared sides
    double rw2;                // wide traversal: (2 min w)^2, partners and third sides below it
    float rw2f;
    // domain decomposition: the cell layers z in [own_z0, own_z1) this context
    // owns (all layers by default); ATM units based or anchored elsewhere and
    // LJ for molecules elsewhere contribute nothing
    int own_z0, own_z1;
};

// the unit (base or anchor cell, index inside its replica) lies in an owned layer
__host__ __device__ __forceinline__ bool unit_owned(const Rep& rp, long long lu)
{
    const int cz = (int)(lu / ((long long)rp.g.nc[0] * rp.g.nc[1]));
    return cz >= rp.own_z0 && cz < rp.own_z1;
}

struct Batch {
    const Rep* rep;          // [R]
    const int* rep_of_cell;  // [ncell] replica of each global cell
    const int* rep_of_mol;   // [ntot] replica of each molecule (either order)
    int R;
    long long ntot, ncell;
};

// cell coordinates of a cell id (z-major lexicographic)
__host__ __device__ __forceinline__ void cell_coords(const Grid& g, long long id, int& cx, int& cy,
                                                     int& cz)
{
    cx = (int)(id % g.nc[0]);
    long long r = id / g.nc[0];
    cy = (int)(r % g.nc[1]);
    cz = (int)(r / g.nc[1]);
}

// neighbour cell id at offset (dx, dy, dz), |d| <= 1, periodic
__host__ __device__ __forceinline__ long long cell_at(const Grid& g, int cx, int cy, int cz, int dx,
                                                      int dy, int dz)
{
    int x = cx + dx, y = cy + dy, z = cz + dz;
    x = x < 0 ? x + g.nc[0] : (x >= g.nc[0] ? x - g.nc[0] : x);
    y = y < 0 ? y + g.nc[1] : (y >= g.nc[1] ? y - g.nc[1] : y);
    z = z < 0 ? z + g.nc[2] : (z >= g.nc[2] ? z - g.nc[2] : z);
    return ((long long)z * g.nc[1] + y) * g.nc[0] + x;
}

// Offsets of the 27-cell neighbourhood by linear index t = (dz+1)*9 + (dy+1)*3 + (dx+1).
// t = 13 is the cell itself; t > 13 are the 13 forward neighbours ((dz,dy,dx) > 0).
__host__ __device__ __forceinline__ void offset27(int t, int& dx, int& dy, int& dz)
{
    dx = t % 3 - 1;
    dy = (t / 3) % 3 - 1;
    dz = t / 9 - 1;
}

// Cell slots staged by each traversal's unit, base cell first.
//  3c01: slot 0 = base, then the other 26 neighbours in linear order.
//  3cw:  slot 0 = base, then the other 124 cells of the 5^3 neighbourhood in
//        linear order ((dz, dy, dx) in -2..2).
//  3c18: slot 0 = base, slots 1..13 = forward neighbours in lexicographic order.
//  3c08 and the corner-anchored 3c08: slot s = offset (s & 1, s >> 1 & 1,
//        s >> 2 & 1) inside the 2x2x2 block.
template <int TRAV>
__host__ __device__ __forceinline__ void slot_offset(int s, int& dx, int& dy, int& dz)
{
    if (TRAV == 0) {
        int t = s == 0 ? 13 : (s <= 13 ? s - 1 : s);
        offset27(t, dx, dy, dz);
    } else if (TRAV == 1) {
        offset27(13 + s, dx, dy, dz);
    } else if (TRAV == 3) {
        int t = s == 0 ? 62 : (s <= 62 ? s - 1 : s);
        dx = t % 5 - 2;
        dy = (t / 5) % 5 - 2;
        dz = t / 25 - 2;
    } else {
        dx = s & 1;
        dy = (s >> 1) & 1;
        dz = (s >> 2) & 1;
    }
}

template <int TRAV>
struct Trav;
template <>
struct Trav<0> {
    static constexpr int S = 27;
};
template <>
struct Trav<1> {
    static constexpr int S = 14;
};
template <>
struct Trav<2> {
    static constexpr int S = 8;
};
template <>
struct Trav<3> {
    static constexpr int S = 125;
};
template <>
struct Trav<4> {
    static constexpr int S = 8;
};

// Arguments of the ATM unit kernels.
template <typename R>
struct AtmArgs {
    Batch b;                  // replicas (geometry, cutoffs, prefilter bands)
    long long n;              // SoA stride = b.ntot
    const R* xl;              // sorted cell-local coordinates, SoA [3n], working precision
    const float* xl32;        // the same in FP32 (prefilter of the FP64 path)
    const int* cell_start;    // [ncell + 1], global sorted indices
    double* fs;               // sorted-order ATM force accumulator, SoA [3n]
    double* unit_ew;          // [2 * ncell]: E3, W3 per unit
    unsigned long long* unit_cnt;  // [2 * ncell]: candidates, interacting
    int* status;
    int* work;                // persistent launch: unit counter (nullptr: one CTA per unit)
    int mcap;                 // staged-molecule capacity of one unit
    int gcap;                 // edge-accumulator capacity (block kernel)
    int use_d;                // block kernel, product rule: dense FP32 distance table in smem
    int acc_mode;             // block kernel, product rule: 0 dense pair scalars, 1 per-molecule atomics
    int pcap;                 // owner kernels: partner-list capacity per warp
    // pair rule of a block traversal in a velocity-Verlet step: the unit also
    // evaluates the LJ forces of its own pairs (3c08 and the corner-anchored
    // 3c08: pairs whose two cells have their bounding box anchored at the
    // unit; 3c18: pairs with a molecule in the base cell) and adds them to the
    // same pair scalars, so fs receives LJ + ATM; per-unit E2, W2 and counts
    // go to unit_ew2 / unit_cnt2 ([2 * ncell] each: E2, W2; half-shell
    // candidates, pairs)
    int lj;
    double* unit_ew2;
    unsigned long long* unit_cnt2;
    // block kernels, unit size classes: the CTAs (or the persistent counter)
    // take the units ulist[0 .. *ucount) instead of 0 .. ncell (nullptr: all)
    const int* ulist;
    const int* ucount;
    // deterministic mode: warps take their work in a fixed order (owner
    // kernels; the block kernels' deterministic instantiations also sum in
    // fixed point and fs holds 64-bit fixed-point sums, see FixBits)
    int det;
    // FP32 pair rule of the block traversals: the evaluation's pair bitmaps
    // (k_pair_masks, [PM_WORDS n] words, nullptr: the units decide their
    // pairs themselves); the units assemble their adjacency from them
    const unsigned* pmask;
    // pair rule of the block traversals: each unit raises *emax to the edge
    // table it needed, in 1/16 edges per staged molecule of this launch
    // (ceil(16 edges / mcap)), so later launches can size the table from it
    // (nullptr: not recorded)
    int* emax;
};

// pair bitmaps: word k - 13 of molecule s (sorted) covers the molecules of
// the cell at offset27(k), k = 13 (its own cell, the later molecules) .. 26
// (the 13 forward cells); a cell holds at most PM_CELL_MAX molecules
constexpr int PM_WORDS = 14;
constexpr int PM_CELL_MAX = 32;

// Shared-memory plan of the owner kernels (3c01, 3cw): staged positions,
// per-warp partner lists of capacity pcap (index, displacement, squared
// distance) and pair queues.
struct OwnerSmem {
    size_t off_pos, off_pos32, off_slot, off_pq, off_pd, off_pa32, off_queue, total;
};

template <typename R>
__host__ __device__ inline OwnerSmem owner_smem_plan(int mcap, int nwarps, int pcap)
{
    OwnerSmem p;
    size_t o = 0;
    auto al = [](size_t v) { return (v + 15) & ~(size_t)15; };
    const bool f64 = sizeof(R) == 8;
    p.off_pos = o;   o = al(o + sizeof(R) * 3 * (size_t)mcap);
    p.off_pos32 = o; o = al(o + (f64 ? sizeof(float) * 3 * (size_t)mcap : 0));
    p.off_slot = o;  o = al(o + (size_t)mcap);
    p.off_pq = o;    o = al(o + sizeof(unsigned short) * (size_t)pcap * nwarps);
    p.off_pd = o;    o = al(o + sizeof(R) * 4 * (size_t)pcap * nwarps);
    p.off_pa32 = o;  o = al(o + (f64 ? sizeof(float) * (size_t)pcap * nwarps : 0));
    p.off_queue = o; o = al(o + sizeof(unsigned) * 64 * (size_t)nwarps);
    p.total = o;
    return p;
}

// Shared-memory plan of the Newton-3 block kernel (3c18 / 3c08).
//  pos / sh      staged cell-local positions and exact base-frame shifts o*w
//  pos32 / sh32  their FP32 copies (FP64 path: prefilter)
//  pair rule:    adjacency bitmask rows and transpose, per-word prefix
//                popcounts, row offsets (edge numbering), third-member slot
//                masks, edge list, FP64 edge vectors (dx, dy, dz, r^2), edge
//                scalars G; the per-molecule fallback accumulators alias G
//  product rule: dense FP32 squared distances D (optional), dense G
//                (acc_mode 0) or per-molecule accumulators (acc_mode 1)
struct BlockSmem {
    int W;
    size_t off_pos, off_sh, off_pos32, off_sh32, off_idx, off_slot, off_adj, off_adjT, off_rowpre,
        off_rowoff, off_memb, off_ed, off_el, off_G, off_D, off_acc, off_queue, total;
};

template <typename R>
__host__ __device__ inline BlockSmem block_smem_plan(int trunc, int mcap, int nwarps, int gcap,
                                                     int use_d, int acc_mode, int det = 0)
{
    BlockSmem p;
    size_t o = 0;
    auto al = [](size_t v) { return (v + 15) & ~(size_t)15; };
    const bool f64 = sizeof(R) == 8, pair = trunc == 0;
    const size_t M = (size_t)mcap, npair = M * (M - 1) / 2, accb = 24 * M;
    p.W = (mcap + 31) >> 5;
    // FP64: SoA x[M], y[M], z[M]; FP32: one float4 (x, y, z, 0) per molecule
    p.off_pos = o;    o = al(o + (f64 ? sizeof(R) * 3 * M : 16 * M));
    p.off_sh = o;     o = al(o + (f64 ? sizeof(R) * 3 * M : 16 * M));
    p.off_pos32 = o;  o = al(o + (f64 ? sizeof(float) * 3 * M : 0));
    p.off_sh32 = o;   o = al(o + (f64 ? sizeof(float) * 3 * M : 0));
    p.off_idx = o;    o = al(o + (f64 ? sizeof(int) * M : 0));  // FP32: in the position rows' w
    p.off_slot = o;   o = al(o + M);
    p.off_adj = o;    o = al(o + (pair ? sizeof(unsigned) * M * p.W : 0));
    p.off_adjT = o;   o = al(o + (pair ? sizeof(unsigned) * M * p.W : 0));
    p.off_rowpre = o; o = al(o + (pair ? sizeof(unsigned short) * M * p.W : 0));
    p.off_rowoff = o; o = al(o + (pair ? sizeof(int) * (M + 1) : 0));
    p.off_memb = o;   o = al(o + (pair ? sizeof(unsigned) * 8 * p.W : 0));
    // pair rule: FP64 with use_d keeps the edge vectors (dx, dy, dz, r^2) of
    // the unit's edges (FP64 work once per edge instead of once per triangle
    // side); otherwise the triplets take the shifted rows.  Both keep the
    // edge list (p | q << 16).
    p.off_ed = o;
    o = al(o + (pair && f64 && use_d ? sizeof(R) * 4 * (size_t)gcap : 0));
    p.off_el = o;     o = al(o + (pair ? sizeof(unsigned) * (size_t)gcap : 0));
    // pair scalars: R, or 64-bit fixed point in the deterministic mode
    const size_t gsz = det ? 8 : sizeof(R);
    const size_t gb = gsz * (pair ? (size_t)gcap : (acc_mode == 0 ? npair : 0));
    p.off_G = o;      o = al(o + (pair ? (gb > accb ? gb : accb) : gb));
    p.off_D = o;      o = al(o + (!pair && use_d ? sizeof(float) * npair : 0));
    p.off_acc = pair ? p.off_G : o;  // pair rule: the fallback accumulators alias G
    o = al(o + (!pair && acc_mode == 1 ? accb : 0));
    p.off_queue = o;  o = al(o + (pair ? 0 : sizeof(unsigned long long) * 64 * (size_t)nwarps));
    p.total = o;
    return p;
}

// Launch configuration of the ATM kernels for units of at most mcap molecules.
// 3c01: 4 warps.  3c18/3c08 pair rule: 4 warps (FP32) or 8 (FP64) and pair
// scalars for gpm16 / 16 edges per staged molecule of the largest unit
// (gpm16 = 256 before any measurement: the rho* = 0.8 liquids have at most
// 14.4 (256k, fcc start) and 15.9 (32k); a context then sizes the table from
// the needs its units recorded), halved until they fit (a unit with more
// edges falls back to per-molecule accumulators);
// product rule: 8 warps (FP32 3c18: 16 when one CTA fills an SM),
// dense distances + dense pair scalars, else dense pair scalars only, else
// per-molecule accumulators.  Returns false if nothing fits.
struct AtmPlan {
    int nwarps, gcap, use_d, acc_mode, pcap;
    size_t smem;
};

// partner capacity of the wide traversal's warps (molecules within twice the
// cell edge: about 380 in a liquid at rho* = 0.8)
constexpr int ATM_WIDE_PCAP = 1024;

inline bool atm_choose_plan_nw(int trav, int trunc, int prec, int mcap, int optin, int nwarps,
                               AtmPlan& P, int det = 0, int gpm16 = 256)
{
    // the kernels' static shared memory (slot tables, reductions; under 2 KB)
    // counts against the same per-block limit as the dynamic part
    optin -= 4096;
    P.nwarps = nwarps;
    P.gcap = 0;
    P.use_d = 0;
    P.acc_mode = 0;
    P.pcap = trav == 3 ? (mcap < ATM_WIDE_PCAP ? mcap : ATM_WIDE_PCAP) : mcap;
    auto bytes = [&]() -> size_t {
        if (trav == 0 || trav == 3)
            return prec == 0 ? owner_smem_plan<double>(mcap, P.nwarps, P.pcap).total
                             : owner_smem_plan<float>(mcap, P.nwarps, P.pcap).total;
        return prec == 0
                   ? block_smem_plan<double>(trunc, mcap, P.nwarps, P.gcap, P.use_d, P.acc_mode, det).total
                   : block_smem_plan<float>(trunc, mcap, P.nwarps, P.gcap, P.use_d, P.acc_mode, det).total;
    };
    if (trav == 0 || trav == 3) {
        P.smem = bytes();
        // the wide traversal: fewer warps, then fewer partner slots, before giving up
        while (trav == 3 && P.smem > (size_t)optin && P.nwarps > 1) {
            P.nwarps /= 2;
            P.smem = bytes();
        }
        while (trav == 3 && P.smem > (size_t)optin && P.pcap > 256) {
            P.pcap /= 2;
            P.smem = bytes();
        }
        return P.smem <= (size_t)optin;
    }
    const long long npair = (long long)mcap * (mcap - 1) / 2;
    if (trunc == 0) {
        auto fit = [&](int use_d) -> bool {
            P.use_d = use_d;
            const long long cap = ((long long)gpm16 * mcap + 15) / 16;
            long long g = npair < cap ? npair : cap;
            for (;;) {
                P.gcap = (int)g;
                P.smem = bytes();
                if (P.smem <= (size_t)optin || g == 0) break;
                g /= 2;
            }
            return P.smem <= (size_t)optin;
        };
        // (the deterministic mode keeps one arithmetic for every launch form:
        // the shifted rows)
        if (prec != 0 || det) return fit(0);
        // FP64: the edge-vector table when it costs no resident CTA.  CTAs per
        // SM from shared memory (228 KB per SM, 1 KB reserved per CTA) and from
        // registers (the FP64 block kernels' cap of 128 per thread).  Measured
        // (liquids, 3c08 / 3c18 pair FP64): the 256k 3c08 units (2 CTAs either
        // way) 10.23 ms with the table, 11.97 without; the 256k 3c18 units
        // (1 CTA with it, 2 without) 16.33 and 13.27; the 32k 3c08 units 1.79
        // and 1.68.
        const bool okn = fit(0);
        const AtmPlan Pn = P;
        const bool oke = fit(1);
        const AtmPlan Pe = P;
        if (!oke || !okn) {
            P = oke ? Pe : Pn;
            return oke || okn;
        }
        const int regs = 65536 / (128 * 32 * P.nwarps);
        auto ctas = [&](size_t smem) {
            const int c = (int)(233472 / (smem + 1024));
            return c < regs ? c : regs;
        };
        P = ctas(Pe.smem) >= ctas(Pn.smem) ? Pe : Pn;
        return true;
    }
    const int modes[3][2] = {{1, 0}, {0, 0}, {0, 1}};
    for (const auto& m : modes) {
        P.use_d = m[0];
        P.acc_mode = m[1];
        P.smem = bytes();
        if (P.smem <= (size_t)optin) return true;
    }
    return false;
}

inline bool atm_choose_plan(int trav, int trunc, int prec, int mcap, int optin, AtmPlan& P,
                            int det = 0, int gpm16 = 256)
{
    if (!atm_choose_plan_nw(trav, trunc, prec, mcap, optin,
                            (trav == 0 || trav == 3 || (trunc == 0 && prec == 1)) ? 4 : 8, P, det,
                            gpm16))
        return false;
    // FP32 3c18 product rule whose tables leave room for one CTA per SM: 16
    // warps (same table mode) hide more of the scan's shared-memory latency
    if (trunc == 1 && prec == 1 && trav == 1 && 2 * P.smem > (size_t)optin) {
        AtmPlan Q;
        if (atm_choose_plan_nw(trav, trunc, prec, mcap, optin, 16, Q, det, gpm16) && Q.use_d == P.use_d &&
            Q.acc_mode == P.acc_mode)
            P = Q;
    }
    return true;
}

}  // namespace atm3

// kernel launchers (defined in atm_fp64.cu / atm_fp32.cu)
namespace atm3 {
// det != 0 selects the block kernels' deterministic instantiations (the
// owner kernels read a.det themselves)
cudaError_t launch_atm_fp64(int trav, int trunc, const AtmArgs<double>& a, int nwarps,
                            size_t smem, int ctas, cudaStream_t s);
cudaError_t launch_atm_fp32(int trav, int trunc, const AtmArgs<float>& a, int nwarps,
                            size_t smem, int ctas, cudaStream_t s);
cudaError_t atm_attr_fp64(int trav, int trunc, size_t smem, int det = 0);
cudaError_t atm_attr_fp32(int trav, int trunc, size_t smem, int det = 0);
int atm_occupancy_fp64(int trav, int trunc, int nwarps, size_t smem, int det = 0);
int atm_occupancy_fp32(int trav, int trunc, int nwarps, size_t smem, int det = 0);
// deterministic instantiations of the block kernels (atm_det64.cu / atm_det32.cu)
cudaError_t launch_block_det64(int trav, int trunc, const AtmArgs<double>& a, int nwarps,
                               size_t smem, int ctas, cudaStream_t s);
cudaError_t launch_block_det32(int trav, int trunc, const AtmArgs<float>& a, int nwarps,
                               size_t smem, int ctas, cudaStream_t s);
cudaError_t attr_block_det64(int trav, int trunc, size_t smem);
cudaError_t attr_block_det32(int trav, int trunc, size_t smem);
int occupancy_block_det64(int trav, int trunc, int nwarps, size_t smem);
int occupancy_block_det32(int trav, int trunc, int nwarps, size_t smem);
}  // namespace atm3
