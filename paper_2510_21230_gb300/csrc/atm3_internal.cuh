// atm3_internal.cuh -- device-side types shared by the CUDA translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace atm3 {

// device status word bits (set by kernels, read back by the host)
enum : int {
    ST_CAPACITY = 1,   // a unit stages more molecules than its shared memory holds
    ST_NONFINITE = 2,  // a non-finite position or velocity was seen
};

// Linked-cell grid (section 3): n_d cells of edge w_d = L_d / n_d per axis.
struct Grid {
    int nc[3];
    double L[3];
    double w[3];
    long long ncell;
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
//  3c18: slot 0 = base, slots 1..13 = forward neighbours in lexicographic order.
//  3c08: slot s = offset (s & 1, s >> 1 & 1, s >> 2 & 1) inside the 2x2x2 block.
template <int TRAV>
__host__ __device__ __forceinline__ void slot_offset(int s, int& dx, int& dy, int& dz)
{
    if (TRAV == 0) {
        int t = s == 0 ? 13 : (s <= 13 ? s - 1 : s);
        offset27(t, dx, dy, dz);
    } else if (TRAV == 1) {
        offset27(13 + s, dx, dy, dz);
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

// Arguments of the ATM unit kernels.
template <typename R>
struct AtmArgs {
    Grid g;
    long long n;
    const R* xl;              // sorted cell-local coordinates, SoA [3n], working precision
    const float* xl32;        // the same in FP32 (prefilter of the FP64 path)
    const int* cell_start;    // [ncell + 1]
    double* fs;               // sorted-order ATM force accumulator, SoA [3n]
    double* unit_ew;          // [2 * ncell]: E3, W3 per unit
    unsigned long long* unit_cnt;  // [2 * ncell]: candidates, interacting
    int* status;
    R w[3];                   // cell edges in the working precision
    float wf[3];              // cell edges in FP32
    R rc2, rc6, nu;
    float p_lo, p_hi;         // FP64 prefilter band of a squared distance (pair rule)
    float q_lo, q_hi, dmin;   // FP64 prefilter band of a sorted product (product rule)
    int mcap;                 // staged-molecule capacity of one unit
    int gcap;                 // edge-accumulator capacity (block kernel)
    int use_d;                // block kernel, product rule: dense FP32 distance table in smem
};

// Shared-memory plan of the 3c01 (owner) kernel: staged positions, per-warp
// partner lists (index, displacement, squared distance) and pair queues.
struct OwnerSmem {
    size_t off_pos, off_pos32, off_slot, off_pq, off_pd, off_pa32, off_queue, total;
};

template <typename R>
__host__ __device__ inline OwnerSmem owner_smem_plan(int mcap, int nwarps)
{
    OwnerSmem p;
    size_t o = 0;
    auto al = [](size_t v) { return (v + 15) & ~(size_t)15; };
    const bool f64 = sizeof(R) == 8;
    p.off_pos = o;   o = al(o + sizeof(R) * 3 * (size_t)mcap);
    p.off_pos32 = o; o = al(o + (f64 ? sizeof(float) * 3 * (size_t)mcap : 0));
    p.off_slot = o;  o = al(o + (size_t)mcap);
    p.off_pq = o;    o = al(o + sizeof(unsigned short) * (size_t)mcap * nwarps);
    p.off_pd = o;    o = al(o + sizeof(R) * 4 * (size_t)mcap * nwarps);
    p.off_pa32 = o;  o = al(o + (f64 ? sizeof(float) * (size_t)mcap * nwarps : 0));
    p.off_queue = o; o = al(o + sizeof(unsigned) * 64 * (size_t)nwarps);
    p.total = o;
    return p;
}

// Shared-memory plan of the Newton-3 block kernel (3c18 / 3c08).
struct BlockSmem {
    int W;
    size_t off_pos, off_pos32, off_idx, off_slot, off_adj, off_adjT, off_rowoff, off_memb, off_G,
        off_D, off_plq, off_queue, total;
};

template <typename R>
__host__ __device__ inline BlockSmem block_smem_plan(int trunc, int mcap, int nwarps, int gcap,
                                                     int use_d)
{
    BlockSmem p;
    size_t o = 0;
    auto al = [](size_t v) { return (v + 15) & ~(size_t)15; };
    const bool f64 = sizeof(R) == 8, pair = trunc == 0;
    const size_t M = (size_t)mcap, npair = M * (M - 1) / 2;
    p.W = (mcap + 31) >> 5;
    p.off_pos = o;    o = al(o + sizeof(R) * 3 * M);
    p.off_pos32 = o;  o = al(o + (f64 ? sizeof(float) * 3 * M : 0));
    p.off_idx = o;    o = al(o + sizeof(int) * M);
    p.off_slot = o;   o = al(o + M);
    p.off_adj = o;    o = al(o + (pair ? sizeof(unsigned) * M * p.W : 0));
    p.off_adjT = o;   o = al(o + (pair ? sizeof(unsigned) * M * p.W : 0));
    p.off_rowoff = o; o = al(o + (pair ? sizeof(int) * (M + 1) : 0));
    p.off_memb = o;   o = al(o + (pair ? sizeof(unsigned) * 8 * p.W : 0));
    p.off_G = o;      o = al(o + sizeof(R) * (pair ? (size_t)gcap : npair));
    p.off_D = o;      o = al(o + (!pair && use_d ? sizeof(float) * npair : 0));
    p.off_plq = o;    o = al(o + (pair ? sizeof(unsigned short) * M * nwarps : 0));
    p.off_queue = o;  o = al(o + sizeof(unsigned long long) * 64 * (size_t)nwarps);
    p.total = o;
    return p;
}

}  // namespace atm3

// kernel launchers (defined in atm_fp64.cu / atm_fp32.cu)
namespace atm3 {
cudaError_t launch_atm_fp64(int trav, int trunc, const AtmArgs<double>& a, int nwarps,
                            size_t smem, cudaStream_t s);
cudaError_t launch_atm_fp32(int trav, int trunc, const AtmArgs<float>& a, int nwarps,
                            size_t smem, cudaStream_t s);
cudaError_t atm_attr_fp64(int trav, int trunc, size_t smem);
cudaError_t atm_attr_fp32(int trav, int trunc, size_t smem);
}  // namespace atm3
