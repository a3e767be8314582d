// pair_masks.cu -- pair bitmaps of the FP32C pair rule (k_pair_masks): every
// pair of a molecule with the later molecules of its cell and the molecules of
// its 13 forward cells decided once per force evaluation, for the block
// traversals' units to assemble their adjacency from.
#include "md_kernels.cuh"

namespace atm3 {

// Pair bitmaps (see launch_pair_masks): one thread per (molecule, offset);
// the threads of a warp share a cell and an offset, so the neighbour rows
// they read are broadcast loads, and each offset's words are written by
// consecutive threads.  The arithmetic is the block kernels' decision term by
// term: (xl_t - xl_s) + delta w per component, delta w exact for
// |delta| <= 1, squares summed x, y, z, compared with the FP32 r_c^2.
__global__ void __launch_bounds__(128) k_pair_masks(Batch B, const int* __restrict__ start,
                                                    const float* __restrict__ xl32,
                                                    const int* __restrict__ cell_sorted,
                                                    unsigned* __restrict__ pm,
                                                    int* __restrict__ status)
{
    const long long n = B.ntot;
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int k = 13 + (int)blockIdx.y;  // the cell itself, then the 13 forward cells
    if (s >= n) return;
    const int c = cell_sorted[s];
    const Rep& rp = B.rep[B.rep_of_cell[c]];
    const int nx = rp.g.nc[0], ny = rp.g.nc[1], nz = rp.g.nc[2];
    const int id = (int)(c - rp.cell0);  // below 2^30
    const int cx = id % nx, cyz = id / nx, cy = cyz % ny, cz = cyz / ny;
    int dx, dy, dz;
    offset27(k, dx, dy, dz);
    int x = cx + dx, y = cy + dy, z = cz + dz;
    x = x < 0 ? x + nx : (x >= nx ? x - nx : x);
    y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
    z = z < 0 ? z + nz : (z >= nz ? z - nz : z);
    const long long c2 = rp.cell0 + ((long long)z * ny + y) * nx + x;
    const int t0 = start[c2], t1 = start[c2 + 1];
    unsigned word = 0u;
    if (t1 - t0 > PM_CELL_MAX) {
        atomicOr(status, ST_CAPACITY);
    } else {
        const float xs = xl32[s], ys = xl32[n + s], zs = xl32[2 * n + s];
        const float sx = __fmul_rn((float)dx, rp.wf[0]);
        const float sy = __fmul_rn((float)dy, rp.wf[1]);
        const float sz = __fmul_rn((float)dz, rp.wf[2]);
        const float rc2 = rp.rc2f;
        // own cell: the later molecules only
#pragma unroll 4
        for (int t = k == 13 ? (int)s + 1 : t0; t < t1; t++) {
            const float ex = __fadd_rn(__fsub_rn(xl32[t], xs), sx);
            const float ey = __fadd_rn(__fsub_rn(xl32[n + t], ys), sy);
            const float ez = __fadd_rn(__fsub_rn(xl32[2 * n + t], zs), sz);
            const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)), __fmul_rn(ez, ez));
            if (d2 < rc2) word |= 1u << (t - t0);
        }
    }
    pm[(long long)(k - 13) * n + s] = word;
}

cudaError_t launch_pair_masks(const Batch& b, const int* start, const float* xl32,
                              const int* cell_sorted, unsigned* pm, int* status, cudaStream_t st)
{
    if (b.ntot <= 0) return cudaSuccess;
    const dim3 grid((unsigned)((b.ntot + 127) / 128), PM_WORDS);
    k_pair_masks<<<grid, 128, 0, st>>>(b, start, xl32, cell_sorted, pm, status);
    return cudaGetLastError();
}

}  // namespace atm3
