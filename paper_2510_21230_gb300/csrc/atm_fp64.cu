// FP64 instantiations of the ATM triplet kernels (3c01 owner kernel,
// 3c18 / 3c08 / corner-anchored 3c08 block kernel).
#include <mutex>

#include "atm_block.cuh"
#include "atm_owner.cuh"

namespace atm3 {

// ctas = 0: one CTA per unit; ctas > 0: a persistent grid of that many CTAs
// taking units from the counter a.work (which must be zero at launch)
cudaError_t launch_atm_fp64(int trav, int trunc, const AtmArgs<double>& a, int nwarps,
                            size_t smem, int ctas, cudaStream_t s)
{
    if (a.b.ncell == 0) return cudaSuccess;
    dim3 grid(ctas > 0 ? (unsigned)ctas : (unsigned)a.b.ncell), block(32 * nwarps);
    if (trav == 0 && trunc == 0) atm_owner_kernel<0, 0, double><<<grid, block, smem, s>>>(a);
    else if (trav == 3 && trunc == 0) atm_owner_kernel<3, 0, double><<<grid, block, smem, s>>>(a);
    else if (trav == 3 && trunc == 1) atm_owner_kernel<3, 1, double><<<grid, block, smem, s>>>(a);
    else if (trav == 0 && trunc == 1) atm_owner_kernel<0, 1, double><<<grid, block, smem, s>>>(a);
    else if (trav == 1 && trunc == 0) atm_block_kernel<1, 0, double><<<grid, block, smem, s>>>(a);
    else if (trav == 1 && trunc == 1) atm_block_kernel<1, 1, double><<<grid, block, smem, s>>>(a);
    else if (trav == 2 && trunc == 0) atm_block_kernel<2, 0, double><<<grid, block, smem, s>>>(a);
    else if (trav == 4 && trunc == 0) atm_block_kernel<4, 0, double><<<grid, block, smem, s>>>(a);
    else if (trav == 2 && trunc == 1) atm_block_kernel<2, 1, double><<<grid, block, smem, s>>>(a);
    else if (trav == 4 && trunc == 1) atm_block_kernel<4, 1, double><<<grid, block, smem, s>>>(a);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

// the shared-memory limit is an attribute of the kernel for the whole
// process (per device), so contexts of different unit sizes share it: it is
// only ever raised, never set below the largest plan any context launched
static cudaError_t set_attr_fp64(int trav, int trunc, size_t smem);

cudaError_t atm_attr_fp64(int trav, int trunc, size_t smem)
{
    static std::mutex mu;
    static size_t done[ATM_MAX_DEVICES][ATM_NTRAV][2] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= ATM_MAX_DEVICES || trav < 0 || trav >= ATM_NTRAV || trunc < 0 || trunc > 1)
        return cudaErrorInvalidValue;
    std::lock_guard<std::mutex> lock(mu);
    if (smem <= done[dev][trav][trunc]) return cudaSuccess;
    e = set_attr_fp64(trav, trunc, smem);
    if (e == cudaSuccess) done[dev][trav][trunc] = smem;
    return e;
}

static cudaError_t set_attr_fp64(int trav, int trunc, size_t smem)
{
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if (trav == 0 && trunc == 0) return cudaFuncSetAttribute(atm_owner_kernel<0, 0, double>, A, (int)smem);
    if (trav == 3 && trunc == 0) return cudaFuncSetAttribute(atm_owner_kernel<3, 0, double>, A, (int)smem);
    if (trav == 3 && trunc == 1) return cudaFuncSetAttribute(atm_owner_kernel<3, 1, double>, A, (int)smem);
    if (trav == 0 && trunc == 1) return cudaFuncSetAttribute(atm_owner_kernel<0, 1, double>, A, (int)smem);
    if (trav == 1 && trunc == 0) return cudaFuncSetAttribute(atm_block_kernel<1, 0, double>, A, (int)smem);
    if (trav == 1 && trunc == 1) return cudaFuncSetAttribute(atm_block_kernel<1, 1, double>, A, (int)smem);
    if (trav == 2 && trunc == 0) return cudaFuncSetAttribute(atm_block_kernel<2, 0, double>, A, (int)smem);
    if (trav == 4 && trunc == 0) return cudaFuncSetAttribute(atm_block_kernel<4, 0, double>, A, (int)smem);
    if (trav == 2 && trunc == 1) return cudaFuncSetAttribute(atm_block_kernel<2, 1, double>, A, (int)smem);
    if (trav == 4 && trunc == 1) return cudaFuncSetAttribute(atm_block_kernel<4, 1, double>, A, (int)smem);
    return cudaErrorInvalidValue;
}

// resident CTAs per SM of the kernel at this block size and shared memory
int atm_occupancy_fp64(int trav, int trunc, int nwarps, size_t smem)
{
    int nb = 0;
    const int bs = 32 * nwarps;
    if (trav == 0 && trunc == 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, atm_owner_kernel<0, 0, double>, bs, smem);
    else if (trav == 3 && trunc == 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, atm_owner_kernel<3, 0, double>, bs, smem);
    else if (trav == 3 && trunc == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, atm_owner_kernel<3, 1, double>, bs, smem);
    else if (trav == 0 && trunc == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, atm_owner_kernel<0, 1, double>, bs, smem);
    else if (trav == 1 && trunc == 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, atm_block_kernel<1, 0, double>, bs, smem);
    else if (trav == 1 && trunc == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, atm_block_kernel<1, 1, double>, bs, smem);
    else if (trav == 2 && trunc == 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, atm_block_kernel<2, 0, double>, bs, smem);
    else if (trav == 4 && trunc == 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, atm_block_kernel<4, 0, double>, bs, smem);
    else if (trav == 2 && trunc == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, atm_block_kernel<2, 1, double>, bs, smem);
    else if (trav == 4 && trunc == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, atm_block_kernel<4, 1, double>, bs, smem);
    return nb;
}

}  // namespace atm3
