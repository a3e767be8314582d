// atm_launch.cuh -- launch, shared-memory attribute and occupancy of the ATM
// triplet kernels of one working precision R and accumulation mode DET.
// Each of atm_fp32.cu, atm_fp64.cu (floating-point sums; owner and block
// kernels) and atm_det32.cu, atm_det64.cu (the block kernels' deterministic
// instantiations) includes it once, so the instantiations compile in parallel.
#pragma once
#include <mutex>

#include "atm_block.cuh"
#include "atm_owner.cuh"

namespace atm3 {

template <typename R>
using AtmKernel = void (*)(const AtmArgs<R>);

// the kernel of (traversal, truncation); owner kernels (3c01, 3cw) only in
// the floating-point instantiation (they are deterministic by a flag)
template <typename R, bool DET>
AtmKernel<R> atm_kernel(int trav, int trunc)
{
    if constexpr (!DET) {
        if (trav == 0 && trunc == 0) return atm_owner_kernel<0, 0, R>;
        if (trav == 0 && trunc == 1) return atm_owner_kernel<0, 1, R>;
        if (trav == 3 && trunc == 0) return atm_owner_kernel<3, 0, R>;
        if (trav == 3 && trunc == 1) return atm_owner_kernel<3, 1, R>;
    }
    if (trav == 1 && trunc == 0) return atm_block_kernel<1, 0, R, DET>;
    if (trav == 1 && trunc == 1) return atm_block_kernel<1, 1, R, DET>;
    if (trav == 2 && trunc == 0) return atm_block_kernel<2, 0, R, DET>;
    if (trav == 2 && trunc == 1) return atm_block_kernel<2, 1, R, DET>;
    if (trav == 4 && trunc == 0) return atm_block_kernel<4, 0, R, DET>;
    if (trav == 4 && trunc == 1) return atm_block_kernel<4, 1, R, DET>;
    return nullptr;
}

// ctas = 0: one CTA per unit; ctas > 0: a persistent grid of that many CTAs
// taking units from the counter a.work (which must be zero at launch)
template <typename R, bool DET>
cudaError_t atm_launch_t(int trav, int trunc, const AtmArgs<R>& a, int nwarps, size_t smem,
                         int ctas, cudaStream_t s)
{
    if (a.b.ncell == 0) return cudaSuccess;
    const AtmKernel<R> k = atm_kernel<R, DET>(trav, trunc);
    if (!k) return cudaErrorInvalidValue;
    dim3 grid(ctas > 0 ? (unsigned)ctas : (unsigned)a.b.ncell), block(32 * nwarps);
    k<<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
}

// The shared-memory limit is an attribute of the kernel for the whole
// process (per device), so contexts of different unit sizes share it: it is
// only ever raised, never set below the largest plan any context launched.
template <typename R, bool DET>
cudaError_t atm_attr_t(int trav, int trunc, size_t smem)
{
    static std::mutex mu;
    static size_t done[ATM_MAX_DEVICES][ATM_NTRAV][2] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= ATM_MAX_DEVICES || trav < 0 || trav >= ATM_NTRAV || trunc < 0 || trunc > 1)
        return cudaErrorInvalidValue;
    const AtmKernel<R> k = atm_kernel<R, DET>(trav, trunc);
    if (!k) return cudaErrorInvalidValue;
    std::lock_guard<std::mutex> lock(mu);
    if (smem <= done[dev][trav][trunc]) return cudaSuccess;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) done[dev][trav][trunc] = smem;
    return e;
}

// resident CTAs per SM of the kernel at this block size and shared memory
// (the kernel's dynamic shared-memory limit is raised to smem first: below
// it the query answers 0, and the answer would depend on which launches came
// before)
template <typename R, bool DET>
int atm_occupancy_t(int trav, int trunc, int nwarps, size_t smem)
{
    const AtmKernel<R> k = atm_kernel<R, DET>(trav, trunc);
    int nb = 0;
    if (k && atm_attr_t<R, DET>(trav, trunc, smem) == cudaSuccess)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, 32 * nwarps, smem);
    return nb;
}

// the block traversals (3c18, 3c08, corner-anchored 3c08) have deterministic
// instantiations
inline bool atm_block_trav(int trav) { return trav == 1 || trav == 2 || trav == 4; }

}  // namespace atm3
