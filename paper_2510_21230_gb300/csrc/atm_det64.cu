// Deterministic FP64 instantiations of the block kernels (3c18, 3c08,
// corner-anchored 3c08): fixed-point sums and a fixed work order.
#include "atm_launch.cuh"

namespace atm3 {

cudaError_t launch_block_det64(int trav, int trunc, const AtmArgs<double>& a, int nwarps,
                               size_t smem, int ctas, cudaStream_t s)
{
    return atm_launch_t<double, true>(trav, trunc, a, nwarps, smem, ctas, s);
}

cudaError_t attr_block_det64(int trav, int trunc, size_t smem)
{
    return atm_attr_t<double, true>(trav, trunc, smem);
}

int occupancy_block_det64(int trav, int trunc, int nwarps, size_t smem)
{
    return atm_occupancy_t<double, true>(trav, trunc, nwarps, smem);
}

}  // namespace atm3
