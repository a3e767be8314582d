// FP64 instantiations of the ATM triplet kernels (3c01 and 3cw owner kernel,
// 3c18 / 3c08 / corner-anchored 3c08 block kernel) with floating-point sums;
// a.det selects the block kernels' deterministic instantiations (atm_det64.cu).
#include "atm_launch.cuh"

namespace atm3 {

cudaError_t launch_atm_fp64(int trav, int trunc, const AtmArgs<double>& a, int nwarps,
                            size_t smem, int ctas, cudaStream_t s)
{
    if (a.det && atm_block_trav(trav)) return launch_block_det64(trav, trunc, a, nwarps, smem, ctas, s);
    return atm_launch_t<double, false>(trav, trunc, a, nwarps, smem, ctas, s);
}

cudaError_t atm_attr_fp64(int trav, int trunc, size_t smem, int det)
{
    if (det && atm_block_trav(trav)) return attr_block_det64(trav, trunc, smem);
    return atm_attr_t<double, false>(trav, trunc, smem);
}

int atm_occupancy_fp64(int trav, int trunc, int nwarps, size_t smem, int det)
{
    if (det && atm_block_trav(trav)) return occupancy_block_det64(trav, trunc, nwarps, smem);
    return atm_occupancy_t<double, false>(trav, trunc, nwarps, smem);
}

}  // namespace atm3
