// FP32 instantiations of the ATM triplet kernels (3c01 and 3cw owner kernel,
// 3c18 / 3c08 / corner-anchored 3c08 block kernel) with floating-point sums;
// a.det selects the block kernels' deterministic instantiations (atm_det32.cu).
#include "atm_launch.cuh"

namespace atm3 {

cudaError_t launch_atm_fp32(int trav, int trunc, const AtmArgs<float>& a, int nwarps,
                            size_t smem, int ctas, cudaStream_t s)
{
    if (a.det && atm_block_trav(trav)) return launch_block_det32(trav, trunc, a, nwarps, smem, ctas, s);
    return atm_launch_t<float, false>(trav, trunc, a, nwarps, smem, ctas, s);
}

cudaError_t atm_attr_fp32(int trav, int trunc, size_t smem, int det)
{
    if (det && atm_block_trav(trav)) return attr_block_det32(trav, trunc, smem);
    return atm_attr_t<float, false>(trav, trunc, smem);
}

int atm_occupancy_fp32(int trav, int trunc, int nwarps, size_t smem, int det)
{
    if (det && atm_block_trav(trav)) return occupancy_block_det32(trav, trunc, nwarps, smem);
    return atm_occupancy_t<float, false>(trav, trunc, nwarps, smem);
}

}  // namespace atm3
