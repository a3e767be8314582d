// FP32 (compensated) instantiations of the ATM unit kernel.
#include "atm_kernels.cuh"

namespace atm3 {
cudaError_t launch_atm_fp32(int trav, int trunc, const AtmArgs<float>& a, int nwarps,
                            size_t smem, cudaStream_t s)
{
    return launch_atm_t<float>(trav, trunc, a, nwarps, smem, s);
}
cudaError_t atm_attr_fp32(int trav, int trunc, size_t smem)
{
    return atm_attr_t<float>(trav, trunc, smem);
}
}  // namespace atm3
