// FP64 instantiations of the ATM unit kernel.
#include "atm_kernels.cuh"

namespace atm3 {
cudaError_t launch_atm_fp64(int trav, int trunc, const AtmArgs<double>& a, int nwarps,
                            size_t smem, cudaStream_t s)
{
    return launch_atm_t<double>(trav, trunc, a, nwarps, smem, s);
}
cudaError_t atm_attr_fp64(int trav, int trunc, size_t smem)
{
    return atm_attr_t<double>(trav, trunc, smem);
}
}  // namespace atm3
