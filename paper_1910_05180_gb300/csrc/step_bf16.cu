// BF16 storage with FP32 compute: instantiations of the step kernel.
#include "step_kernel.cuh"

namespace spfm {
cudaError_t launch_step_bf16(const StepCoef<float> &c, const __nv_bfloat16 *src,
                             __nv_bfloat16 *dst, LaunchCfg cfg, cudaStream_t st)
{
    return launch_step_t<__nv_bfloat16, float, 8, 16>(c, src, dst, cfg, st);
}
}  // namespace spfm
