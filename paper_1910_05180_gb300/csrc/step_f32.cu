// FP32 storage, FP32 (packed f32x2) compute: instantiations of the step kernel.
#include "step_kernel.cuh"

namespace spfm {
cudaError_t launch_step_f32(const StepCoef<float> &c, const float *src, float *dst, LaunchCfg cfg,
                            cudaStream_t st)
{
    return launch_step_t<float, float, 16, 16>(c, src, dst, cfg, st);
}
}  // namespace spfm
