// FP64 storage and compute: instantiations of the step kernel.
#include "step_kernel.cuh"

namespace spfm {
cudaError_t launch_step_f64(const StepCoef<double> &c, const double *src, double *dst,
                            LaunchCfg cfg, cudaStream_t st)
{
    return launch_step_t<double, double, 16, 16>(c, src, dst, cfg, st);
}
}  // namespace spfm
