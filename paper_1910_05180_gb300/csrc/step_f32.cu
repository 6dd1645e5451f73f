// FP32 storage, FP32 (packed f32x2) compute: instantiations of the step kernel.
#include "step_kernel.cuh"

// tile of the FP32 kernel: SPFM_F32_TX threads of 4 cells in x, SPFM_F32_TY rows
#ifndef SPFM_F32_TX
#define SPFM_F32_TX 16
#endif
#ifndef SPFM_F32_TY
#define SPFM_F32_TY 16
#endif

namespace spfm {
cudaError_t launch_step_f32(const StepCoef<float> &c, const float *src, float *dst, int *err,
                            LaunchCfg cfg, TmaCache *tma, int which, cudaStream_t st)
{
    using Sh = TileShape<float, float, SPFM_F32_TX, SPFM_F32_TY>;
    const CUtensorMap *map = cached_map(tma, which, c.g, SPFM_F32, src, Sh::SW, Sh::ROWS);
    return launch_step_t<float, float, SPFM_F32_TX, SPFM_F32_TY>(c, src, dst, err, cfg, map, st);
}
}  // namespace spfm
