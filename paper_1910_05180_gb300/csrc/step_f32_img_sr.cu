// FP32 storage, FP32 (packed f32x2) compute, all faces periodic, stochastic
// rounding of the update: the step kernels that also write the periodic ghost
// images of their new cells.
#include "step_kernel.cuh"
#include "tiles.h"

namespace spfm {
cudaError_t launch_step_f32_img_sr(const StepCoef<float> &c, const float *src, float *dst, int *err,
                                   LaunchCfg cfg, TmaCache *tma, int which, cudaStream_t st)
{
    using Sh = TileShape<float, float, SPFM_F32_TX, SPFM_F32_TY>;
    const CUtensorMap *map = cached_map(tma, which, c.g, SPFM_F32, src, Sh::SW, Sh::ROWS);
    return launch_step_t<float, float, SPFM_F32_TX, SPFM_F32_TY, true, true>(c, src, dst, err, cfg, map, st);
}
}  // namespace spfm
