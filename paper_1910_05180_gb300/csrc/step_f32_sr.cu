// FP32 storage, FP32 (packed f32x2) compute, stochastic rounding of the
// update (SPFM_ROUND_STOCHASTIC): the single-grid step kernels without
// periodic images, and the persistent batch kernels of both tile shapes.
#include "step_kernel.cuh"
#include "tiles.h"

namespace spfm {
cudaError_t launch_step_f32_sr(const StepCoef<float> &c, const float *src, float *dst, int *err, LaunchCfg cfg,
                               TmaCache *tma, int which, cudaStream_t st)
{
    using Sh = TileShape<float, float, SPFM_F32_TX, SPFM_F32_TY>;
    const CUtensorMap *map = cached_map(tma, which, c.g, SPFM_F32, src, Sh::SW, Sh::ROWS);
    return launch_step_t<float, float, SPFM_F32_TX, SPFM_F32_TY, false, true>(c, src, dst, err, cfg, map, st);
}

cudaError_t launch_batch_f32_sr(const void *grids, const BatchItem *work, int nwork, int parity, int *err,
                                int stencil, int kind, cudaStream_t st, int shape, const long long *steps, int sub,
                                int fwd)
{
    if (shape == 1)
        return launch_batch_t<float, float, kSqTX, kSqTY, true, true>(grids, work, nwork, parity, err, stencil,
                                                                       kind, st, steps, sub, fwd);
    return launch_batch_t<float, float, SPFM_F32_TX, SPFM_F32_TY, false, true>(grids, work, nwork, parity, err,
                                                                               stencil, kind, st, steps, sub, fwd);
}
}  // namespace spfm
