// BF16 storage with FP32 compute, all faces periodic: the step kernels that
// also write the periodic ghost images of their new cells.
#include "step_kernel.cuh"
#include "tiles.h"

namespace spfm {
cudaError_t launch_step_bf16_img(const StepCoef<float> &c, const __nv_bfloat16 *src, __nv_bfloat16 *dst,
                                 int *err, LaunchCfg cfg, TmaCache *tma, int which, cudaStream_t st)
{
    if (cfg.rounding == SPFM_ROUND_STOCHASTIC) return launch_step_bf16_img_sr(c, src, dst, err, cfg, tma, which, st);
    using Sh = TileShape<__nv_bfloat16, float, kBfTX, kBfTY>;
    const CUtensorMap *map = cached_map(tma, which, c.g, SPFM_BF16, src, Sh::SW, Sh::ROWS);
    return launch_step_t<__nv_bfloat16, float, kBfTX, kBfTY, true>(c, src, dst, err, cfg, map, st);
}
}  // namespace spfm
