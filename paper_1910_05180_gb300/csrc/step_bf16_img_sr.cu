// BF16 storage with FP32 compute, all faces periodic, stochastic rounding of
// the update to BF16: the step kernels that also write the periodic ghost
// images of their new cells.
#include "step_kernel.cuh"
#include "tiles.h"

namespace spfm {
cudaError_t launch_step_bf16_img_sr(const StepCoef<float> &c, const __nv_bfloat16 *src, __nv_bfloat16 *dst,
                                    int *err, LaunchCfg cfg, TmaCache *tma, int which, cudaStream_t st)
{
    using Sh = TileShape<__nv_bfloat16, float, kBfTX, kBfTY>;
    const CUtensorMap *map = cached_map(tma, which, c.g, SPFM_BF16, src, Sh::SW, Sh::ROWS);
    return launch_step_t<__nv_bfloat16, float, kBfTX, kBfTY, true, true>(c, src, dst, err, cfg, map, st);
}
}  // namespace spfm
