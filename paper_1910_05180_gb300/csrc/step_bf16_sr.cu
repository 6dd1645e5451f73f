// BF16 storage with FP32 compute, stochastic rounding of the update to BF16
// (SPFM_ROUND_STOCHASTIC): the single-grid step kernels without periodic
// images, and the persistent batch kernel.
#include "step_kernel.cuh"
#include "tiles.h"

namespace spfm {
cudaError_t launch_step_bf16_sr(const StepCoef<float> &c, const __nv_bfloat16 *src, __nv_bfloat16 *dst,
                                int *err, LaunchCfg cfg, TmaCache *tma, int which, cudaStream_t st)
{
    using Sh = TileShape<__nv_bfloat16, float, kBfTX, kBfTY>;
    const CUtensorMap *map = cached_map(tma, which, c.g, SPFM_BF16, src, Sh::SW, Sh::ROWS);
    return launch_step_t<__nv_bfloat16, float, kBfTX, kBfTY, false, true>(c, src, dst, err, cfg, map, st);
}

cudaError_t launch_batch_bf16_sr(const void *grids, const BatchItem *work, int nwork, int parity, int *err,
                                 int stencil, int kind, cudaStream_t st, const long long *steps, int sub, int fwd)
{
    return launch_batch_t<__nv_bfloat16, float, kBfTX, kBfTY, false, true>(grids, work, nwork, parity, err,
                                                                           stencil, kind, st, steps, sub, fwd);
}
}  // namespace spfm
