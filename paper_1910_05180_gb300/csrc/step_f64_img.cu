// FP64 storage and compute, all faces periodic: the step kernels that also
// write the periodic ghost images of their new cells.
#include "step_kernel.cuh"

namespace spfm {
cudaError_t launch_step_f64_img(const StepCoef<double> &c, const double *src, double *dst, int *err,
                                LaunchCfg cfg, TmaCache *tma, int which, cudaStream_t st)
{
    using Sh = TileShape<double, double, 16, 16>;
    const CUtensorMap *map = cached_map(tma, which, c.g, SPFM_F64, src, Sh::SW, Sh::ROWS);
    return launch_step_t<double, double, 16, 16, true>(c, src, dst, err, cfg, map, st);
}
}  // namespace spfm
