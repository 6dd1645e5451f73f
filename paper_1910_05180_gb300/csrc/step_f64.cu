// FP64 storage and compute: instantiations of the step kernel.
#include "step_kernel.cuh"

namespace spfm {
cudaError_t launch_step_f64(const StepCoef<double> &c, const double *src, double *dst, int *err,
                            LaunchCfg cfg, TmaCache *tma, int which, cudaStream_t st)
{
    if (cfg.mode & kImages) return launch_step_f64_img(c, src, dst, err, cfg, tma, which, st);
    using Sh = TileShape<double, double, 16, 16>;
    const CUtensorMap *map = cached_map(tma, which, c.g, SPFM_F64, src, Sh::SW, Sh::ROWS);
    return launch_step_t<double, double, 16, 16, false>(c, src, dst, err, cfg, map, st);
}

size_t batch_grid_bytes_f64() { return sizeof(BatchGrid<double>); }

int batch_items_f64(const GridGeom &g, int grid_index, int zchunk, BatchItem *out, int)
{
    return batch_items_t<double, double, 16, 16>(g, grid_index, zchunk, out, 0);
}

void batch_fill_grid_f64(void *slot, const StepCoef<double> &c, void *const field[2], int cur,
                          TmaCache *tma)
{
    using Sh = TileShape<double, double, 16, 16>;
    BatchGrid<double> *b = (BatchGrid<double> *)slot;
    b->C = c;
    b->PC = make_pack_coef<double>(c);
    b->field[0] = field[0];
    b->field[1] = field[1];
    b->cur = cur;
    const CUtensorMap *m0 = cached_map(tma, 0, c.g, SPFM_F64, field[0], Sh::SW, Sh::ROWS);
    const CUtensorMap *m1 = cached_map(tma, 1, c.g, SPFM_F64, field[1], Sh::SW, Sh::ROWS);
    b->has_map = (m0 && m1) ? 1 : 0;
    if (b->has_map) {
        b->map[0] = *m0;
        b->map[1] = *m1;
    }
    b->has_map_sq = 0;
}

cudaError_t launch_batch_f64(const void *grids, const BatchItem *work, int nwork, int parity,
                              int *err, int stencil, int kind, cudaStream_t st, int fwd)
{
    return launch_batch_t<double, double, 16, 16>(grids, work, nwork, parity, err, stencil, kind, st, nullptr, 0,
                                                  fwd);
}
}  // namespace spfm
