// FP32 storage, FP32 (packed f32x2) compute: instantiations of the step kernel.
#include "step_kernel.cuh"
#include "tiles.h"

namespace spfm {
cudaError_t launch_step_f32(const StepCoef<float> &c, const float *src, float *dst, int *err,
                            LaunchCfg cfg, TmaCache *tma, int which, cudaStream_t st)
{
    if (cfg.mode & kImages) return launch_step_f32_img(c, src, dst, err, cfg, tma, which, st);
    if (cfg.rounding == SPFM_ROUND_STOCHASTIC) return launch_step_f32_sr(c, src, dst, err, cfg, tma, which, st);
    using Sh = TileShape<float, float, SPFM_F32_TX, SPFM_F32_TY>;
    const CUtensorMap *map = cached_map(tma, which, c.g, SPFM_F32, src, Sh::SW, Sh::ROWS);
    return launch_step_t<float, float, SPFM_F32_TX, SPFM_F32_TY, false>(c, src, dst, err, cfg, map, st);
}

size_t batch_grid_bytes_f32() { return sizeof(BatchGrid<float>); }

int batch_items_f32(const GridGeom &g, int grid_index, int zchunk, BatchItem *out, int shape)
{
    if (shape == 1) return batch_items_t<float, float, kSqTX, kSqTY>(g, grid_index, zchunk, out, 1);
    return batch_items_t<float, float, SPFM_F32_TX, SPFM_F32_TY>(g, grid_index, zchunk, out, 0);
}

void batch_fill_grid_f32(void *slot, const StepCoef<float> &c, void *const field[2], int cur,
                          TmaCache *tma)
{
    using Sh = TileShape<float, float, SPFM_F32_TX, SPFM_F32_TY>;
    BatchGrid<float> *b = (BatchGrid<float> *)slot;
    b->C = c;
    b->PC = make_pack_coef<float>(c);
    b->field[0] = field[0];
    b->field[1] = field[1];
    b->cur = cur;
    const CUtensorMap *m0 = cached_map(tma, 0, c.g, SPFM_F32, field[0], Sh::SW, Sh::ROWS);
    const CUtensorMap *m1 = cached_map(tma, 1, c.g, SPFM_F32, field[1], Sh::SW, Sh::ROWS);
    b->has_map = (m0 && m1) ? 1 : 0;
    if (b->has_map) {
        b->map[0] = *m0;
        b->map[1] = *m1;
    }
    using Sq = TileShape<float, float, kSqTX, kSqTY>;
    const CUtensorMap *q0 = cached_map(tma, 2, c.g, SPFM_F32, field[0], Sq::SW, Sq::ROWS);
    const CUtensorMap *q1 = cached_map(tma, 3, c.g, SPFM_F32, field[1], Sq::SW, Sq::ROWS);
    b->has_map_sq = (q0 && q1) ? 1 : 0;
    if (b->has_map_sq) {
        b->map_sq[0] = *q0;
        b->map_sq[1] = *q1;
    }
}

cudaError_t launch_batch_f32(const void *grids, const BatchItem *work, int nwork, int parity,
                              int *err, int stencil, int kind, cudaStream_t st, int shape, int sr,
                              const long long *steps, int sub, int fwd)
{
    if (sr) return launch_batch_f32_sr(grids, work, nwork, parity, err, stencil, kind, st, shape, steps, sub, fwd);
    if (shape == 1)
        return launch_batch_t<float, float, kSqTX, kSqTY, true>(grids, work, nwork, parity, err, stencil, kind, st,
                                                                 nullptr, 0, fwd);
    return launch_batch_t<float, float, SPFM_F32_TX, SPFM_F32_TY>(grids, work, nwork, parity, err, stencil, kind, st,
                                                                   nullptr, 0, fwd);
}
}  // namespace spfm
