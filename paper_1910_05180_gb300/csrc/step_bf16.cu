// BF16 storage with FP32 compute: instantiations of the step kernel.
#include "step_kernel.cuh"
#include "tiles.h"

namespace spfm {
cudaError_t launch_step_bf16(const StepCoef<float> &c, const __nv_bfloat16 *src, __nv_bfloat16 *dst, int *err,
                            LaunchCfg cfg, TmaCache *tma, int which, cudaStream_t st)
{
    if (cfg.mode & kImages) return launch_step_bf16_img(c, src, dst, err, cfg, tma, which, st);
    if (cfg.rounding == SPFM_ROUND_STOCHASTIC) return launch_step_bf16_sr(c, src, dst, err, cfg, tma, which, st);
    using Sh = TileShape<__nv_bfloat16, float, kBfTX, kBfTY>;
    const CUtensorMap *map = cached_map(tma, which, c.g, SPFM_BF16, src, Sh::SW, Sh::ROWS);
    return launch_step_t<__nv_bfloat16, float, kBfTX, kBfTY, false>(c, src, dst, err, cfg, map, st);
}

size_t batch_grid_bytes_bf16() { return sizeof(BatchGrid<float>); }

int batch_items_bf16(const GridGeom &g, int grid_index, int zchunk, BatchItem *out, int)
{
    return batch_items_t<__nv_bfloat16, float, kBfTX, kBfTY>(g, grid_index, zchunk, out, 0);
}

void batch_fill_grid_bf16(void *slot, const StepCoef<float> &c, void *const field[2], int cur,
                          TmaCache *tma)
{
    using Sh = TileShape<__nv_bfloat16, float, kBfTX, kBfTY>;
    BatchGrid<float> *b = (BatchGrid<float> *)slot;
    b->C = c;
    b->PC = make_pack_coef<float>(c);
    b->field[0] = field[0];
    b->field[1] = field[1];
    b->cur = cur;
    const CUtensorMap *m0 = cached_map(tma, 0, c.g, SPFM_BF16, field[0], Sh::SW, Sh::ROWS);
    const CUtensorMap *m1 = cached_map(tma, 1, c.g, SPFM_BF16, field[1], Sh::SW, Sh::ROWS);
    b->has_map = (m0 && m1) ? 1 : 0;
    if (b->has_map) {
        b->map[0] = *m0;
        b->map[1] = *m1;
    }
    b->has_map_sq = 0;
}

cudaError_t launch_batch_bf16(const void *grids, const BatchItem *work, int nwork, int parity,
                              int *err, int stencil, int kind, cudaStream_t st, int sr, const long long *steps,
                              int sub, int fwd)
{
    if (sr) return launch_batch_bf16_sr(grids, work, nwork, parity, err, stencil, kind, st, steps, sub, fwd);
    return launch_batch_t<__nv_bfloat16, float, kBfTX, kBfTY>(grids, work, nwork, parity, err, stencil, kind, st,
                                                               nullptr, 0, fwd);
}
}  // namespace spfm
