// tma.cu -- host-side encoding of the TMA tensor maps over ghosted field buffers.
//
// The driver's cuTensorMapEncodeTiled is reached through the runtime's driver
// entry point, so the library needs no link against libcuda.  A map describes
// the buffer as a 3D tensor (pitch, ny + 2, nz + 2) of the storage type with a
// (box_x, box_y, 1) box; the step kernel loads one box per plane.
#include <cudaTypedefs.h>
#include <string.h>

#include "spfm_internal.h"

namespace spfm {

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static int tried = 0;
    if (!tried) {
        tried = 1;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

int encode_field_map(CUtensorMap *map, const GridGeom &g, int dtype, const void *base, int box_x,
                     int box_y)
{
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return -1;
    const CUtensorMapDataType t = dtype == SPFM_F64   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                  : dtype == SPFM_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                      : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const cuuint64_t es = dtype == SPFM_F64 ? 8 : (dtype == SPFM_F32 ? 4 : 2);
    const cuuint64_t dims[3] = {(cuuint64_t)g.pitch, (cuuint64_t)(g.ny + 2), (cuuint64_t)(g.nz + 2)};
    const cuuint64_t strides[2] = {(cuuint64_t)g.pitch * es, (cuuint64_t)g.plane * es};
    const cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = fn(map, t, 3, const_cast<void *>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : (int)r;
}

const CUtensorMap *cached_map(TmaCache *cache, int which, const GridGeom &g, int dtype,
                              const void *base, int box_x, int box_y)
{
    if (!cache || which < 0 || which > 3) return nullptr;
    if (cache->state[which] == 1 && cache->base[which] == base) return &cache->map[which];
    if (cache->state[which] == -1 && cache->base[which] == base) return nullptr;
    cache->base[which] = base;
    cache->state[which] = encode_field_map(&cache->map[which], g, dtype, base, box_x, box_y) == 0 ? 1 : -1;
    return cache->state[which] == 1 ? &cache->map[which] : nullptr;
}

}  // namespace spfm
