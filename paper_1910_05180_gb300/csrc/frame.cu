// frame.cu -- the moving frame of the 1D friction study (Sec. 3.1).
//
// The paper keeps its 1D runs to 50 grid points by moving the whole system
// back by one grid point whenever the favoured phase fills half of it.  Here
// that move copies the interior of the current buffer into the other one,
// shifted along x: phi_i <- phi_{i+cells}, the cells that open up taking the
// value of the row's end cell (the bulk phase there).
#include "spfm_internal.h"

namespace spfm {

namespace {

template <class S>
__global__ void __launch_bounds__(256) shift_x_kernel(const GridGeom g, const S *src, S *dst, int cells)
{
    const long long rows = (long long)g.ny * g.nz;
    for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
        const long long base = cell_index(g, 0, (int)(row % g.ny), (int)(row / g.ny));
        for (int i = threadIdx.x; i < g.nx; i += blockDim.x) {
            int s = i + cells;
            s = s < 0 ? 0 : (s > g.nx - 1 ? g.nx - 1 : s);
            dst[base + i] = src[base + s];
        }
    }
}

}  // namespace

cudaError_t launch_shift_x(const GridGeom &g, int dtype, const void *src, void *dst, int cells, cudaStream_t st)
{
    const long long rows = (long long)g.ny * g.nz;
    const int blocks = (int)(rows < 4096 ? rows : 4096);
    if (dtype == SPFM_F64)
        shift_x_kernel<double><<<blocks, 256, 0, st>>>(g, (const double *)src, (double *)dst, cells);
    else if (dtype == SPFM_F32)
        shift_x_kernel<float><<<blocks, 256, 0, st>>>(g, (const float *)src, (float *)dst, cells);
    else
        shift_x_kernel<__nv_bfloat16><<<blocks, 256, 0, st>>>(g, (const __nv_bfloat16 *)src,
                                                              (__nv_bfloat16 *)dst, cells);
    return cudaGetLastError();
}

}  // namespace spfm
