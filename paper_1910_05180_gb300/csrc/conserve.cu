// conserve.cu -- the constant-volume correction of a step (Sec. 3.3).
//
// The shape relaxation of Sec. 3.3 keeps the particle volume fixed with a
// homogeneous, time-dependent driving force.  The driving term of one step is
// -dt (4 M dF / (lambda Gamma)) q(phi) per cell (q = phi (1 - phi), the h3
// term), so after the ordinary step at dF = 0 has written phi* = phi + dt R0,
// the dF that leaves sum_p phi_p unchanged subtracts alpha q(phi_p) from every
// cell with
//     alpha = sum_p (phi*_p - phi_p) / sum_p q(phi_p),
//     dF    = alpha lambda Gamma / (4 M dt).
// Pass 1 reduces the two sums in FP64 (rows dealt round-robin to the blocks,
// fixed order, so the result is reproducible); pass 2 has every block add the
// partials in the same order, form alpha, and correct its rows of phi*.
#include "spfm_internal.h"

namespace spfm {

namespace {

template <class S> __device__ __forceinline__ double ld64(const S *f, long long i);
template <> __device__ __forceinline__ double ld64<double>(const double *f, long long i) { return f[i]; }
template <> __device__ __forceinline__ double ld64<float>(const float *f, long long i) { return (double)f[i]; }
template <> __device__ __forceinline__ double ld64<__nv_bfloat16>(const __nv_bfloat16 *f, long long i)
{
    return (double)__bfloat162float(f[i]);
}
template <class S> __device__ __forceinline__ S st_of(double v);
template <> __device__ __forceinline__ double st_of<double>(double v) { return v; }
template <> __device__ __forceinline__ float st_of<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ __nv_bfloat16 st_of<__nv_bfloat16>(double v)
{
    return __float2bfloat16_rn((float)v);
}

// sum of two doubles over the block, result in thread 0
__device__ __forceinline__ void block_sum2(double &a, double &b)
{
    __shared__ double sa[32], sb[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, off);
        b += __shfl_down_sync(0xffffffffu, b, off);
    }
    if (lane == 0) {
        sa[warp] = a;
        sb[warp] = b;
    }
    __syncthreads();
    if (warp == 0) {
        a = lane < nw ? sa[lane] : 0.0;
        b = lane < nw ? sb[lane] : 0.0;
        for (int off = 16; off > 0; off >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, off);
            b += __shfl_down_sync(0xffffffffu, b, off);
        }
    }
}

template <class S>
__global__ void __launch_bounds__(256) conserve_sums_kernel(const GridGeom g, const S *src, const S *dst,
                                                            double *partials)
{
    double dsum = 0.0, qsum = 0.0;
    const long long rows = (long long)g.ny * g.nz;
    for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
        const long long base = cell_index(g, 0, (int)(row % g.ny), (int)(row / g.ny));
        for (int i = threadIdx.x; i < g.nx; i += blockDim.x) {
            const double p = ld64<S>(src, base + i);
            dsum += ld64<S>(dst, base + i) - p;
            qsum += p * (1.0 - p);
        }
    }
    block_sum2(dsum, qsum);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = dsum;
        partials[2 * blockIdx.x + 1] = qsum;
    }
}

template <class S>
__global__ void __launch_bounds__(256) conserve_apply_kernel(const GridGeom g, const S *src, S *dst,
                                                             const double *partials, int nblk,
                                                             double *alpha_out)
{
    __shared__ double s_alpha;
    if (threadIdx.x == 0) {
        double d = 0.0, q = 0.0;
        for (int b = 0; b < nblk; ++b) {   // the same order in every block
            d += partials[2 * b];
            q += partials[2 * b + 1];
        }
        s_alpha = q != 0.0 ? d / q : 0.0;
        if (blockIdx.x == 0) *alpha_out = s_alpha;
    }
    __syncthreads();
    const double alpha = s_alpha;
    const long long rows = (long long)g.ny * g.nz;
    for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
        const long long base = cell_index(g, 0, (int)(row % g.ny), (int)(row / g.ny));
        for (int i = threadIdx.x; i < g.nx; i += blockDim.x) {
            const double p = ld64<S>(src, base + i);
            dst[base + i] = st_of<S>(ld64<S>(dst, base + i) - alpha * (p * (1.0 - p)));
        }
    }
}

}  // namespace

cudaError_t launch_conserve(const GridGeom &g, int dtype, const void *src, void *dst, double *partials,
                            double *alpha_out, cudaStream_t st)
{
    const long long rows = (long long)g.ny * g.nz;
    const int nblk = (int)(rows < kStatsBlocks ? rows : kStatsBlocks);
    if (dtype == SPFM_F64) {
        conserve_sums_kernel<double><<<nblk, 256, 0, st>>>(g, (const double *)src, (const double *)dst, partials);
        conserve_apply_kernel<double><<<nblk, 256, 0, st>>>(g, (const double *)src, (double *)dst, partials,
                                                            nblk, alpha_out);
    } else if (dtype == SPFM_F32) {
        conserve_sums_kernel<float><<<nblk, 256, 0, st>>>(g, (const float *)src, (const float *)dst, partials);
        conserve_apply_kernel<float><<<nblk, 256, 0, st>>>(g, (const float *)src, (float *)dst, partials, nblk,
                                                           alpha_out);
    } else {
        conserve_sums_kernel<__nv_bfloat16><<<nblk, 256, 0, st>>>(g, (const __nv_bfloat16 *)src,
                                                                  (const __nv_bfloat16 *)dst, partials);
        conserve_apply_kernel<__nv_bfloat16><<<nblk, 256, 0, st>>>(g, (const __nv_bfloat16 *)src,
                                                                   (__nv_bfloat16 *)dst, partials, nblk,
                                                                   alpha_out);
    }
    return cudaGetLastError();
}

}  // namespace spfm
