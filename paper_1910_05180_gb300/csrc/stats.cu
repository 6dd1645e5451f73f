// stats.cu -- ideal-profile initialisation and FP64 interface
// diagnostics on the ghosted field layout (spfm_internal.h).
//
// init: Eq. 3 (planar) or its radial form, evaluated in FP64 per cell and
// rounded once to the storage type (the caller then fills the ghost layer).
//
// stats: one pass over the interior accumulating in FP64, per thread in a
// fixed row order, then warp-shuffle and shared-memory block reductions into
// kStatsBlocks partials, then one CTA reducing the partials in a fixed order,
// so the result is bit-reproducible for a given grid size.  Sums over the band
// 1e-6 < phi < 1 - 1e-6 invert the ideal profile (Sec. 2.3):
//   position  c = sum q (p.n - (lambda/2) artanh(1-2phi)) / sum q
//   radius    R = sum q (|p - ctr| + (lambda/2) artanh(1-2phi)) / sum q
// The optional interface energy is Eq. 1 at dF = 0; its forward differences
// read the ghost layer.
#include <math.h>

#include "spfm_internal.h"

namespace spfm {

template <class S> __device__ __forceinline__ double rd(const S *f, long long i);
template <> __device__ __forceinline__ double rd<double>(const double *f, long long i) { return f[i]; }
template <> __device__ __forceinline__ double rd<float>(const float *f, long long i) { return (double)f[i]; }
template <> __device__ __forceinline__ double rd<__nv_bfloat16>(const __nv_bfloat16 *f, long long i)
{
    return (double)__bfloat162float(f[i]);
}

template <class S> __device__ __forceinline__ S wr(double v);
template <> __device__ __forceinline__ double wr<double>(double v) { return v; }
template <> __device__ __forceinline__ float wr<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ __nv_bfloat16 wr<__nv_bfloat16>(double v)
{
    return __float2bfloat16_rn((float)v);
}

template <class S>
__global__ void init_kernel(const InitArgs a, S *f)
{
    const long long rows = (long long)(a.g.ny + 2) * (a.g.nz + 2);
    for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
        const int j = (int)(row % (a.g.ny + 2)) - 1;
        const int k = (int)(row / (a.g.ny + 2)) - 1;
        S *r = f + row * a.g.pitch;
        const bool inner = j >= 0 && j < a.g.ny && k >= 0 && k < a.g.nz;
        for (int x = threadIdx.x; x < a.g.pitch; x += blockDim.x) {
            const int i = x - a.g.off;
            double v = 0.0;
            if (inner && i >= 0 && i < a.g.nx) {
                const double px = a.dx * i, py = a.dx * j, pz = a.dx * k;
                if (a.sphere) {
                    const double rx = px - a.ctr[0], ry = py - a.ctr[1], rz = pz - a.ctr[2];
                    const double rr = sqrt(rx * rx + ry * ry + rz * rz);
                    v = 0.5 * (1.0 - tanh(2.0 * (a.R - rr) / a.lambda));
                } else {
                    const double pn = px * a.n[0] + py * a.n[1] + pz * a.n[2];
                    v = 0.5 * (1.0 - tanh(2.0 * (pn - a.c) / a.lambda));
                }
            }
            r[x] = wr<S>(v);
        }
    }
}

cudaError_t launch_init(const InitArgs &a, void *field, cudaStream_t st)
{
    const long long rows = (long long)(a.g.ny + 2) * (a.g.nz + 2);
    const int blocks = (int)(rows < 8192 ? rows : 8192);
    if (a.dtype == SPFM_F64) init_kernel<double><<<blocks, 128, 0, st>>>(a, (double *)field);
    else if (a.dtype == SPFM_F32) init_kernel<float><<<blocks, 128, 0, st>>>(a, (float *)field);
    else init_kernel<__nv_bfloat16><<<blocks, 128, 0, st>>>(a, (__nv_bfloat16 *)field);
    return cudaGetLastError();
}

// Eq. 6 (TI) or the CF quartic per direction; lam2_r2 = lambda^2/|r_k|^2
__device__ __forceinline__ double potential(double phi, double a, double lam2_r2, int cf)
{
    const double q = phi * (1.0 - phi), s = 1.0 - 2.0 * phi;
    if (cf) return 8.0 * q * q / 3.0;
    const double A = a * a;
    if (A < 1e-8) return lam2_r2 * 2.0 * A * q * q;
    return lam2_r2 * (q + (1.0 - A) / (4.0 * A) * log((1.0 - A) / (1.0 - A * s * s)));
}

__device__ __forceinline__ void warp_reduce(double *v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int i = 0; i < kNStat; ++i) {
            const double o = __shfl_down_sync(0xffffffffu, v[i], off);
            if (i == 4) v[i] = fmin(v[i], o);
            else if (i == 5) v[i] = fmax(v[i], o);
            else v[i] += o;
        }
    }
}

__device__ __forceinline__ void block_reduce_store(double *v, double *out)
{
    __shared__ double sm[32][kNStat];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    warp_reduce(v);
    if (lane == 0)
        for (int i = 0; i < kNStat; ++i) sm[warp][i] = v[i];
    __syncthreads();
    if (warp == 0) {
        for (int i = 0; i < kNStat; ++i)
            v[i] = lane < nw ? sm[lane][i] : (i == 4 ? INFINITY : (i == 5 ? -INFINITY : 0.0));
        warp_reduce(v);
        if (lane == 0)
            for (int i = 0; i < kNStat; ++i) out[i] = v[i];
    }
}

// Per-thread partials: [0] sum phi, [1] S_w, [2] S_c, [3] S_r, [4] min, [5] max,
// [6] non-finite count, [7] energy density sum, [8..11] unused.
// Screening type of a storage type: comparisons (finite, min, max, band) are
// exact in the storage precision, so only the sums run in FP64.
template <class S> struct Scr { using T = float; };
template <> struct Scr<double> { using T = double; };
template <class S> __device__ __forceinline__ typename Scr<S>::T scr(const S *f, long long i);
template <> __device__ __forceinline__ double scr<double>(const double *f, long long i) { return f[i]; }
template <> __device__ __forceinline__ float scr<float>(const float *f, long long i) { return f[i]; }
template <> __device__ __forceinline__ float scr<__nv_bfloat16>(const __nv_bfloat16 *f, long long i)
{
    return __bfloat162float(f[i]);
}

// Partial sums of one block over its contiguous range of rows: block b of nb
// takes rows [b * rows / nb, (b + 1) * rows / nb), rows ordered (j fastest, k).
template <class S>
__device__ __forceinline__ void stats_pass(const StatsArgs &a, const S *f, double *partial_out,
                                           long long blk, long long nblk)
{
    using R = typename Scr<S>::T;
    double v[kNStat];
#pragma unroll
    for (int i = 0; i < kNStat; ++i) v[i] = 0.0;
    R mn = R(INFINITY), mx = R(-INFINITY);
    const double e_pref = a.Gamma / (a.C_gamma * a.lambda);
    const int nd = a.stencil == 6 ? 3 : (a.stencil == 18 ? 9 : 13);
    const R lo = R(0.5e-6), hi = R(1.0 - 0.5e-6);   // conservative pre-filter of the FP64 band test
    const long long rows = (long long)a.g.ny * a.g.nz;
    const long long r0 = blk * rows / nblk, r1 = (blk + 1) * rows / nblk;
    int j = (int)(r0 % a.g.ny), k = (int)(r0 / a.g.ny);
    for (long long row = r0; row < r1; ++row) {
        const long long rbase = cell_index(a.g, 0, j, k);
        for (int i = threadIdx.x; i < a.g.nx; i += blockDim.x) {
            const R r = scr<S>(f, rbase + i);
            if (!isfinite(r)) { v[6] += 1.0; continue; }
            const double ph = (double)r;   // exact
            v[0] += ph;
            mn = r < mn ? r : mn;
            mx = r > mx ? r : mx;
            if (r > lo && r < hi && ph > 1e-6 && ph < 1.0 - 1e-6) {
                const double q = ph * (1.0 - ph);
                const double psi = 0.5 * a.lambda * atanh(1.0 - 2.0 * ph);
                const double px = a.dx * i, py = a.dx * j, pz = a.dx * k;
                const double pn = px * a.n[0] + py * a.n[1] + pz * a.n[2];
                const double rx = px - a.ctr[0], ry = py - a.ctr[1], rz = pz - a.ctr[2];
                v[1] += q;
                v[2] += q * (pn - psi);
                v[3] += q * (sqrt(rx * rx + ry * ry + rz * rz) + psi);
            }
            if (a.energy) {
                double e = 0.0;
                for (int kk = 0; kk < nd; ++kk) {
                    const Dir d = grid_dir(kk);
                    const double r2 = (double)d.shell * a.dx * a.dx;
                    const double nb = rd<S>(f, cell_index(a.g, i + d.x, j + d.y, k + d.z));
                    const double dp = nb - ph;
                    e += a.w[kk] * (0.5 * a.lambda * a.lambda * dp * dp / r2 +
                                    potential(ph, a.a[kk], a.lambda * a.lambda / r2, a.scheme == SPFM_FD));
                }
                v[7] += e_pref * e;
            }
        }
        if (++j == a.g.ny) { j = 0; ++k; }
    }
    v[4] = (double)mn;
    v[5] = (double)mx;
    block_reduce_store(v, partial_out);
}

template <class S>
__global__ void __launch_bounds__(256) stats_kernel(const StatsArgs a, const S *f, double *partials)
{
    stats_pass<S>(a, f, partials + (long long)blockIdx.x * kNStat, blockIdx.x, gridDim.x);
}

// blockIdx.y selects the grid of the batch
template <class S>
__global__ void __launch_bounds__(256) stats_batch_kernel(const StatsJob *jobs, double *partials)
{
    const StatsJob &j = jobs[blockIdx.y];
    stats_pass<S>(j.a, (const S *)j.field[j.cur],
                  partials + ((long long)blockIdx.y * kBatchStatsBlocks + blockIdx.x) * kNStat,
                  blockIdx.x, gridDim.x);
}

// blockIdx.x selects a grid: reduce its nblocks partials into out[blockIdx.x]
__global__ void __launch_bounds__(256) stats_final_kernel(const double *partials, int nblocks, double *out)
{
    partials += (long long)blockIdx.x * nblocks * kNStat;
    out += (long long)blockIdx.x * kNStat;
    double v[kNStat];
#pragma unroll
    for (int i = 0; i < kNStat; ++i) v[i] = 0.0;
    v[4] = INFINITY;
    v[5] = -INFINITY;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
#pragma unroll
        for (int i = 0; i < kNStat; ++i) {
            const double x = partials[(long long)b * kNStat + i];
            if (i == 4) v[i] = fmin(v[i], x);
            else if (i == 5) v[i] = fmax(v[i], x);
            else v[i] += x;
        }
    }
    block_reduce_store(v, out);
}

size_t stats_scratch_bytes()
{
    return sizeof(double) * (size_t)kNStat * (kStatsBlocks + 1);
}

size_t grid_scratch_bytes()
{
    return scratch_err_offset() + 16;
}

cudaError_t launch_stats(const StatsArgs &a, const void *field, double *partials, double *final_out,
                         cudaStream_t st)
{
    if (a.dtype == SPFM_F64)
        stats_kernel<double><<<kStatsBlocks, 256, 0, st>>>(a, (const double *)field, partials);
    else if (a.dtype == SPFM_F32)
        stats_kernel<float><<<kStatsBlocks, 256, 0, st>>>(a, (const float *)field, partials);
    else
        stats_kernel<__nv_bfloat16><<<kStatsBlocks, 256, 0, st>>>(a, (const __nv_bfloat16 *)field, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    stats_final_kernel<<<1, 256, 0, st>>>(partials, kStatsBlocks, final_out);
    return cudaGetLastError();
}

cudaError_t launch_stats_batch(const StatsJob *jobs, int n, int dtype, double *partials, double *finals,
                               cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const dim3 grid(kBatchStatsBlocks, n);
    if (dtype == SPFM_F64) stats_batch_kernel<double><<<grid, 256, 0, st>>>(jobs, partials);
    else if (dtype == SPFM_F32) stats_batch_kernel<float><<<grid, 256, 0, st>>>(jobs, partials);
    else stats_batch_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(jobs, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    stats_final_kernel<<<n, 256, 0, st>>>(partials, kBatchStatsBlocks, finals);
    return cudaGetLastError();
}

}  // namespace spfm
