// sphericity.cu -- residual anisotropy of a particle (Sec. 3.3, a6) on the GPU.
//
// Pass 1 reduces the particle's barycentre, weighting each interior cell by
// its fraction of the particle phase (1 - phi for a particle with phi = 0
// inside, phi otherwise).  Pass 2 finds the phi = l contour point on every grid
// edge along x, y, z whose two interior end cells lie on opposite sides of l,
// places it by the nonlinear interpolation of Sec. 2.3 (Eqs. 8-10, the two
// positions blended linearly with the division restored), and reduces the
// count, sum, minimum and maximum of the distances R_i from the barycentre.
// Then eps_eff = (R_max - R_min) / (2 R_mean).  FP64 throughout; both passes
// reduce in a fixed order into the grid's scratch partials.
#include <math.h>

#include "host_internal.h"

namespace spfm {

namespace {

constexpr int kSphBlocks = kStatsBlocks;

template <class S> __device__ __forceinline__ double rdd(const S *f, long long i);
template <> __device__ __forceinline__ double rdd<double>(const double *f, long long i) { return f[i]; }
template <> __device__ __forceinline__ double rdd<float>(const float *f, long long i) { return (double)f[i]; }
template <> __device__ __forceinline__ double rdd<__nv_bfloat16>(const __nv_bfloat16 *f, long long i)
{
    return (double)__bfloat162float(f[i]);
}

// v[0..3] sums, v[4] min, v[5] max (the stats reduction's convention)
__device__ void block_reduce6(double *v, double *out)
{
    __shared__ double sm[32][6];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int off = 16; off > 0; off >>= 1)
        for (int i = 0; i < 6; ++i) {
            const double o = __shfl_down_sync(0xffffffffu, v[i], off);
            v[i] = i == 4 ? fmin(v[i], o) : (i == 5 ? fmax(v[i], o) : v[i] + o);
        }
    if (lane == 0)
        for (int i = 0; i < 6; ++i) sm[warp][i] = v[i];
    __syncthreads();
    if (warp == 0) {
        for (int i = 0; i < 6; ++i) v[i] = lane < nw ? sm[lane][i] : (i == 4 ? INFINITY : (i == 5 ? -INFINITY : 0.0));
        for (int off = 16; off > 0; off >>= 1)
            for (int i = 0; i < 6; ++i) {
                const double o = __shfl_down_sync(0xffffffffu, v[i], off);
                v[i] = i == 4 ? fmin(v[i], o) : (i == 5 ? fmax(v[i], o) : v[i] + o);
            }
        if (lane == 0)
            for (int i = 0; i < 6; ++i) out[i] = v[i];
    }
    __syncthreads();
}

template <class S>
__global__ void __launch_bounds__(256) bary_kernel(const GridGeom g, const S *f, int inside, double dx,
                                                   double *part)
{
    double v[6] = {0.0, 0.0, 0.0, 0.0, INFINITY, -INFINITY};
    const long long rows = (long long)g.ny * g.nz;
    for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
        const int j = (int)(row % g.ny), k = (int)(row / g.ny);
        const long long rb = cell_index(g, 0, j, k);
        for (int i = threadIdx.x; i < g.nx; i += blockDim.x) {
            const double ph = rdd<S>(f, rb + i);
            const double w = inside == 0 ? 1.0 - ph : ph;
            v[0] += w;
            v[1] += w * dx * i;
            v[2] += w * dx * j;
            v[3] += w * dx * k;
        }
    }
    block_reduce6(v, part + (long long)blockIdx.x * 6);
}

// |artanh((l - phi)/(2 l phi - phi - l))| of Eqs. 8-10
__device__ __forceinline__ double contour_arg(double phi, double l)
{
    return fabs(atanh((l - phi) / (2.0 * l * phi - phi - l)));
}

template <class S>
__global__ void __launch_bounds__(256) contour_kernel(const GridGeom g, const S *f, double l, double dx,
                                                      double bx, double by, double bz, double *part)
{
    double v[6] = {0.0, 0.0, 0.0, 0.0, INFINITY, -INFINITY};   // count, sum R, -, -, min R, max R
    const long long rows = (long long)g.ny * g.nz;
    for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
        const int j = (int)(row % g.ny), k = (int)(row / g.ny);
        for (int i = threadIdx.x; i < g.nx; i += blockDim.x) {
            const double pa = rdd<S>(f, cell_index(g, i, j, k));
            for (int ax = 0; ax < 3; ++ax) {
                const int ii = i + (ax == 0), jj = j + (ax == 1), kk = k + (ax == 2);
                if (ii >= g.nx || jj >= g.ny || kk >= g.nz) continue;
                const double pb = rdd<S>(f, cell_index(g, ii, jj, kk));
                if ((pa < l) == (pb < l)) continue;
                const double Aa = contour_arg(pa, l), Ab = contour_arg(pb, l);
                const int ca = ax == 0 ? i : (ax == 1 ? j : k), cb = ax == 0 ? ii : (ax == 1 ? jj : kk);
                const double lam_hat = 2.0 * dx / (Aa + Ab);          // Eq. 10
                double xa = dx * ca + 0.5 * lam_hat * Aa;             // Eq. 8
                double xb = dx * cb - 0.5 * lam_hat * Ab;             // Eq. 9
                if (isinf(Aa) && !isinf(Ab)) xa = xb = dx * cb;
                if (isinf(Ab) && !isinf(Aa)) xa = xb = dx * ca;
                if (!(Aa + Ab > 0.0)) xa = xb = dx * (ca + 0.5);
                const double x = (pb != pa) ? (xb * (l - pa) + xa * (pb - l)) / (pb - pa) : xa;
                const double px = ax == 0 ? x : dx * i, py = ax == 1 ? x : dx * j, pz = ax == 2 ? x : dx * k;
                const double R = sqrt((px - bx) * (px - bx) + (py - by) * (py - by) + (pz - bz) * (pz - bz));
                v[0] += 1.0;
                v[1] += R;
                v[4] = fmin(v[4], R);
                v[5] = fmax(v[5], R);
            }
        }
    }
    block_reduce6(v, part + (long long)blockIdx.x * 6);
}

__global__ void __launch_bounds__(256) reduce6_final(double *part, int nblocks, double *out)
{
    double v[6] = {0.0, 0.0, 0.0, 0.0, INFINITY, -INFINITY};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        for (int i = 0; i < 6; ++i) {
            const double x = part[(long long)b * 6 + i];
            v[i] = i == 4 ? fmin(v[i], x) : (i == 5 ? fmax(v[i], x) : v[i] + x);
        }
    block_reduce6(v, out);
}

template <class S>
cudaError_t run_pass(int which, const GridGeom &g, const void *f, double a0, double a1, double b0, double b1,
                     double b2, double *part, double *fin, cudaStream_t st)
{
    if (which == 0) bary_kernel<S><<<kSphBlocks, 256, 0, st>>>(g, (const S *)f, (int)a0, a1, part);
    else contour_kernel<S><<<kSphBlocks, 256, 0, st>>>(g, (const S *)f, a0, a1, b0, b1, b2, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    reduce6_final<<<1, 256, 0, st>>>(part, kSphBlocks, fin);
    return cudaGetLastError();
}

cudaError_t pass(int dtype, int which, const GridGeom &g, const void *f, double a0, double a1, double b0,
                 double b1, double b2, double *part, double *fin, cudaStream_t st)
{
    if (dtype == SPFM_F64) return run_pass<double>(which, g, f, a0, a1, b0, b1, b2, part, fin, st);
    if (dtype == SPFM_F32) return run_pass<float>(which, g, f, a0, a1, b0, b1, b2, part, fin, st);
    return run_pass<__nv_bfloat16>(which, g, f, a0, a1, b0, b1, b2, part, fin, st);
}

}  // namespace
}  // namespace spfm

using namespace spfm;
using namespace spfm_host;

extern "C" spfm_status spfm_sphericity(spfm_grid *g, int inside_phase, double *out)
{
    if (!g || !out) return fail(g, SPFM_EINVAL, "spfm_sphericity: NULL argument");
    if (inside_phase != 0 && inside_phase != 1)
        return fail(g, SPFM_EINVAL, "spfm_sphericity: inside_phase must be 0 or 1");
    const double dx = g->dx > 0.0 ? g->dx : 1.0;
    double *part = (double *)g->d.scratch;
    double *fin = (double *)((char *)g->d.scratch + scratch_final_offset());
    cudaStream_t s = stream_of(g);
    double h[6];
    cudaError_t e = pass(g->d.dtype, 0, g->geom, g->d.field[g->cur], inside_phase, dx, 0, 0, 0, part, fin, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, fin, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(g, e, "spfm_sphericity");
    if (!(h[0] > 0.0)) return fail(g, SPFM_EINVAL, "spfm_sphericity: the grid holds no particle phase");
    const double bx = h[1] / h[0], by = h[2] / h[0], bz = h[3] / h[0];
    e = pass(g->d.dtype, 1, g->geom, g->d.field[g->cur], 0.5, dx, bx, by, bz, part, fin, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, fin, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(g, e, "spfm_sphericity");
    const double n = h[0], mean = n > 0.0 ? h[1] / n : NAN;
    out[0] = n > 0.0 ? (h[5] - h[4]) / (2.0 * mean) : NAN;   // eps_eff
    out[1] = mean;
    out[2] = h[4];
    out[3] = h[5];
    out[4] = n;
    out[5] = bx;
    out[6] = by;
    out[7] = bz;
    return SPFM_OK;
}
