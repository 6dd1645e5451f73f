// stats_static.cu -- interface diagnostics that allocate nothing.
//
// spfm_interface_stats needs a grid handle, whose creation requires a scratch
// buffer from the caller.  Some callers cannot provide one: a host program
// whose device memory is owned by another framework's pool and that may not
// allocate after start-up, or a loop that measures a field it only borrows.
// spfm_interface_stats_static serves them: the caller passes the field and
// its description, and the reduction partials live in a fixed array inside
// this library (kStaticPlanes planes of kStaticStat doubles, 96 KiB), which
// every GPU that loads the library holds until the process exits.
//
// The first call on a device resolves the array's device address with
// cudaGetSymbolAddress (host code cannot use the array's name as a device
// address); make that first call before any stream capture begins.  The
// address is that of the current device, so desc->stream must belong to the
// current device (a stream of another device is refused with SPFM_EINVAL).
// One CTA reduces one z plane into its slot of the array, then one CTA sums
// the slots in plane order, so the result is reproducible.  Every slot that is
// read was written by the same call, so nothing has to be cleared between
// calls; but all calls share the array, so calls whose kernels overlap on the
// GPU (for example on two streams) race and must be serialised by the caller.
#include <math.h>
#include <string.h>

#include <mutex>

#include "host_internal.h"

namespace {

constexpr int kStaticPlanes = 1024;   // largest nz served
constexpr int kStaticStat = 12;       // doubles per partial (as the grid stats)

// partials of up to kStaticPlanes planes, then the final reduction
static __device__ __align__(256) double s_static_scratch[(kStaticPlanes + 1) * kStaticStat];

struct PlaneArgs {
    spfm::GridGeom g;
    double n[3], ctr[3];
    double lambda, dx;
};

template <class S> __device__ __forceinline__ double rdv(const S *f, long long i);
template <> __device__ __forceinline__ double rdv<double>(const double *f, long long i) { return f[i]; }
template <> __device__ __forceinline__ double rdv<float>(const float *f, long long i) { return (double)f[i]; }
template <> __device__ __forceinline__ double rdv<__nv_bfloat16>(const __nv_bfloat16 *f, long long i)
{
    return (double)__bfloat162float(f[i]);
}

__device__ __forceinline__ void reduce_into(double *v, double *out)
{
    __shared__ double sm[32][kStaticStat];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int off = 16; off > 0; off >>= 1)
        for (int i = 0; i < kStaticStat; ++i) {
            const double o = __shfl_down_sync(0xffffffffu, v[i], off);
            v[i] = i == 4 ? fmin(v[i], o) : (i == 5 ? fmax(v[i], o) : v[i] + o);
        }
    if (lane == 0)
        for (int i = 0; i < kStaticStat; ++i) sm[warp][i] = v[i];
    __syncthreads();
    if (warp == 0) {
        for (int i = 0; i < kStaticStat; ++i)
            v[i] = lane < nw ? sm[lane][i] : (i == 4 ? INFINITY : (i == 5 ? -INFINITY : 0.0));
        for (int off = 16; off > 0; off >>= 1)
            for (int i = 0; i < kStaticStat; ++i) {
                const double o = __shfl_down_sync(0xffffffffu, v[i], off);
                v[i] = i == 4 ? fmin(v[i], o) : (i == 5 ? fmax(v[i], o) : v[i] + o);
            }
        if (lane == 0)
            for (int i = 0; i < kStaticStat; ++i) out[i] = v[i];
    }
}

// CTA k: the interior cells of plane k (same sums as the grid stats, Sec. 2.3)
template <class S>
__global__ void __launch_bounds__(256) plane_stats_kernel(const PlaneArgs a, const S *f, double *scratch)
{
    double v[kStaticStat];
    for (int i = 0; i < kStaticStat; ++i) v[i] = 0.0;
    v[4] = INFINITY;
    v[5] = -INFINITY;
    const int k = blockIdx.x;
    for (int j = 0; j < a.g.ny; ++j) {
        const long long rbase = spfm::cell_index(a.g, 0, j, k);
        for (int i = threadIdx.x; i < a.g.nx; i += blockDim.x) {
            const double ph = rdv<S>(f, rbase + i);
            if (!isfinite(ph)) { v[6] += 1.0; continue; }
            v[0] += ph;
            v[4] = fmin(v[4], ph);
            v[5] = fmax(v[5], ph);
            if (ph > 1e-6 && ph < 1.0 - 1e-6) {
                const double q = ph * (1.0 - ph);
                const double psi = 0.5 * a.lambda * atanh(1.0 - 2.0 * ph);
                const double px = a.dx * i, py = a.dx * j, pz = a.dx * k;
                const double pn = px * a.n[0] + py * a.n[1] + pz * a.n[2];
                const double rx = px - a.ctr[0], ry = py - a.ctr[1], rz = pz - a.ctr[2];
                v[1] += q;
                v[2] += q * (pn - psi);
                v[3] += q * (sqrt(rx * rx + ry * ry + rz * rz) + psi);
            }
        }
    }
    reduce_into(v, scratch + (long long)k * kStaticStat);
}

__global__ void __launch_bounds__(256) planes_final_kernel(double *scratch, int nplanes)
{
    double v[kStaticStat];
    for (int i = 0; i < kStaticStat; ++i) v[i] = 0.0;
    v[4] = INFINITY;
    v[5] = -INFINITY;
    for (int b = threadIdx.x; b < nplanes; b += blockDim.x)
        for (int i = 0; i < kStaticStat; ++i) {
            const double x = scratch[(long long)b * kStaticStat + i];
            v[i] = i == 4 ? fmin(v[i], x) : (i == 5 ? fmax(v[i], x) : v[i] + x);
        }
    reduce_into(v, scratch + (long long)kStaticPlanes * kStaticStat);
}

// device address of the array, resolved once per device with that device current
std::mutex g_mutex;
double *g_addr[128];

double *static_scratch_address(int *err_code)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 128) {
        *err_code = (int)e;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, s_static_scratch);
        if (e != cudaSuccess || !p) {
            *err_code = (int)e;
            return nullptr;
        }
        g_addr[dev] = (double *)p;
    }
    return g_addr[dev];
}

}  // namespace

extern "C" spfm_status spfm_interface_stats_static(const spfm_grid_desc *desc, const void *field,
                                                   double lambda, double dx, spfm_stats *out)
{
    using spfm_host::fail;
    if (!desc || !field || !out) return fail(nullptr, SPFM_EINVAL, "spfm_interface_stats_static: NULL argument");
    if (!(lambda > 0.0) || !(dx > 0.0))
        return fail(nullptr, SPFM_EINVAL, "spfm_interface_stats_static: lambda and dx must be > 0");
    size_t px = 0, off = 0;
    spfm_status st = spfm_layout(desc, &px, &off, nullptr, nullptr);
    if (st != SPFM_OK) return st;
    st = spfm_host::check_extent(desc, px, "spfm_interface_stats_static");
    if (st != SPFM_OK) return st;
    const double nn = desc->n[0] * desc->n[0] + desc->n[1] * desc->n[1] + desc->n[2] * desc->n[2];
    if (!(fabs(nn - 1.0) < 1e-9))
        return fail(nullptr, SPFM_EINVAL, "spfm_interface_stats_static: |n| = %g, must be 1", sqrt(nn));
    if (desc->nz > kStaticPlanes)
        return fail(nullptr, SPFM_EINVAL,
                    "spfm_interface_stats_static: nz = %d exceeds the %d planes its fixed scratch holds",
                    desc->nz, kStaticPlanes);
    if ((uintptr_t)field & 15)
        return fail(nullptr, SPFM_EINVAL, "spfm_interface_stats_static: field not 16-byte aligned");
    // the array's address is resolved for the current device, so the stream
    // must belong to that device
    cudaStream_t s = (cudaStream_t)desc->stream;
    int cur_dev = -1, stream_dev = -1;
    cudaError_t de = cudaGetDevice(&cur_dev);
    if (de == cudaSuccess) de = cudaStreamGetDevice(s, &stream_dev);
    if (de != cudaSuccess)
        return fail(nullptr, SPFM_ECUDA, "spfm_interface_stats_static: %s", cudaGetErrorString(de));
    if (stream_dev != cur_dev)
        return fail(nullptr, SPFM_EINVAL,
                    "spfm_interface_stats_static: desc->stream belongs to device %d, the current device is %d",
                    stream_dev, cur_dev);
    int code = 0;
    double *scratch = static_scratch_address(&code);
    if (!scratch)
        return fail(nullptr, SPFM_ECUDA, "spfm_interface_stats_static: no address for the fixed scratch (%s)",
                    cudaGetErrorString((cudaError_t)code));
    PlaneArgs a;
    memset(&a, 0, sizeof a);
    a.g.nx = desc->nx;
    a.g.ny = desc->ny;
    a.g.nz = desc->nz;
    a.g.pitch = (int)px;
    a.g.off = (int)off;
    a.g.plane = (long long)px * (desc->ny + 2);
    for (int i = 0; i < 3; ++i) { a.n[i] = desc->n[i]; a.ctr[i] = desc->center[i]; }
    a.lambda = lambda;
    a.dx = dx;
    if (desc->dtype == SPFM_F64) plane_stats_kernel<double><<<desc->nz, 256, 0, s>>>(a, (const double *)field, scratch);
    else if (desc->dtype == SPFM_F32) plane_stats_kernel<float><<<desc->nz, 256, 0, s>>>(a, (const float *)field, scratch);
    else plane_stats_kernel<__nv_bfloat16><<<desc->nz, 256, 0, s>>>(a, (const __nv_bfloat16 *)field, scratch);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        planes_final_kernel<<<1, 256, 0, s>>>(scratch, desc->nz);
        e = cudaGetLastError();
    }
    double h[kStaticStat];
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h, scratch + (long long)kStaticPlanes * kStaticStat, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(nullptr, SPFM_ECUDA, "spfm_interface_stats_static: %s", cudaGetErrorString(e));
    out->volume = h[0] * dx * dx * dx;
    out->S_w = h[1];
    out->S_c = h[2];
    out->S_r = h[3];
    out->phi_min = h[4];
    out->phi_max = h[5];
    out->nonfinite = h[6];
    out->position = h[1] > 0.0 ? h[2] / h[1] : NAN;
    out->radius = h[1] > 0.0 ? h[3] / h[1] : NAN;
    out->energy = NAN;
    out->steps = 0.0;
    out->time = 0.0;
    if (h[6] > 0.0) return fail(nullptr, SPFM_ENONFINITE, "field holds %.0f non-finite cells", h[6]);
    return SPFM_OK;
}
