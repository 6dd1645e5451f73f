// boundary.cu -- refresh of the ghost layer from the interior.
//
// Every ghost cell takes the value of the interior cell its boundary map
// points at (periodic wrap, no-flux copy of the adjacent cell), shifted by
// Eq. 7 with the signed coupling a = tanh(2 (x_ghost - x_source).n / lambda) on
// contact faces.  A ghost outside several faces maps every outside coordinate
// at once; the shifts compose in any order because each is a translation of
// the ideal profile, so no face has to be filled before another.
//
// The ghost cells are enumerated face by face so that consecutive threads
// touch consecutive x where the face allows it:
//   z faces  k in {-1, nz}, all (i, j) in [-1, nx] x [-1, ny]
//   y faces  j in {-1, ny}, (i, k) in [-1, nx] x [0, nz)
//   x faces  i in {-1, nx}, (j, k) in [0, ny) x [0, nz)
// Arithmetic in the step kernels' compute type.
#include "spfm_internal.h"

namespace spfm {

template <class S> struct Cmp { using T = float; };
template <> struct Cmp<double> { using T = double; };
__device__ __forceinline__ double ld_ct(const double *f, long long i) { return f[i]; }
__device__ __forceinline__ float ld_ct(const float *f, long long i) { return f[i]; }
__device__ __forceinline__ float ld_ct(const __nv_bfloat16 *f, long long i) { return __bfloat162float(f[i]); }
__device__ __forceinline__ void st_ct(double *f, long long i, double v) { f[i] = v; }
__device__ __forceinline__ void st_ct(float *f, long long i, float v) { f[i] = v; }
__device__ __forceinline__ void st_ct(__nv_bfloat16 *f, long long i, float v) { f[i] = __float2bfloat16_rn(v); }

struct FaceArgs {
    GridGeom g;
    double aface[6];
    long long nzf, nyf, nxf;   // ghost counts of the z, y and x faces (both sides)
    int zper, yper, xper;      // ghost cells per side of each face
};

template <class S>
__device__ __forceinline__ void ghost_faces(const FaceArgs &a, S *f, long long t0, long long stride)
{
    using T = typename Cmp<S>::T;
    const GridGeom &g = a.g;
    const long long total = a.nzf + a.nyf + a.nxf;
    for (long long t = t0; t < total; t += stride) {
        int i, j, k;
        if (t < a.nzf) {
            const int u = (int)t, side = u >= a.zper, r = u - side * a.zper;
            k = side ? g.nz : -1;
            j = r / (g.nx + 2) - 1;
            i = r - (j + 1) * (g.nx + 2) - 1;
        } else if (t < a.nzf + a.nyf) {
            const int u = (int)(t - a.nzf), side = u >= a.yper, r = u - side * a.yper;
            j = side ? g.ny : -1;
            k = r / (g.nx + 2);
            i = r - k * (g.nx + 2) - 1;
        } else {
            const int u = (int)(t - a.nzf - a.nyf), side = u >= a.xper, r = u - side * a.xper;
            i = side ? g.nx : -1;
            k = r / g.ny;
            j = r - k * g.ny;
        }
        int fx, fy, fz;
        const int sx = map_axis(i, g.nx, g.bc[0], g.bc[1], &fx, 0);
        const int sy = map_axis(j, g.ny, g.bc[2], g.bc[3], &fy, 2);
        const int sz = map_axis(k, g.nz, g.bc[4], g.bc[5], &fz, 4);
        T v = ld_ct(f, cell_index(g, sx, sy, sz));
        if (fx >= 0) v = contact_shift_rn(v, (T)a.aface[fx]);
        if (fy >= 0) v = contact_shift_rn(v, (T)a.aface[fy]);
        if (fz >= 0) v = contact_shift_rn(v, (T)a.aface[fz]);
        st_ct(f, cell_index(g, i, j, k), v);
    }
}

template <class S>
__global__ void __launch_bounds__(256) ghost_kernel(const FaceArgs a, S *f)
{
    // the next step kernel may launch now: its boxes that touch a face wait for
    // this grid to complete (griddepcontrol.wait), the others read no ghost
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    ghost_faces<S>(a, f, blockIdx.x * (long long)blockDim.x + threadIdx.x,
                   (long long)gridDim.x * blockDim.x);
}

__host__ __device__ inline FaceArgs face_args(const GridGeom &g, const double *aface, int x_faces)
{
    FaceArgs a;
    a.g = g;
    for (int f = 0; f < 6; ++f) a.aface[f] = aface[f];
    a.zper = (g.nx + 2) * (g.ny + 2);
    a.yper = (g.nx + 2) * g.nz;
    a.xper = g.ny * g.nz;
    a.nzf = 2LL * a.zper;
    a.nyf = 2LL * a.yper;
    a.nxf = x_faces ? 2LL * a.xper : 0;
    return a;
}

// blockIdx.y selects the grid of the batch
template <class S>
__global__ void __launch_bounds__(256) ghost_batch_kernel(const GhostJob *jobs, int parity)
{
    const GhostJob &j = jobs[blockIdx.y];
    const FaceArgs a = face_args(j.g, j.aface, 1);
    ghost_faces<S>(a, (S *)j.field[j.cur ^ parity], blockIdx.x * (long long)blockDim.x + threadIdx.x,
                   (long long)gridDim.x * blockDim.x);
}

cudaError_t launch_fill_ghosts_batch(const GhostJob *jobs, int n, int dtype, int parity, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const dim3 grid(16, n);
    if (dtype == SPFM_F64) ghost_batch_kernel<double><<<grid, 256, 0, st>>>(jobs, parity);
    else if (dtype == SPFM_F32) ghost_batch_kernel<float><<<grid, 256, 0, st>>>(jobs, parity);
    else ghost_batch_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(jobs, parity);
    return cudaGetLastError();
}

cudaError_t launch_fill_ghosts(const GridGeom &g, int dtype, const double aface[6], void *field,
                               cudaStream_t st, int x_faces)
{
    const FaceArgs a = face_args(g, aface, x_faces);
    const long long total = a.nzf + a.nyf + a.nxf;
    long long blocks = (total + 255) / 256;
    if (blocks > 2 * 152 * 8) blocks = 2 * 152 * 8;
    if (dtype == SPFM_F64) ghost_kernel<double><<<(int)blocks, 256, 0, st>>>(a, (double *)field);
    else if (dtype == SPFM_F32) ghost_kernel<float><<<(int)blocks, 256, 0, st>>>(a, (float *)field);
    else ghost_kernel<__nv_bfloat16><<<(int)blocks, 256, 0, st>>>(a, (__nv_bfloat16 *)field);
    return cudaGetLastError();
}

}  // namespace spfm
