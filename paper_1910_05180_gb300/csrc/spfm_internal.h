// spfm_internal.h -- shared definitions of the GB300 SPFM library (host + device).
//
// Parameter blocks handed to the kernels, the boundary-aware element loader
// (periodic / no-flux / contact-angle ghosts, Eq. 7), and the launcher
// declarations that connect the C ABI (api.cu) to the kernels.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/spfm.h"

namespace spfm {

constexpr int kMaxTerms = 13;    // grid directions of the 26-neighbour stencil (Tab. 1)
constexpr int kStatsBlocks = 608;  // most stats partials; a launch takes one full wave of at most this
constexpr int kNStat = 12;       // doubles per partial (see stats.cu)

// Grid vectors of Tab. 1, one per +/- pair: shell 1 (k = 0..2), shell 2
// (3..8), shell 3 (9..12).
struct Dir { int x, y, z, shell; };
__host__ __device__ inline Dir grid_dir(int k)
{
    switch (k) {
    case 0: return {1, 0, 0, 1};
    case 1: return {0, 1, 0, 1};
    case 2: return {0, 0, 1, 1};
    case 3: return {1, 1, 0, 2};
    case 4: return {0, 1, 1, 2};
    case 5: return {1, 0, 1, 2};
    case 6: return {1, -1, 0, 2};
    case 7: return {0, 1, -1, 2};
    case 8: return {1, 0, -1, 2};
    case 9: return {1, 1, 1, 3};
    case 10: return {-1, 1, 1, 3};
    case 11: return {1, -1, 1, 3};
    default: return {1, 1, -1, 3};
    }
}

// Geometry of one grid buffer as the kernels see it.  Every buffer carries a
// one-cell ghost layer: interior cell (i, j, k), i in [0, nx), sits at
//   ((k + 1) * (ny + 2) + (j + 1)) * pitch + off + i,
// ghosts at i = -1, nx, j = -1, ny, k = -1, nz.  off = 32 bytes of elements, so
// interior rows start on a 32-byte sector, and the x ghosts sit in sectors of
// their own; pitch is a 32-byte multiple >= off + nx + 1.
struct GridGeom {
    int nx, ny, nz;
    int pitch;          // elements per padded row
    int off;            // x offset of interior cell 0 (32 bytes of elements)
    long long plane;    // pitch * (ny + 2)
    int bc[6];          // SPFM_PERIODIC / NOFLUX / CONTACT per face
};

__host__ __device__ inline long long cell_index(const GridGeom &g, int i, int j, int k)
{
    return (long long)(k + 1) * g.plane + (long long)(j + 1) * g.pitch + g.off + i;
}

// Step coefficients of one grid, precomputed on the host in FP64 (a1) and
// rounded to the compute type T.
template <class T>
struct StepCoef {
    GridGeom g;
    T aface[6];             // signed contact coupling per face, tanh(2 (x_g - x_s).n / lambda)
    T c1, c2, c3;           // Laplacian shell coefficients D w_j / |r_j|^2
    T dt, kmu, kappa;       // Euler step, h3 driving 4 M dF/(lambda Gamma), CF potential
    int nterms;             // TI: distinct non-zero A_k after grouping
    T beta[kMaxTerms];      // TI: summed 4 c_k A_k of each group
    T A[kMaxTerms];         // TI: the group's A_k = a_k^2
    // the same coefficients multiplied by dt in FP64 before rounding (the step
    // kernels fold the Euler update into them): c_j dt, the weight of
    // t = (phi_{z-1} - phi) + (phi_{z+1} - phi), -beta dt, -kmu dt, -kappa dt
    T c1dt, c2dt, c3dt, ctdt, nkmudt, nkapdt;
    T nbetadt[kMaxTerms];
    // TI_n (local normal): per-direction c_k; the scale that turns a central
    // difference of the kernels' log-odds ln or log2((1 - phi)/phi) into the
    // gradient of psi (FP32: (lambda/4) ln 2 / (2 dx), FP64: (lambda/4) / (2 dx));
    // 2 dx/lambda; the clamp of phi
    T ck[kMaxTerms];
    T psi_grad, two_dx_over_lam, eps;
    // CF models: interpolation function of the driving term, 0 h3, 1 h5, 2 h_Abel
    int interp;
    // stochastic rounding of the update (SPFM_ROUND_STOCHASTIC): the grid's mixed
    // seed, and the key of the step a single-grid launch computes (sr_step_key)
    uint32_t sr_seed, sr_key;
};

// Counter-based random bits of the stochastic rounding: the 32-bit integer
// hash "lowbias32" of C. Wellons ("Prospecting for hash functions", 2018),
// applied to (padded cell index) xor (step key); the step key mixes the grid's
// seed with its own step count, so a grid draws the same bits alone and in any
// batch.
__host__ __device__ inline uint32_t sr_hash(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}
__host__ __device__ inline uint32_t sr_seed_mix(unsigned long long seed)
{
    return sr_hash((uint32_t)seed ^ sr_hash((uint32_t)(seed >> 32) + 0x9e3779b9u));
}
__host__ __device__ inline uint32_t sr_step_key(uint32_t seed_mix, long long step)
{
    const unsigned long long s = (unsigned long long)step;
    return sr_hash(seed_mix ^ sr_hash((uint32_t)s ^ sr_hash((uint32_t)(s >> 32))));
}

// the CF models of Tab. 2 (any interpolation function)
__host__ __device__ inline bool is_fd_scheme(int scheme)
{
    return scheme == SPFM_FD || scheme == SPFM_FD_H5 || scheme == SPFM_FD_HABEL;
}

// Ghost mapping for one axis: at most one cell outside [0, n).  Returns the
// source coordinate and sets *contact when a contact-angle transform applies.
__host__ __device__ inline int map_axis(int c, int n, int bc_lo, int bc_hi, int *face_hit,
                                        int face_lo)
{
    *face_hit = -1;
    if (c < 0) {
        if (bc_lo == SPFM_PERIODIC) return c + n;
        if (bc_lo == SPFM_CONTACT) *face_hit = face_lo;
        return 0;
    }
    if (c >= n) {
        if (bc_hi == SPFM_PERIODIC) return c - n;
        if (bc_hi == SPFM_CONTACT) *face_hit = face_lo + 1;
        return n - 1;
    }
    return c;
}

// Eq. 7 with a signed coupling a: value at a ghost displaced from its source.
template <class T>
__host__ __device__ inline T contact_shift(T v, T a)
{
    return (T(1) - a) * v / (T(1) - a * (T(2) * v - T(1)));
}
// The same with every operation rounded on its own (no contraction into FMAs),
// so that the ghost layer is a fixed function of the interior, bit for bit
// (the face kernel uses it).
#ifdef __CUDACC__
__device__ inline float contact_shift_rn(float v, float a)
{
    const float d = __fsub_rn(1.0f, __fmul_rn(a, __fsub_rn(__fmul_rn(2.0f, v), 1.0f)));
    return __fdiv_rn(__fmul_rn(__fsub_rn(1.0f, a), v), d);
}
__device__ inline double contact_shift_rn(double v, double a)
{
    const double d = __dsub_rn(1.0, __dmul_rn(a, __dsub_rn(__dmul_rn(2.0, v), 1.0)));
    return __ddiv_rn(__dmul_rn(__dsub_rn(1.0, a), v), d);
}
#endif


// ---------------------------------------------------------------- launchers

struct LaunchCfg {
    int stencil;   // 6, 18, 26
    int scheme;    // SPFM_TI_GLOBAL, SPFM_TI_LOCAL, SPFM_FD
    int mode;      // kWaitFaces | kWaitAll | kImages
    int rounding = SPFM_ROUND_NEAREST;   // SPFM_ROUND_STOCHASTIC: the *_sr kernels
    int zchunk = 0;   // planes per CTA; 0: pick_zchunk
    int *zchunk_used = nullptr;   // receives the planes per CTA of the launch (host, optional)
};

// Planes per CTA of a step launch of `tiles` xy tiles over nz planes by kernel
// `kern` of `threads` threads (launch_shape.cu); target: the CTA count of six
// rounds at the kernel family's design occupancy.  Cached per kernel and shape.
int pick_zchunk(const void *kern, int threads, int tiles, int nz, int target);

// How a step launch sits in the stream (programmatic dependent launch):
//   kWaitFaces  the previous kernel refreshes src's ghosts: boxes touching a face wait for it
//   kWaitAll    every box waits for the previous kernel
//   kImages     all faces periodic: the step writes the ghost images of its new cells
//               itself (no face kernel follows) and lets the next step launch early
//   kSkipCopy   test of the bounded waits: the first CTA skips one plane's copy
//               (spfm_debug_skip_copy), its waits give up and set the error word
//   kEarly      no face kernel follows (no periodic face: the step computes the
//               ghosts of the non-periodic faces as it reads them): the step lets
//               the next one launch at its start, like the image-writing kernels
constexpr int kWaitFaces = 1, kWaitAll = 2, kImages = 4, kSkipCopy = 8, kEarly = 16;

// TMA tensor maps of a grid's two field buffers, encoded on first use (tma.cu).
struct TmaCache {
    CUtensorMap map[4];   // [buffer] for the single-grid box, [2 + buffer] for the square batch box
    const void *base[4];
    int state[4];   // 0 not encoded, 1 encoded, -1 encoding unavailable (row copies)
};

// Encode a 3D tiled map over a ghosted buffer with a (box_x, box_y, 1) box.
// Returns 0 on success.
int encode_field_map(CUtensorMap *map, const GridGeom &g, int dtype, const void *base, int box_x,
                     int box_y);

// The map of buffer `which` (base), encoded on demand; NULL when unavailable.
const CUtensorMap *cached_map(TmaCache *cache, int which, const GridGeom &g, int dtype,
                              const void *base, int box_x, int box_y);

// One explicit step src -> dst of one grid (step_f32.cu / step_f64.cu / step_bf16.cu;
// with kImages in cfg.mode the *_img.cu kernels).
// err: device word that a kernel sets when one of its bounded waits gives up.
// tma: map cache of the grid (NULL: row-wise bulk copies); which: index of src.
cudaError_t launch_step_f32(const StepCoef<float> &c, const float *src, float *dst, int *err,
                            LaunchCfg cfg, TmaCache *tma, int which, cudaStream_t st);
cudaError_t launch_step_f64(const StepCoef<double> &c, const double *src, double *dst, int *err,
                            LaunchCfg cfg, TmaCache *tma, int which, cudaStream_t st);
cudaError_t launch_step_bf16(const StepCoef<float> &c, const __nv_bfloat16 *src,
                             __nv_bfloat16 *dst, int *err, LaunchCfg cfg, TmaCache *tma, int which,
                             cudaStream_t st);
// the same, for all-periodic grids whose step writes its own ghost images (kImages)
cudaError_t launch_step_f32_img(const StepCoef<float> &c, const float *src, float *dst, int *err,
                                LaunchCfg cfg, TmaCache *tma, int which, cudaStream_t st);
cudaError_t launch_step_f64_img(const StepCoef<double> &c, const double *src, double *dst, int *err,
                                LaunchCfg cfg, TmaCache *tma, int which, cudaStream_t st);
cudaError_t launch_step_bf16_img(const StepCoef<float> &c, const __nv_bfloat16 *src,
                                 __nv_bfloat16 *dst, int *err, LaunchCfg cfg, TmaCache *tma, int which,
                                 cudaStream_t st);
// the same with stochastic rounding of the update (step_*_sr.cu; cfg.rounding
// set; the dispatch above forwards to them)
cudaError_t launch_step_f32_sr(const StepCoef<float> &c, const float *src, float *dst, int *err, LaunchCfg cfg,
                               TmaCache *tma, int which, cudaStream_t st);
cudaError_t launch_step_f32_img_sr(const StepCoef<float> &c, const float *src, float *dst, int *err,
                                   LaunchCfg cfg, TmaCache *tma, int which, cudaStream_t st);
cudaError_t launch_step_bf16_sr(const StepCoef<float> &c, const __nv_bfloat16 *src, __nv_bfloat16 *dst,
                                int *err, LaunchCfg cfg, TmaCache *tma, int which, cudaStream_t st);
cudaError_t launch_step_bf16_img_sr(const StepCoef<float> &c, const __nv_bfloat16 *src, __nv_bfloat16 *dst,
                                    int *err, LaunchCfg cfg, TmaCache *tma, int which, cudaStream_t st);

// Initial ideal profiles and FP64 diagnostics (stats.cu).
struct InitArgs {
    GridGeom g;
    int dtype;
    int shape;            // 0 planar (n, c), 1 radial (ctr, R), 2 cube (ctr, half)
    double n[3], c;
    double ctr[3], R, half;
    double lambda, dx;
};
cudaError_t launch_init(const InitArgs &a, void *field, cudaStream_t st);

// Constant-volume correction after a step at dF = 0 (conserve.cu): dst -=
// alpha q(src) with alpha = sum(dst - src) / sum q(src); partials holds
// 2 * kStatsBlocks doubles, alpha_out (device) receives alpha.
cudaError_t launch_conserve(const GridGeom &g, int dtype, const void *src, void *dst, double *partials,
                            double *alpha_out, cudaStream_t st);

// Interior of dst = interior of src shifted along x by cells (frame.cu).
cudaError_t launch_shift_x(const GridGeom &g, int dtype, const void *src, void *dst, int cells, cudaStream_t st);

// Ghost layer of a buffer from its interior: all faces (x_faces = 1) or the y
// and z faces only.  Face sizes must stay below 2^31 cells.
cudaError_t launch_fill_ghosts(const GridGeom &g, int dtype, const double aface[6], void *field,
                               cudaStream_t st, int x_faces);

struct StatsArgs {
    GridGeom g;
    int dtype;
    double n[3], ctr[3];
    double lambda, dx;
    int energy;           // 1: also accumulate the interface energy
    int scheme, stencil;  // energy model
    double Gamma, C_gamma;
    double w[kMaxTerms];  // w_k = gamma_j nu_j (0 where inactive)
    double a[kMaxTerms];  // TI coupling a_k(n)
};
// Writes kNStat doubles of the final reduction to final_out (device).
cudaError_t launch_stats(const StatsArgs &a, const void *field, double *partials,
                         double *final_out, cudaStream_t st);

// Scratch of one grid: stats partials, the final reduction, then the error word.
size_t stats_scratch_bytes();
inline size_t scratch_final_offset() { return sizeof(double) * (size_t)kNStat * kStatsBlocks; }
inline size_t scratch_err_offset() { return sizeof(double) * (size_t)kNStat * (kStatsBlocks + 1); }
size_t grid_scratch_bytes();

// ---------------------------------------------------------------- batches

// One tile of a batch's packed work-list: grid, tile column/row, z range.
struct BatchItem {
    int grid, bx, by, zc0, zc1;
    int shape;   // tile shape of the item (0: the single-grid shape; 1: the square FP32 shape)
};

// Per-dtype pieces of the persistent batch kernel (step_f32.cu / ...):
// bytes of one device-side grid record, the work-list items of one grid, the
// record of one grid, and the launch of one step over the whole work-list
// (kind: 0 CF, else TI with up to 13 groups).
size_t batch_grid_bytes_f32();
size_t batch_grid_bytes_f64();
size_t batch_grid_bytes_bf16();
// (shape 1 exists for FP32 only; the FP64 and BF16 items are always shape 0)
int batch_items_f32(const GridGeom &g, int grid_index, int zchunk, BatchItem *out, int shape);
int batch_items_f64(const GridGeom &g, int grid_index, int zchunk, BatchItem *out, int shape);
int batch_items_bf16(const GridGeom &g, int grid_index, int zchunk, BatchItem *out, int shape);
void batch_fill_grid_f32(void *slot, const StepCoef<float> &c, void *const field[2], int cur, TmaCache *tma);
void batch_fill_grid_f64(void *slot, const StepCoef<double> &c, void *const field[2], int cur, TmaCache *tma);
void batch_fill_grid_bf16(void *slot, const StepCoef<float> &c, void *const field[2], int cur, TmaCache *tma);
// sr: stochastic rounding (the *_sr kernels), whose step keys come from
// steps[grid] (device: each grid's step count at the start of the call) + sub
// (the launch's position in the call)
// fwd: no grid of the batch has a periodic face; the kernel stages the ghosts
// of the faces and no ghost kernel has to run
cudaError_t launch_batch_f32(const void *grids, const BatchItem *work, int nwork, int parity, int *err,
                             int stencil, int kind, cudaStream_t st, int shape, int sr, const long long *steps,
                             int sub, int fwd);
cudaError_t launch_batch_f64(const void *grids, const BatchItem *work, int nwork, int parity, int *err,
                             int stencil, int kind, cudaStream_t st, int fwd);
cudaError_t launch_batch_bf16(const void *grids, const BatchItem *work, int nwork, int parity, int *err,
                              int stencil, int kind, cudaStream_t st, int sr, const long long *steps, int sub,
                              int fwd);
cudaError_t launch_batch_f32_sr(const void *grids, const BatchItem *work, int nwork, int parity, int *err,
                                int stencil, int kind, cudaStream_t st, int shape, const long long *steps, int sub,
                                int fwd);
cudaError_t launch_batch_bf16_sr(const void *grids, const BatchItem *work, int nwork, int parity, int *err,
                                 int stencil, int kind, cudaStream_t st, const long long *steps, int sub, int fwd);
// steps[i] += k for the n grids of a batch (after the k steps of a call or graph)
cudaError_t launch_advance_steps(long long *steps, int n, int k, cudaStream_t st);

// Ghost refresh of every grid of a batch: job i fills buffer cur ^ parity of grid i.
struct GhostJob {
    GridGeom g;
    double aface[6];
    void *field[2];
    int cur;
};
cudaError_t launch_fill_ghosts_batch(const GhostJob *jobs, int n, int dtype, int parity, cudaStream_t st);

// Diagnostics of every grid of a batch: job i reads buffer cur of grid i; the
// final reduction of grid i lands in finals[i * kNStat ..].
struct StatsJob {
    StatsArgs a;
    const void *field[2];
    int cur;
};
constexpr int kBatchStatsBlocks = 32;   // partial blocks per grid
cudaError_t launch_stats_batch(const StatsJob *jobs, int n, int dtype, double *partials, double *finals,
                               cudaStream_t st);

}  // namespace spfm
