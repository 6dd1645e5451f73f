// stats.cu -- ideal-profile initialisation and FP64 interface
// diagnostics on the ghosted field layout (spfm_internal.h).
//
// init: Eq. 3 (planar), its radial form, or a cube as the product of three 1D
// profiles (the start of the Sec. 3.3 shape relaxation), evaluated in FP64 per cell and
// rounded once to the storage type (the caller then fills the ghost layer).
//
// stats: one pass over the interior with sums per lane in a fixed order
// (double-float pairs for the band sums, FP64 otherwise, see below), then
// FP64 warp-shuffle and shared-memory block reductions into
// kStatsBlocks partials, then one CTA reducing the partials in a fixed order,
// so the result is bit-reproducible for a given grid size.  Sums over the band
// 1e-6 < phi < 1 - 1e-6 invert the ideal profile (Sec. 2.3):
//   position  c = sum q (p.n - (lambda/2) artanh(1-2phi)) / sum q
//   radius    R = sum q (|p - ctr| + (lambda/2) artanh(1-2phi)) / sum q
// The optional interface energy is Eq. 1 at dF = 0; its forward differences
// read the ghost layer.
#include <math.h>

#include <mutex>

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
                if (a.shape == 1) {
                    const double rx = px - a.ctr[0], ry = py - a.ctr[1], rz = pz - a.ctr[2];
                    const double rr = sqrt(rx * rx + ry * ry + rz * rz);
                    v = 0.5 * (1.0 - tanh(2.0 * (a.R - rr) / a.lambda));
                } else if (a.shape == 2) {
                    // cube: product of the three 1D particle fractions
                    const double d[3] = {px - a.ctr[0], py - a.ctr[1], pz - a.ctr[2]};
                    double inside = 1.0;
                    for (int ax = 0; ax < 3; ++ax) inside *= 0.5 * (1.0 - tanh(2.0 * (fabs(d[ax]) - a.half) / a.lambda));
                    v = 1.0 - inside;
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

// Per-lane partials: [0] sum phi, [1] S_w, [2] S_c, [3] S_r, [4] min, [5] max,
// [6] non-finite count, [7] energy density sum, [8..11] unused.
//
// The pass is bound by the FP64 work of the band cells (GB300 issues FP64 at
// 1/64 of the FP32 rate), so everything else stays out of FP64:
//   - each warp walks whole rows with 16-byte loads; finiteness, min, max and
//     the band test run in the storage precision, where they are exact (the
//     band limits 1e-6 and 1 - 1e-6 are not floats, so the first float above
//     and the last float below them decide exactly the same cells);
//   - an FP32 field's volume is summed per lane and row as an unevaluated pair
//     (TwoSum, Knuth TAOCP vol. 2, 4.2.2), carried in 2^-48 fixed point;
//   - band cells are queued per warp and evaluated 32 at a time, so the FP64
//     inversion of the profile runs with every lane busy.
template <class S> struct Scr { using T = float; };
template <> struct Scr<double> { using T = double; };
template <class S> __device__ __forceinline__ typename Scr<S>::T scr(const S *f, long long i);
template <> __device__ __forceinline__ double scr<double>(const double *f, long long i) { return f[i]; }
template <> __device__ __forceinline__ float scr<float>(const float *f, long long i) { return f[i]; }
template <> __device__ __forceinline__ float scr<__nv_bfloat16>(const __nv_bfloat16 *f, long long i)
{
    return __bfloat162float(f[i]);
}

// 16 bytes of a row as storage elements, widened to the screening type
template <class S> struct Row16;
template <> struct Row16<float> {
    static constexpr int E = 4;
    static __device__ __forceinline__ float get(const uint4 &w, int e)
    {
        return __uint_as_float(e == 0 ? w.x : e == 1 ? w.y : e == 2 ? w.z : w.w);
    }
};
template <> struct Row16<__nv_bfloat16> {
    static constexpr int E = 8;
    static __device__ __forceinline__ float get(const uint4 &w, int e)
    {
        const unsigned u = (e >> 1) == 0 ? w.x : (e >> 1) == 1 ? w.y : (e >> 1) == 2 ? w.z : w.w;
        return __uint_as_float((e & 1) ? (u & 0xffff0000u) : (u << 16));
    }
};
template <> struct Row16<double> {
    static constexpr int E = 2;
    static __device__ __forceinline__ double get(const uint4 &w, int e)
    {
        return e == 0 ? __hiloint2double((int)w.y, (int)w.x) : __hiloint2double((int)w.w, (int)w.z);
    }
};

// 1e-6 < x < 1 - 1e-6 for an FP32 x: the limits are not FP32 numbers, so the
// test compares with the first float above 1e-6 and the last float below
// 1 - 1e-6 (written out: a rounding conversion here would run on the FP64 pipe
// for every cell)
__device__ __forceinline__ bool in_band(float x)
{
    return x >= 0x1.0c6f7cp-20f && x <= 0x1.ffffdep-1f;
}
__device__ __forceinline__ bool in_band(double x) { return x > 1e-6 && x < 1.0 - 1e-6; }

// y * 2^48 truncated toward zero, for |y| < 2^14 (the bits below 2^-48 drop)
__device__ __forceinline__ long long fix48(float y)
{
    const unsigned b = __float_as_uint(y);
    const int E = (int)((b >> 23) & 0xffu);
    if (E < 78) return 0;   // |y| < 2^-49
    const long long m = (long long)((b & 0x7fffffu) | 0x800000u);   // |y| = m 2^(E - 150)
    const int sh = E - 102;
    const long long v = sh >= 0 ? (m << sh) : (m >> (-sh));
    return (b >> 31) ? -v : v;
}

// Volume of one lane.  FP32 values: each row as an unevaluated pair s + c
// (TwoSum), then the pair in 2^-48 fixed point (exact to the dropped bits,
// below 4e-15 per row), carried into FP64 every 64 rows, before the fixed
// point could overflow.
template <class R> struct VolSum;
template <> struct VolSum<float> {
    float s = 0.0f, c = 0.0f;
    long long fix = 0;
    double sum = 0.0;
    int rows = 0;
    __device__ __forceinline__ void add(float x)
    {
        const float t = s + x, z = t - s;
        c += (s - (t - z)) + (x - z);
        s = t;
    }
    __device__ __forceinline__ void end_row()
    {
        if (fabsf(s) < 256.0f) fix += fix48(s) + fix48(c);
        else sum += (double)s + (double)c;
        s = c = 0.0f;
        if (++rows == 64) {
            sum += (double)fix * 0x1p-48;
            fix = 0;
            rows = 0;
        }
    }
    __device__ __forceinline__ double total() const { return sum + (double)fix * 0x1p-48; }
};
template <> struct VolSum<double> {
    double sum = 0.0;
    __device__ __forceinline__ void add(double x) { sum += x; }
    __device__ __forceinline__ void end_row() {}
    __device__ __forceinline__ double total() const { return sum; }
};

// ---- double-float arithmetic: a value is hi + lo in two FP32 numbers with
// |lo| <= ulp(hi)/2 (Dekker, Numer. Math. 18, 1971; Knuth, TAOCP 2, 4.2.2).
// About 48 significant bits at the FP32 rate, 64 times the FP64 rate of this
// GPU.  The error-free transforms use the _rn intrinsics, which the compiler
// neither contracts into FMAs nor reassociates.
struct DF {
    float hi, lo;
};
__device__ __forceinline__ DF df_two_sum(float a, float b)   // a + b exactly
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ DF df_fast_sum(float a, float b)  // a + b exactly, |a| >= |b| or a = 0
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF df_two_prod(float a, float b)  // a b exactly
{
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
// a + b with absolute error about 2^-48 max(|a|, |b|)
__device__ __forceinline__ DF df_add(DF a, DF b)
{
    const DF s = df_two_sum(a.hi, b.hi);
    return df_fast_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
// a + b with the low parts also added error-free, for running sums
__device__ __forceinline__ DF df_add_acc(DF a, DF b)
{
    DF s = df_two_sum(a.hi, b.hi);
    const DF t = df_two_sum(a.lo, b.lo);
    s = df_fast_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return df_fast_sum(s.hi, __fadd_rn(s.lo, t.lo));
}
__device__ __forceinline__ DF df_neg(DF a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ DF df_mul(DF a, DF b)
{
    const DF p = df_two_prod(a.hi, b.hi);
    return df_fast_sum(p.hi, __fadd_rn(p.lo, __fmaf_rn(a.hi, b.lo, __fmul_rn(a.lo, b.hi))));
}
__device__ __forceinline__ DF df_mul_f(DF a, float b)
{
    const DF p = df_two_prod(a.hi, b);
    return df_fast_sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}
__host__ __device__ __forceinline__ DF df_of(double x)
{
    const float h = (float)x;
    return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ double df_to_double(DF a) { return (double)a.hi + (double)a.lo; }
// an integer index as an exact pair (|n| < 2^48)
__device__ __forceinline__ DF df_of_int(int n)
{
    const float h = (float)n;
    return {h, (float)(n - (int)h)};
}
// sqrt of a non-negative value: the FP32 root s and one Newton step,
// s + (a - s^2) / (2 s), with s^2 formed exactly
__device__ __forceinline__ DF df_sqrt(DF a)
{
    if (!(a.hi > 0.0f)) return {0.0f, 0.0f};
    const float s = sqrtf(a.hi);
    const DF s2 = df_two_prod(s, s);
    const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, s2.hi), s2.lo), a.lo);
    // the correction is about 2^-24 of s: an approximate reciprocal keeps the pair's accuracy
    return df_fast_sum(s, __fmul_rn(r, __fdividef(0.5f, s)));
}

// Tables of the band evaluation, as double-float pairs written from FP64:
// g_ln_tab[j] = (ln F_j, 1/F_j) for F_j = 1 + j/256, g_kln2[k + 64] = k ln 2.
__device__ float4 g_ln_tab[256];
__device__ float2 g_kln2[128];

__global__ void ln_table_kernel()
{
    const int j = threadIdx.x;
    const double F = 1.0 + j / 256.0;
    const DF l = df_of(log(F)), r = df_of(1.0 / F);
    g_ln_tab[j] = make_float4(l.hi, l.lo, r.hi, r.lo);
    if (j < 128) {
        const DF k = df_of((double)(j - 64) * 0.69314718055994530942);
        g_kln2[j] = make_float2(k.hi, k.lo);
    }
}

// ln y for y = hi + lo in [2^-126, 1], table-driven (Tang, ACM TOMS 16, 1990):
// hi = 2^k m, m in [1, 2); F = 1 + j/256 takes the top 8 fraction bits of m, so
// f = (m - F) + lo 2^-k holds y 2^-k - F to double-float accuracy and u = f/F
// lies in (-2^-24, 2^-8).  ln(1 + u) is its Taylor series: u - u^2/2 in
// double-float, the terms u^3/3 - u^4/4 + u^5/5 (below 2e-8) in FP32,
// truncation below u^6/6 < 6e-16.  Returned as k, ln F and ln(1 + u).
struct LnParts {
    int k;
    DF lnF, s;
};
__device__ __forceinline__ LnParts ln_parts(DF y, const float4 *tab)
{
    const int bits = __float_as_int(y.hi);
    LnParts r;
    r.k = ((bits >> 23) & 0xff) - 127;
    const int j = (bits >> 15) & 0xff;
    const float m = __int_as_float((bits & 0x007fffff) | 0x3f800000);
    const float F = __int_as_float(0x3f800000 | (j << 15));
    const float lo = __fmul_rn(y.lo, __int_as_float((127 - r.k) << 23));   // lo 2^-k, exact
    const float4 t = tab[j];
    r.lnF = {t.x, t.y};
    const DF u = df_mul(df_two_sum(__fsub_rn(m, F), lo), DF{t.z, t.w});
    const DF u2 = df_mul(u, u);
    const float uh = u.hi;
    const float tail = uh * uh * uh * fmaf(uh, fmaf(uh, 0.2f, -0.25f), 1.0f / 3.0f);
    r.s = df_add(df_add(u, DF{-0.5f * u2.hi, -0.5f * u2.lo}), DF{tail, 0.0f});
    return r;
}

// one band cell waiting in its warp's queue: value, x index, and its row's
// share of p.n and of |p - ctr|^2
template <class R> struct BandCell {
    R phi;
    int i;
    DF pn_row, ryz2;
};

// Sec. 2.3 sums of one band cell, in double-float: q = phi(1 - phi),
// psi = (lambda/2) artanh(1 - 2 phi) = (lambda/4) (ln(1 - phi) - ln phi),
// p = dx (i, j, k).  Absolute error of psi below about 1e-13.
struct BandConst {
    DF dxn0, dxn1, dxn2, dx, neg_c0, neg_c1, neg_c2, quarter_lambda;
};
template <class R> struct BandPhi;
template <> struct BandPhi<float> {   // FP32 and BF16 storage: phi exact, 1 - phi exact as a pair
    static __device__ __forceinline__ void get(float x, DF &ph, DF &om)
    {
        ph = {x, 0.0f};
        om = df_fast_sum(1.0f, -x);
    }
};
template <> struct BandPhi<double> {  // FP64 storage: 1 - phi in FP64, then both as pairs
    static __device__ __forceinline__ void get(double x, DF &ph, DF &om)
    {
        ph = df_of(x);
        om = df_of(1.0 - x);
    }
};
struct BandSums {
    DF w{0.0f, 0.0f}, c{0.0f, 0.0f}, r{0.0f, 0.0f};   // S_w, S_c, S_r
};
template <class R>
__device__ __forceinline__ void band_cell(const BandConst &bc, const BandCell<R> &c, const float4 *tab,
                                          const float2 *kln2, BandSums &acc)
{
    DF ph, om;
    BandPhi<R>::get(c.phi, ph, om);
    const DF q = df_mul(ph, om);
    const LnParts l1 = ln_parts(om, tab), l0 = ln_parts(ph, tab);
    const float2 kl = kln2[l1.k - l0.k + 64];
    DF d = df_add(DF{kl.x, kl.y}, df_add(l1.lnF, df_neg(l0.lnF)));
    d = df_add(d, df_add(l1.s, df_neg(l0.s)));
    const DF psi = df_mul(bc.quarter_lambda, d);
    const DF fi = df_of_int(c.i);
    const DF pn = df_add(c.pn_row, df_mul(bc.dxn0, fi));
    const DF rx = df_add(df_mul(bc.dx, fi), bc.neg_c0);
    const DF r = df_sqrt(df_add(df_mul(rx, rx), c.ryz2));
    acc.w = df_add_acc(acc.w, q);
    acc.c = df_add_acc(acc.c, df_mul(q, df_add(pn, df_neg(psi))));
    acc.r = df_add_acc(acc.r, df_mul(q, df_add(r, psi)));
}

// Partial sums of block b of nb (256 threads): rows ordered (j fastest, k) are
// dealt round-robin to the nb * 8 warps, so every block samples the whole
// grid and the band work (which sits in a few planes) is spread evenly.
template <class S>
__device__ __forceinline__ void stats_pass(const StatsArgs &a, const S *f, double *partial_out,
                                           long long blk, long long nblk)
{
    using R = typename Scr<S>::T;
    constexpr int E = Row16<S>::E;        // elements per 16-byte load
    constexpr int V = 16 / E;             // loads per lane and sweep
    constexpr int kWarps = 8;
    // Per warp: a ring of band cells (value, x index) with the slot of their
    // row's shares; a sweep is queued in four parts of at most 128 cells and
    // full warps of 32 are evaluated after each, so fewer than 32 wait between
    // parts and a part always fits.  Waiting cells come from fewer than 32 rows,
    // so 32 row slots, taken in turn, are never overwritten while referenced.
    constexpr int kRing = 256, kRowSlots = 32;
    __shared__ R ring_phi[kWarps][kRing];
    __shared__ int ring_i[kWarps][kRing];
    __shared__ unsigned char ring_slot[kWarps][kRing];
    __shared__ DF row_tab[kWarps][kRowSlots][2];
    const float4 *tab = g_ln_tab;
    const float2 *kln2 = g_kln2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double v[kNStat];
#pragma unroll
    for (int i = 0; i < kNStat; ++i) v[i] = 0.0;
    R mn = R(INFINITY), mx = R(-INFINITY);
    int nonfinite = 0;
    const BandConst bconst = {df_of(a.dx * a.n[0]), df_of(a.dx * a.n[1]), df_of(a.dx * a.n[2]), df_of(a.dx),
                              df_of(-a.ctr[0]),      df_of(-a.ctr[1]),      df_of(-a.ctr[2]), df_of(0.25 * a.lambda)};
    BandSums sums;
    int head = 0, tail = 0, band_rows = 0;   // ring positions and band rows so far (warp-uniform)
    // evaluate the waiting cell at ring position q (this lane's)
    auto eval_at = [&](int q) {
        const int r = q & (kRing - 1);
        BandCell<R> c;
        c.phi = ring_phi[warp][r];
        c.i = ring_i[warp][r];
        const int sl = ring_slot[warp][r];
        c.pn_row = row_tab[warp][sl][0];
        c.ryz2 = row_tab[warp][sl][1];
        band_cell<R>(bconst, c, tab, kln2, sums);
    };
    VolSum<R> vol;
    const long long rows = (long long)a.g.ny * a.g.nz;
    const int nvec = (a.g.nx + E - 1) / E;
    // rows (j, k) dealt round-robin to the warps; ny nz < 2^30, and (j, k)
    // advance by the stride's split so that no row divides (64-bit division
    // is emulated in FP64, the slow pipe of this GPU)
    const long long row0 = blk * kWarps + warp, stride = nblk * kWarps;
    const int sj = (int)(stride % a.g.ny), sk = (int)(stride / a.g.ny);
    for (int j = (int)(row0 % a.g.ny), k = (int)(row0 / a.g.ny); k < a.g.nz;
         j += sj, k += sk, (j >= a.g.ny ? (j -= a.g.ny, ++k) : 0)) {
        bool row_known = false;   // the row's shares are in its slot
        int slot = 0;
        const uint4 *src = (const uint4 *)(f + cell_index(a.g, 0, j, k));
        for (int v0 = 0; v0 < nvec; v0 += 32 * V) {
            uint4 w[V];
#pragma unroll
            for (int t = 0; t < V; ++t) {
                const int vi = v0 + 32 * t + lane;
                w[t] = vi < nvec ? __ldg(src + vi) : make_uint4(0u, 0u, 0u, 0u);
            }
            unsigned bm = 0u;   // band cells of this lane among its E * V
#pragma unroll
            for (int t = 0; t < V; ++t)
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int i = (v0 + 32 * t + lane) * E + e;
                    const R x = Row16<S>::get(w[t], e);
                    if (i < a.g.nx) {
                        if (!isfinite(x)) {
                            ++nonfinite;
                        } else {
                            vol.add(x);
                            mn = x < mn ? x : mn;
                            mx = x > mx ? x : mx;
                            if (in_band(x)) bm |= 1u << (t * E + e);
                        }
                    }
                }
            if (__any_sync(0xffffffffu, bm != 0u)) {
                if (!row_known) {
                    // the row's shares of p.n and |p - ctr|^2, in double-float (FP64
                    // is the slow pipe of this GPU)
                    slot = band_rows++ & (kRowSlots - 1);
                    if (lane == 0) {
                        const DF fj = df_of_int(j), fk = df_of_int(k);
                        const DF ry = df_add(df_mul(bconst.dx, fj), bconst.neg_c1);
                        const DF rz = df_add(df_mul(bconst.dx, fk), bconst.neg_c2);
                        row_tab[warp][slot][0] = df_add(df_mul(bconst.dxn1, fj), df_mul(bconst.dxn2, fk));
                        row_tab[warp][slot][1] = df_add(df_mul(ry, ry), df_mul(rz, rz));
                    }
                    row_known = true;
                }
                // queue the sweep's band cells in four parts (a warp prefix sum
                // places each lane's cells), evaluating full warps after each
#pragma unroll
                for (int part = 0; part < 4; ++part) {
                    const unsigned m = (bm >> (4 * part)) & 0xfu;
                    const int c = __popc(m);
                    int incl = c;
#pragma unroll
                    for (int d = 1; d < 32; d <<= 1) {
                        const int y = __shfl_up_sync(0xffffffffu, incl, d);
                        if (lane >= d) incl += y;
                    }
                    int pos = tail + incl - c;
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        constexpr int kE = E;
                        const int b = 4 * part + u;
                        if (m & (1u << u)) {
                            const int r = pos & (kRing - 1);
                            ring_phi[warp][r] = Row16<S>::get(w[b / kE], b % kE);
                            ring_i[warp][r] = (v0 + 32 * (b / kE) + lane) * kE + b % kE;
                            ring_slot[warp][r] = (unsigned char)slot;
                            ++pos;
                        }
                    }
                    tail += __shfl_sync(0xffffffffu, incl, 31);
                    __syncwarp();
                    for (; tail - head >= 32; head += 32) eval_at(head + lane);
                    __syncwarp();   // reads of evaluated cells before the next part's writes
                }
            }
        }
        vol.end_row();
    }
    v[0] = vol.total();
    if (lane < tail - head) eval_at(head + lane);
    v[1] = df_to_double(sums.w);
    v[2] = df_to_double(sums.c);
    v[3] = df_to_double(sums.r);
    v[4] = (double)mn;
    v[5] = (double)mx;
    v[6] = (double)nonfinite;
    if (a.energy) {   // Eq. 1 at dF = 0, one cell per thread, contiguous rows per block
        const long long r0 = blk * rows / nblk, r1 = (blk + 1) * rows / nblk;
        const double e_pref = a.Gamma / (a.C_gamma * a.lambda);
        const int nd = a.stencil == 6 ? 3 : (a.stencil == 18 ? 9 : 13);
        for (long long row = r0; row < r1; ++row) {
            const int j = (int)(row % a.g.ny), k = (int)(row / a.g.ny);
            const long long rbase = cell_index(a.g, 0, j, k);
            for (int i = threadIdx.x; i < a.g.nx; i += blockDim.x) {
                const double ph = rd<S>(f, rbase + i);
                if (!isfinite(ph)) continue;
                double e = 0.0;
                for (int kk = 0; kk < nd; ++kk) {
                    const Dir d = grid_dir(kk);
                    const double r2 = (double)d.shell * a.dx * a.dx;
                    const double nb = rd<S>(f, cell_index(a.g, i + d.x, j + d.y, k + d.z));
                    const double dp = nb - ph;
                    e += a.w[kk] * (0.5 * a.lambda * a.lambda * dp * dp / r2 +
                                    potential(ph, a.a[kk], a.lambda * a.lambda / r2, is_fd_scheme(a.scheme)));
                }
                v[7] += e_pref * e;
            }
        }
    }
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

// The logarithm table of the band evaluation, written once per device by a
// kernel on the calling stream and waited for, so that calls on other streams
// can rely on it.  Inside a stream capture the writer is recorded into the
// graph instead (it cannot be waited for there) and the device stays unmarked.
static cudaError_t ensure_ln_table(cudaStream_t st)
{
    static std::mutex mu;
    static bool ready[128];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (ready[dev]) return cudaSuccess;
    ln_table_kernel<<<1, 256, 0, st>>>();
    e = cudaGetLastError();
    if (e != cudaSuccess || cs != cudaStreamCaptureStatusNone) return e;
    e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) ready[dev] = true;
    return e;
}

// One full wave of stats blocks on this device (at most kStatsBlocks): the
// band cells sit in a few planes and are spread over all warps, so a partial
// second wave would idle SMs.
template <class S> static int stats_blocks()
{
    static int cached[128];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return kStatsBlocks;
    if (!cached[dev]) {
        int per = 0, sms = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, stats_kernel<S>, 256, 0) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return kStatsBlocks;
        const int n = per * sms;
        cached[dev] = n < 1 ? 1 : (n > kStatsBlocks ? kStatsBlocks : n);
    }
    return cached[dev];
}

cudaError_t launch_stats(const StatsArgs &a, const void *field, double *partials, double *final_out,
                         cudaStream_t st)
{
    cudaError_t e = ensure_ln_table(st);
    if (e != cudaSuccess) return e;
    int nb;
    if (a.dtype == SPFM_F64) {
        nb = stats_blocks<double>();
        stats_kernel<double><<<nb, 256, 0, st>>>(a, (const double *)field, partials);
    } else if (a.dtype == SPFM_F32) {
        nb = stats_blocks<float>();
        stats_kernel<float><<<nb, 256, 0, st>>>(a, (const float *)field, partials);
    } else {
        nb = stats_blocks<__nv_bfloat16>();
        stats_kernel<__nv_bfloat16><<<nb, 256, 0, st>>>(a, (const __nv_bfloat16 *)field, partials);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    stats_final_kernel<<<1, 256, 0, st>>>(partials, nb, final_out);
    return cudaGetLastError();
}

cudaError_t launch_stats_batch(const StatsJob *jobs, int n, int dtype, double *partials, double *finals,
                               cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    cudaError_t e = ensure_ln_table(st);
    if (e != cudaSuccess) return e;
    const dim3 grid(kBatchStatsBlocks, n);
    if (dtype == SPFM_F64) stats_batch_kernel<double><<<grid, 256, 0, st>>>(jobs, partials);
    else if (dtype == SPFM_F32) stats_batch_kernel<float><<<grid, 256, 0, st>>>(jobs, partials);
    else stats_batch_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(jobs, partials);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    stats_final_kernel<<<n, 256, 0, st>>>(partials, kBatchStatsBlocks, finals);
    return cudaGetLastError();
}

}  // namespace spfm
