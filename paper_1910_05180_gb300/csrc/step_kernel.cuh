// step_kernel.cuh -- z-marching 2.5D stencil kernel of one explicit SPFM / CF step.
//
// Data movement.  Every field buffer carries a one-cell ghost layer in HBM
// (spfm_internal.h), so a tile plus its halo is a set of plain, in-bounds,
// 16-byte-aligned rows.  One CTA owns an xy tile of TX*VX by TY cells
// (VX = cells per 16 bytes) and marches a chunk of z planes.  A producer warp
// brings each plane's tile plus halo into a ring of NS shared-memory stages
// with one TMA tensor copy (cp.async.bulk.tensor.3d over a tensor map of the
// ghosted buffer), or, where no map could be encoded, with one bulk copy per
// halo row (cp.async.bulk); both complete on the stage's "full" mbarrier by
// transaction count.  TX*TY consumer threads wait on "full", read the stage,
// and release it on its "empty" barrier.  There is no __syncthreads in the
// march, and NS-1 planes stay in flight per CTA.  Every wait is bounded: on
// timeout the thread sets the error word and leaves.
//
// Boundary conditions.  The kernel reads the ghost layer.  In general it
// writes interior cells only and a face kernel (boundary.cu) refreshes the
// ghosts of the new field after each step; under programmatic dependent launch
// the next step starts while that kernel runs, and tiles whose halo touches a
// face wait for it (griddepcontrol.wait), interior tiles do not.  When every
// face is periodic and a row is a whole number of 32-byte sectors, the ghosts
// are plain periodic images: the thread that writes a cell next to a face also
// writes its image(s) on the far side (x images as whole 32-byte sectors of
// the row pads, two threads a sector), so no face kernel runs, and the next
// step waits for this one in every tile.
//
// Arithmetic.  From each plane every thread forms, for its cells,
//   C  = phi at the cell,
//   F' = sum of the 4 in-plane face neighbours minus C (each as a difference),
//   E' = sum of the 4 in-plane diagonal neighbours minus C,
// kept in registers for the planes z-1, z, z+1 (the z loop is unrolled by
// three with rotating register roles).  The shell sums then follow:
//   S1 - 6 phi  = F'_z + t,             t = (C_{z-1} - phi) + (C_{z+1} - phi)
//   S2 - 12 phi = E'_z + F'_{z-1} + F'_{z+1} + 4 t
//   S3 - 8 phi  = E'_{z-1} + E'_{z+1} + 4 t
// Every term is a difference of neighbouring values, which keeps FP32 drift far
// below a plain sum of neighbours.  FP32 runs on packed f32x2 pairs
// (FFMA2/FADD2/FMUL2 of sm_100+) of adjacent cells; FP64 on scalar doubles.
#pragma once

#include <cuda.h>   // CUtensorMap (the map is encoded on the host, see tma.cu)

#include "spfm_internal.h"

namespace spfm {

constexpr long long kWaitCycles = 4000000000LL;   // ~2 s at 2 GHz per bounded wait

#ifndef SPFM_STAGES
#define SPFM_STAGES 6         // planes in flight per CTA
#endif
#ifndef SPFM_MIN_CTAS
#define SPFM_MIN_CTAS 3       // resident CTAs per SM the register budget is sized for
#endif

// ------------------------------------------------------------ pack arithmetic

template <class T> struct Pk;

// The FP32 packs run on the paired FP32 instructions.  The code generator
// fuses a paired multiply whose result feeds a paired add into one paired FMA,
// explicit rounding modifier or not, and decides per inlined copy; so the step
// code never adds or subtracts a product as a separate operation: where a
// product is summed the code writes the FMA.  Every unrolled copy of the
// z-march then computes the same expression, and a cell gets the same bits
// whichever CTA, z-chunk or kernel (single grid or batch) computes it.
template <> struct Pk<float> {
    using P = float2;
    static __device__ __forceinline__ P mk(float a, float b) { return make_float2(a, b); }
    static __device__ __forceinline__ P add(P a, P b) { return __fadd2_rn(a, b); }
    static __device__ __forceinline__ P mul(P a, P b) { return __fmul2_rn(a, b); }
    static __device__ __forceinline__ P fma(P a, P b, P c) { return __ffma2_rn(a, b, c); }
    static __device__ __forceinline__ P sub(P a, P b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
    // a / b as a * rcp(b): two MUFU reciprocals (|rel. error| < 2^-22) and one
    // packed multiply, the accuracy of __fdividef without splitting the pack
    static __device__ __forceinline__ P div(P a, P b)
    {
        float2 r;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r.x) : "f"(b.x));
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r.y) : "f"(b.y));
        return __fmul2_rn(a, r);
    }
    static __device__ __forceinline__ P rsqrt(P a) { return make_float2(rsqrtf(a.x), rsqrtf(a.y)); }
};

struct D2 { double x, y; };

template <> struct Pk<double> {
    using P = D2;
    static __device__ __forceinline__ P mk(double a, double b) { return {a, b}; }
    static __device__ __forceinline__ P add(P a, P b) { return {__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y)}; }
    static __device__ __forceinline__ P mul(P a, P b) { return {__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y)}; }
    static __device__ __forceinline__ P fma(P a, P b, P c)
    {
        return {__fma_rn(a.x, b.x, c.x), __fma_rn(a.y, b.y, c.y)};
    }
    static __device__ __forceinline__ P sub(P a, P b) { return {__dsub_rn(a.x, b.x), __dsub_rn(a.y, b.y)}; }
    static __device__ __forceinline__ P div(P a, P b) { return {a.x / b.x, a.y / b.y}; }
    static __device__ __forceinline__ P rsqrt(P a) { return {::rsqrt(a.x), ::rsqrt(a.y)}; }
};

template <class T> struct PackT;
template <> struct PackT<float> { using P = float2; static P splat(float v) { return make_float2(v, v); } };
template <> struct PackT<double> { using P = D2; static P splat(double v) { return {v, v}; } };

// Step coefficients pre-splatted into packs (kernel parameter space), with dt
// folded in: phi' = phi + c1 dt S1' + c2 dt S2' + c3 dt S3'
//                 + q (s sum_k (-beta_k dt)/(1 - A_k s^2) - kmu dt)      (TI)
//                 + q (s (-kappa dt) - kmu dt)                          (CF)
template <class T>
struct PackCoef {
    using P = typename PackT<T>::P;
    P one, m2, m4, c1, c2, c3, ct, nkmu, nkap;
    P nA[kMaxTerms], nbeta[kMaxTerms];   // -A_k and -beta_k dt of the coupling groups
    int nterms;
    // the same pairs side by side (one 16- or 32-byte load each), read by the
    // run-time group count path, whose coefficients may sit in global memory
    struct __align__(2 * sizeof(P)) Pair {
        P nA, nbeta;
    };
    Pair pair[kMaxTerms];
};

template <class T>
inline PackCoef<T> make_pack_coef(const StepCoef<T> &c)
{
    using PT = PackT<T>;
    PackCoef<T> p;
    p.one = PT::splat(T(1));
    p.m2 = PT::splat(T(-2));
    p.m4 = PT::splat(T(-4));
    p.c1 = PT::splat(c.c1dt);
    p.c2 = PT::splat(c.c2dt);
    p.c3 = PT::splat(c.c3dt);
    p.ct = PT::splat(c.ctdt);
    p.nkmu = PT::splat(c.nkmudt);
    p.nkap = PT::splat(c.nkapdt);
    for (int k = 0; k < kMaxTerms; ++k) {
        p.nA[k] = PT::splat(-c.A[k]);
        p.nbeta[k] = PT::splat(c.nbetadt[k]);
        p.pair[k].nA = p.nA[k];
        p.pair[k].nbeta = p.nbeta[k];
    }
    p.nterms = c.nterms;
    return p;
}

// ------------------------------------------------------ storage <-> compute

template <class S, class T> struct Io;

template <> struct Io<float, float> {
    static constexpr int VX = 4;
    static __device__ __forceinline__ void lds(const float *p, float *v)   // 16 B of shared
    {
        const float4 r = *reinterpret_cast<const float4 *>(p);
        v[0] = r.x; v[1] = r.y; v[2] = r.z; v[3] = r.w;
    }
    static __device__ __forceinline__ void st(float *p, const float *v)
    {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
    static __device__ __forceinline__ float cvt_in(float s) { return s; }
    static __device__ __forceinline__ float cvt_out(float t) { return t; }
};

template <> struct Io<double, double> {
    static constexpr int VX = 2;
    static __device__ __forceinline__ void lds(const double *p, double *v)
    {
        const double2 r = *reinterpret_cast<const double2 *>(p);
        v[0] = r.x; v[1] = r.y;
    }
    static __device__ __forceinline__ void st(double *p, const double *v)
    {
        *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
    }
    static __device__ __forceinline__ double cvt_in(double s) { return s; }
    static __device__ __forceinline__ double cvt_out(double t) { return t; }
};

template <> struct Io<__nv_bfloat16, float> {
    static constexpr int VX = 8;
    static __device__ __forceinline__ void lds(const __nv_bfloat16 *p, float *v)
    {
        const uint4 r = *reinterpret_cast<const uint4 *>(p);
        const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            v[2 * i] = __uint_as_float(w[i] << 16);
            v[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
        }
    }
    static __device__ __forceinline__ void st(__nv_bfloat16 *p, const float *v)
    {
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
            w[i] = *reinterpret_cast<uint32_t *>(&h);
        }
        *reinterpret_cast<uint4 *>(p) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    static __device__ __forceinline__ float cvt_in(__nv_bfloat16 s) { return __bfloat162float(s); }
    static __device__ __forceinline__ __nv_bfloat16 cvt_out(float t) { return __float2bfloat16_rn(t); }
};

// --------------------------------------------------------------- mbarrier

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// One test of the phase; a thread whose phase is not complete is suspended in
// hardware for up to the hint (ns) instead of spinning on issue slots.
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(1000000u)
        : "memory");
    return ok != 0;
}

// Wait for the barrier phase with the given parity; false after ~2 s.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > kWaitCycles) return false;
    return true;
}

// Bulk asynchronous copy global -> shared, completing bytes on bar.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Producer-side wait: polls with a nanosleep back-off so a waiting producer does
// not take issue slots from the consumers; false after ~2 s.
__device__ __forceinline__ bool mbar_wait_sleep(uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    unsigned ns = 32;
    while (!mbar_try_wait(bar, parity)) {
        __nanosleep(ns);
        ns = ns < 256 ? 2 * ns : 256;
        if (clock64() - t0 > kWaitCycles) return false;
    }
    return true;
}

// TMA tile copy of a 3D box (x, y, z start in elements) into shared memory.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// -------------------------------------------------------------------- tile

#ifndef SPFM_ROWS_PER_THREAD
#define SPFM_ROWS_PER_THREAD 2
#endif

template <class S, class T, int TX, int TY, int RPT_ = SPFM_ROWS_PER_THREAD>
struct TileShape {
    static constexpr int VX = Io<S, T>::VX;
    static constexpr int NP = VX / 2;
    static constexpr int RPT = RPT_;   // rows of the tile per consumer thread
    static constexpr int W = TX * VX;
    static constexpr int SW = W + 2 * VX;   // staged row: one 16-byte chunk of halo per side
    static constexpr int ROWS = TY + 2;
    static constexpr int BOX_BYTES = ROWS * SW * (int)sizeof(S);          // one TMA box
    static constexpr int STAGE = ((BOX_BYTES + 127) / 128 * 128) / (int)sizeof(S);   // 128-B aligned
    static constexpr int NS = SPFM_STAGES;  // pipeline depth (planes)
    static constexpr int NCONS = TX * TY / RPT;   // consumer threads
    static constexpr int NTHREADS = NCONS + 32;
};

// Per plane and pack: c = phi, h = c1 dt F' + c2 dt E' (the plane as the centre
// plane of an output), g = c2 dt F' + c3 dt E' (as the plane above or below);
// with 6 neighbours h = F', with 18 g = F' (their coefficients are applied in
// the update, by FMA).
template <class T, int NP>
struct PlaneQ {
    using P = typename Pk<T>::P;
    P c[NP], h[NP], g[NP];
    P psi[NP], gx[NP], gy[NP];   // TI_n only: log-odds of phi and its in-plane differences
};

// ----------------------------------------------------------------- TI_n

// Inversion of the ideal profile, psi = (lambda/2) artanh(1 - 2 phi)
// = (lambda/4) ln((1 - phi)/phi), with phi clamped to [eps, 1 - eps] (TI_n).
// The kernels keep the log-odds only (FP32 log2, FP64 ln) and scale their
// central differences by StepCoef::psi_grad; the FP32 log-odds is the
// hardware log2 itself, no product, so differences of equal values are 0.
__device__ __forceinline__ float log_odds(float phi, float eps)
{
    const float pc = fminf(fmaxf(phi, eps), 1.0f - eps);
    return __log2f(__fdividef(1.0f - pc, pc));
}
__device__ __forceinline__ double log_odds(double phi, double eps)
{
    const double pc = fmin(fmax(phi, eps), 1.0 - eps);
    return log((1.0 - pc) / pc);
}
template <class T>
__device__ __forceinline__ typename Pk<T>::P log_odds_pack(typename Pk<T>::P v, T eps)
{
    return Pk<T>::mk(log_odds(v.x, eps), log_odds(v.y, eps));
}
// tanh of a pack.  FP32: Lambert's continued fraction for tanh truncated
// after the term x^2/11, x (10395 + 1260 y + 21 y^2) / (10395 + 4725 y + 210 y^2 + y^3)
// with y = x^2 (|error| < 3.3e-10 for |x| <= 1, < 3e-8 for |x| <= 1.5), written
// as x - x y (3465 + 189 y + y^2) / den so that the result is an FMA and sums
// of tanh values fuse nothing; callers whose arguments can exceed 1.5 pass
// small = false and get tanhf.  FP64: tanh.
template <class T> struct TanhPk;
template <> struct TanhPk<float> {
    static __device__ __forceinline__ float2 eval(float2 x, bool small)
    {
        if (!small) return make_float2(tanhf(x.x), tanhf(x.y));
        const float2 y = __fmul2_rn(x, x);
        const float2 poly = __ffma2_rn(__ffma2_rn(x, x, make_float2(189.f, 189.f)), y, make_float2(3465.f, 3465.f));
        const float2 den = __ffma2_rn(__ffma2_rn(__ffma2_rn(x, x, make_float2(210.f, 210.f)), y,
                                                 make_float2(4725.f, 4725.f)),
                                      y, make_float2(10395.f, 10395.f));
        const float2 r = Pk<float>::div(__fmul2_rn(y, poly), den);
        return __ffma2_rn(r, __ffma2_rn(x, make_float2(-1.f, -1.f), make_float2(0.f, 0.f)), x);
    }
};
template <> struct TanhPk<double> {
    static __device__ __forceinline__ D2 eval(D2 x, bool) { return {tanh(x.x), tanh(x.y)}; }
};

// ---------------------------------------------------- stochastic rounding

// Stochastic rounding of the update phi + inc to the storage type S (FP32 or
// BF16): with a the largest value of S not above the exact sum and g the
// spacing of S above a, the stored value is a + g with probability
// (phi + inc - a) / g and a otherwise, so that its expectation is the exact
// update; an exactly representable sum (inc = 0 in particular) is stored as
// is.  It is computed as round-down(phi + (inc + u g)) with u uniform in
// [0, 1) on a 2^-16 grid (16 bits of h per cell): since inc + u g spans
// exactly one spacing above a, the round-down lands on a or a + g.  The
// rounding of inc + u g in FP32 (2^-24 of g) is far below the step.
template <class S> struct MantBits;
template <> struct MantBits<float> { static constexpr int v = 23; };
template <> struct MantBits<__nv_bfloat16> { static constexpr int v = 7; };

// spacing of S above a >= 0 (from a's exponent; 0 for |a| < 2^(bits - 126))
__device__ __forceinline__ float spacing_above(float a, int bits)
{
    const int e = (int)(__float_as_uint(a) & 0x7f800000u) - (bits << 23);
    return __int_as_float(e > 0 ? e : 0);
}

// the largest BF16 value not above v (v an FP32 value)
__device__ __forceinline__ float bf16_round_down(float v)
{
    uint32_t b = __float_as_uint(v);
    if ((b & 0x80000000u) && (b & 0xffffu)) b = (b & 0xffff0000u) + 0x10000u;   // away from zero
    else b &= 0xffff0000u;
    return __uint_as_float(b);
}

template <class S>
__device__ __forceinline__ float2 sr_update(float2 ph, float2 inc, uint32_t h)
{
    constexpr int mb = MantBits<S>::v;
    float2 a = __fadd2_rd(ph, inc);
    if constexpr (mb == 7) { a.x = bf16_round_down(a.x); a.y = bf16_round_down(a.y); }
    const float2 g = make_float2(spacing_above(fabsf(a.x), mb), spacing_above(fabsf(a.y), mb));
    const float2 u = __fadd2_rn(make_float2(__uint_as_float(0x3f800000u | ((h << 7) & 0x007fff80u)),
                                            __uint_as_float(0x3f800000u | ((h >> 9) & 0x007fff80u))),
                                make_float2(-1.0f, -1.0f));
    float2 x = __fadd2_rd(ph, __ffma2_rn(u, g, inc));
    if constexpr (mb == 7) { x.x = bf16_round_down(x.x); x.y = bf16_round_down(x.y); }
    return x;
}

// TI_n factor w = -dt (potential / q + 4 M dF / (lambda Gamma)) of a pack of
// cells with s = 1 - 2 phi, u = s^2 and the profile-inversion gradient g
// (Sec. 2.1, TI_n): n = g / |g|, t_i = tanh(2 dx n_i / lambda), the 13
// couplings a = N / D from the tanh addition theorem, and the potential sum
// sum_k 4 c_k a_k^2 / (1 - a_k^2 s^2) = sum_k 4 c_k N^2 / (D^2 - N^2 s^2).
// c_k is one value per shell, so each shell's terms are summed as one running
// fraction and the three shells are joined with one reciprocal.  Where
// |g| < 1e-8 the normal is undefined and the cell takes the CF potential.
template <class T, int STENCIL>
__device__ __forceinline__ typename Pk<T>::P ti_local_w(const StepCoef<T> &C, typename Pk<T>::P sg,
                                                        typename Pk<T>::P u, typename Pk<T>::P gx,
                                                        typename Pk<T>::P gy, typename Pk<T>::P gz)
{
    using K = Pk<T>;
    using P = typename K::P;
    const P one = K::mk(T(1), T(1));
    const P zero = K::mk(T(0), T(0));
    const P neg_u = K::sub(zero, u);   // -s^2
    const P g2 = K::fma(gx, gx, K::fma(gy, gy, K::mul(gz, gz)));
    const P kin = K::mul(K::mk(C.two_dx_over_lam, C.two_dx_over_lam), K::rsqrt(g2));
    const bool small = C.two_dx_over_lam <= T(1.5);
    const P a = TanhPk<T>::eval(K::mul(gx, kin), small);
    const P b = TanhPk<T>::eval(K::mul(gy, kin), small);
    const P c = TanhPk<T>::eval(K::mul(gz, kin), small);
    // (num, den) += n / d as one fraction
    auto acc = [&](P &num, P &den, P n, P d) {
        num = K::fma(num, d, K::mul(n, den));
        den = K::mul(den, d);
    };
    // shell 1: N = t_i, D = 1
    const P a2 = K::mul(a, a), b2 = K::mul(b, b), c2 = K::mul(c, c);
    P n1 = a2, d1 = K::fma(a2, neg_u, one);
    acc(n1, d1, b2, K::fma(b2, neg_u, one));
    acc(n1, d1, c2, K::fma(c2, neg_u, one));
    P num = K::mul(K::mk(T(-4) * C.dt * C.ck[0], T(-4) * C.dt * C.ck[0]), n1), den = d1;
    // Shells 2 and 3 come in pairs of directions whose couplings are
    // N = x +- y, D = y' +- x' for one (x, y, x', y').  With S = x^2 + y^2,
    // B = x'^2 + y'^2 (S and B are the squares summed over the pair), R = 2 x y
    // (= 2 x' y'), P = B - S u and v = 1 - u, the pair's two terms
    // n/d = (S +- R) / (P +- R v) add up to 2 (S P - R^2 v) / (P^2 - R^2 v^2).
    const P v = K::fma(K::sub(zero, sg), sg, one);   // 1 - s^2
    const P m4 = K::mk(T(-4), T(-4));
    auto pair = [&](P &pn, P &pd, P S, P B, P r) {   // r = x^2 y^2 = R^2 / 4
        const P Pv = K::fma(S, neg_u, B);
        const P rv = K::mul(r, v);
        acc(pn, pd, K::fma(rv, m4, K::mul(S, Pv)), K::fma(K::mul(rv, v), m4, K::mul(Pv, Pv)));
    };
    if (STENCIL >= 18 && C.ck[3] != T(0)) {
        // shell 2: (1,+-1,0), (0,1,+-1), (1,0,+-1): x, y = t_i, t_j and x', y' = t_i t_j, 1
        P n2 = zero, d2 = one;
        const P ab = K::mul(a2, b2), bc = K::mul(b2, c2), ac = K::mul(a2, c2);
        pair(n2, d2, K::fma(a, a, b2), K::fma(a2, b2, one), ab);
        pair(n2, d2, K::fma(b, b, c2), K::fma(b2, c2, one), bc);
        pair(n2, d2, K::fma(a, a, c2), K::fma(a2, c2, one), ac);
        acc(num, den, K::mul(K::mk(T(-8) * C.dt * C.ck[3], T(-8) * C.dt * C.ck[3]), n2), d2);
    }
    if (STENCIL >= 26 && C.ck[9] != T(0)) {
        // shell 3: tanh(x + y + z) = (tx + ty + tz + tx ty tz) / (1 + tx ty + ty tz + tx tz).
        // (1,1,+-1): N = al +- tz be, D = be +- tz al with al = tx + ty, be = 1 + tx ty;
        // (-1,1,1), (1,-1,1): the same with al = ty - tx, be = 1 - tx ty.
        P n3 = zero, d3 = one;
        const P al1 = K::add(a, b), be1 = K::fma(a, b, one);
        const P al2 = K::sub(b, a), be2 = K::fma(K::sub(zero, a), b, one);
        const P A1 = K::mul(al1, al1), B1 = K::mul(be1, be1);
        const P A2 = K::mul(al2, al2), B2 = K::mul(be2, be2);
        pair(n3, d3, K::fma(c2, B1, A1), K::fma(c2, A1, B1), K::mul(K::mul(A1, B1), c2));
        pair(n3, d3, K::fma(c2, B2, A2), K::fma(c2, A2, B2), K::mul(K::mul(A2, B2), c2));
        acc(num, den, K::mul(K::mk(T(-8) * C.dt * C.ck[9], T(-8) * C.dt * C.ck[9]), n3), d3);
    }
    const P nkmu = K::mk(-C.dt * C.kmu, -C.dt * C.kmu);
    const P w = K::fma(sg, K::div(num, den), nkmu);
    const P wcf = K::fma(sg, K::mk(-C.dt * C.kappa, -C.dt * C.kappa), nkmu);
    const T lim = T(1e-16);
    return K::mk(g2.x >= lim ? w.x : wcf.x, g2.y >= lim ? w.y : wcf.y);
}

// The packs of one staged row around a thread's cells (adjacent pairs):
// c[p] = (x+2p, x+2p+1), w[p] = c shifted by -1, e[p] = shifted by +1.
template <class S, class T, int VX>
__device__ __forceinline__ void get_row(const S *r, typename Pk<T>::P *c, typename Pk<T>::P *w,
                                        typename Pk<T>::P *e)
{
    using K = Pk<T>;
    T v[VX + 2];
    Io<S, T>::lds(r, v + 1);
    v[0] = Io<S, T>::cvt_in(r[-1]);
    v[VX + 1] = Io<S, T>::cvt_in(r[VX]);
#pragma unroll
    for (int p = 0; p < VX / 2; ++p) {
        c[p] = K::mk(v[2 * p + 1], v[2 * p + 2]);
        w[p] = K::mk(v[2 * p], v[2 * p + 1]);
        e[p] = K::mk(v[2 * p + 2], v[2 * p + 3]);
    }
}

// Periodic images across the z faces of the 16 bytes of new cells at
// (x.., y, z) of an all-periodic grid: z + nz on plane 0, z - nz on plane
// nz - 1, each also shifted by the cells' x and y images (edges, corners).
template <class S>
__device__ __forceinline__ void store_z_images(const GridGeom &g, S *dst, int x, int y, int z, uint4 v,
                                               int ximg, int yimg)
{
    const bool zu[2] = {z == 0, z == g.nz - 1};
    const int zs[2] = {g.nz, -g.nz};
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        if (!zu[c]) continue;
        S *p = dst + cell_index(g, x, y, z + zs[c]);
        *reinterpret_cast<uint4 *>(p) = v;
        if (ximg) *reinterpret_cast<uint4 *>(p + ximg) = v;
        if (yimg) *reinterpret_cast<uint4 *>(p + yimg) = v;
        if (ximg && yimg) *reinterpret_cast<uint4 *>(p + yimg + ximg) = v;
    }
}

// ------------------------------------------------ ghosts of non-periodic faces

// Ghost value of a non-periodic face from its source cell v: the
// contact-angle value of Eq. 7 with the face's signed coupling a,
// (1 - a) v / (1 - a (2 v - 1)) = k1 v / (k2 - k3 v), or a copy (no-flux).
// FP32 takes the approximate reciprocal (the face kernel divides exactly, so
// the two differ in the last unit; the ghosts are not kept in memory here).
template <class T> struct FaceMap {
    T k1, k2, k3;
    bool copy;
};
template <class T>
__device__ __forceinline__ FaceMap<T> face_map(int bc, T a)
{
    return FaceMap<T>{T(1) - a, T(1) + a, T(2) * a, bc != SPFM_CONTACT};
}
__device__ __forceinline__ float face_value(float v, const FaceMap<float> &m)
{
    if (m.copy) return v;
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(__fmaf_rn(-m.k3, v, m.k2)));
    return m.k1 * v * r;
}
__device__ __forceinline__ double face_value(double v, const FaceMap<double> &m)
{
    return m.copy ? v : m.k1 * v / (m.k2 - m.k3 * v);
}

// The staged plane st (ROWS x SW, the tile plus halo) of a grid whose faces
// are all non-periodic gets the ghost values of the faces it touches, from the
// interior cells next to them, in the face kernel's order: the x ghost columns
// of every row, then the y ghost rows (x ghosts included).  Run by the 32
// lanes of the producer warp; no face kernel then runs between steps.
template <class S, class T, int VX, int SW, int ROWS>
__device__ __forceinline__ void fix_xy(S *st, const GridGeom &g, const T *aface, int x0, int y0, int W, int TY,
                                       int lane)
{
    const bool xlo = x0 == 0;
    const int xhi = (g.nx - 1 >= x0 && g.nx - 1 < x0 + W) ? g.nx - x0 + VX : -1;   // column of x = nx
    const bool ylo = y0 == 0;
    const int yhi = (g.ny - 1 >= y0 && g.ny - 1 < y0 + TY) ? g.ny - y0 + 1 : -1;    // row of y = ny
    if (xlo || xhi >= 0) {
        const FaceMap<T> ml = face_map<T>(g.bc[0], aface[0]), mh = face_map<T>(g.bc[1], aface[1]);
        for (int k = lane; k < ROWS; k += 32) {
            S *row = st + k * SW;
            if (xlo) row[VX - 1] = Io<S, T>::cvt_out(face_value(Io<S, T>::cvt_in(row[VX]), ml));
            if (xhi >= 0) row[xhi] = Io<S, T>::cvt_out(face_value(Io<S, T>::cvt_in(row[xhi - 1]), mh));
        }
        __syncwarp();
    }
    if (ylo) {
        const FaceMap<T> m = face_map<T>(g.bc[2], aface[2]);
        for (int c = lane; c < SW; c += 32) st[c] = Io<S, T>::cvt_out(face_value(Io<S, T>::cvt_in(st[SW + c]), m));
    }
    if (yhi >= 0) {
        const FaceMap<T> m = face_map<T>(g.bc[3], aface[3]);
        for (int c = lane; c < SW; c += 32)
            st[yhi * SW + c] = Io<S, T>::cvt_out(face_value(Io<S, T>::cvt_in(st[(yhi - 1) * SW + c]), m));
    }
}

// A z ghost plane (plane -1 or nz) staged from its adjacent interior plane
// (already carrying its x and y ghosts): every value shifted by the z face.
template <class S, class T, int SW, int ROWS>
__device__ __forceinline__ void fix_z(S *dst, const S *src, const GridGeom &g, const T *aface, int face, int lane)
{
    const FaceMap<T> m = face_map<T>(g.bc[face], aface[face]);
    for (int i = lane; i < ROWS * SW; i += 32) dst[i] = Io<S, T>::cvt_out(face_value(Io<S, T>::cvt_in(src[i]), m));
}

// phi + dt (Laplacian part of Eq. 1) of a pack from its plane records: t the
// z-neighbour differences, h of the centre plane, g of the planes below and
// above (6 neighbours: h = F'; 18: g = F'; 26: h, g with their coefficients).
// SR: the increment alone (phi is added in sr_update).  Products are summed by
// FMAs only.
template <bool SR, int STENCIL, class P, class PCoef>
__device__ __forceinline__ P laplace_update(const PCoef &PC, P t, P ph, P h, P gm, P gp)
{
    using K = Pk<decltype(P().x)>;
    P acc;
    if constexpr (STENCIL == 6) acc = K::fma(PC.c1, h, SR ? K::mul(PC.ct, t) : K::fma(PC.ct, t, ph));
    else acc = SR ? K::fma(PC.ct, t, h) : K::add(K::fma(PC.ct, t, ph), h);
    if constexpr (STENCIL == 18) acc = K::fma(PC.c2, K::add(gm, gp), acc);
    if constexpr (STENCIL == 26) acc = K::add(acc, K::add(gm, gp));
    return acc;
}

// KIND: 0 = CF potential; 1..4 = TI global with exactly KIND coupling groups;
// 5 = TI global with up to 13 groups (count read at run time)
// One tile (bx, by) of planes zc0..zc1-1.  The stage ring continues across the
// tiles a CTA processes: plane i of this tile is ring slot base + i.  The
// producer waits for its copies in flight before returning when drain is set.
// Returns false when a bounded wait gave up (the error word is set).
// SR: stochastic rounding of the update (FP32 compute only), random bits from
// sr_hash(padded cell index xor sr_key).
// ROLL (KIND 5): the group loop stays a loop, for coefficients in the kernel's
// parameters (single grids); from a batch's grid records in global memory the
// unrolled loop overlaps the pairs' loads.  Same operations, same bits.
template <class S, class T, int STENCIL, int KIND, int TX, int TY, int RPT_, bool IMG = false, bool SR = false,
          bool ROLL = false>
__device__ __forceinline__ bool step_tile(const StepCoef<T> &C, const PackCoef<T> &PC,
                                          const S *__restrict__ src, S *__restrict__ dst,
                                          int *__restrict__ err, const CUtensorMap *tmap, int bx,
                                          int by, int zc0, int zc1, S *__restrict__ stages,
                                          uint64_t *full, uint64_t *empty, int base, bool drain,
                                          int mode = 0, uint32_t sr_key = 0, uint64_t *ready = nullptr,
                                          bool fwd = false)
{
    static_assert(!SR || sizeof(T) == 4, "stochastic rounding is for FP32 compute");
    using Sh = TileShape<S, T, TX, TY, RPT_>;
    using K = Pk<T>;
    using P = typename K::P;
    constexpr int VX = Sh::VX, NP = Sh::NP, W = Sh::W, SW = Sh::SW, ROWS = Sh::ROWS;
    constexpr int STAGE = Sh::STAGE, NS = Sh::NS;
    constexpr int NTMAX = KIND >= 1 && KIND <= 4 ? KIND : kMaxTerms;
    static_assert(KIND != 6 || RPT_ == 1, "TI_n runs one row per thread");

    const GridGeom &g = C.g;
    const int tid = threadIdx.x;
    const int x0 = bx * W, y0 = by * TY;
    const int nplanes = zc1 - zc0 + 2;   // planes zc0-1 .. zc1

    if (tid >= Sh::NCONS) {
        // ------------------------------------------------------- producer warp
        // fwd (every face non-periodic): the whole warp builds the ghosts of the
        // faces a staged plane touches (fix_xy, fix_z) and then releases it to
        // the consumers on its "ready" barrier, NS - 2 planes behind the copies,
        // so that as many copies stay in flight; otherwise one lane issues the
        // copies and the consumers wait on "full".
        const int plane_lane = tid - Sh::NCONS;
        if (!fwd && plane_lane != 0) return true;
        const bool lead = plane_lane == 0;
        // The kernel may start while the previous launch still runs (programmatic
        // dependent launch).  After a ghost-face refresh of src, a box that holds
        // no ghost cell reads only interior cells, which the step before that
        // wrote, so only boxes touching a face wait for the previous grid; after
        // anything else (a step that wrote its own images, the first step of a
        // call) every box waits.
        if (lead && ((mode & kWaitAll) ||
                     ((mode & kWaitFaces) &&
                      (bx == 0 || x0 + W >= g.nx || by == 0 || y0 + TY >= g.ny || zc0 == 0 || zc1 == g.nz))))
            asm volatile("griddepcontrol.wait;" ::: "memory");
        // kSkipCopy (a test of the bounded waits): the first CTA never fills the
        // stage of its plane 1, so its consumers' wait for that stage gives up
        const bool skip = (mode & kSkipCopy) && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0;
        const bool zlo = fwd && zc0 == 0, zhi = fwd && zc1 == g.nz;
        auto stage = [&](int j) { return stages + ((base + j) % NS) * STAGE; };
        // waits on the forwarding path suspend in hardware until the phase
        // completes (no sleep back-off: the consumers wait behind them)
        auto wait_full = [&](int j) {
            return __all_sync(0xffffffffu, mbar_wait(&full[(base + j) % NS], ((base + j) / NS) & 1));
        };
        auto release = [&](int j) {
            __syncwarp();
            if (lead) mbar_arrive(&ready[(base + j) % NS]);
        };
        // plane j to the consumers: its x/y ghosts, or (a z ghost plane) all of it
        // from the adjacent interior plane; plane 0 of a z- face follows plane 1
        auto forward = [&](int j) -> bool {
            if (zlo && j == 0) return true;
            if (!wait_full(j)) return false;
            if (zhi && j == nplanes - 1) fix_z<S, T, SW, ROWS>(stage(j), stage(j - 1), g, C.aface, 5, plane_lane);
            else fix_xy<S, T, VX, SW, ROWS>(stage(j), g, C.aface, x0, y0, W, TY, plane_lane);
            release(j);
            if (zlo && j == 1) {
                if (!wait_full(0)) return false;
                fix_z<S, T, SW, ROWS>(stage(0), stage(1), g, C.aface, 4, plane_lane);
                release(0);
            }
            return true;
        };
        // lag NS - 2: plane 0 of a z- face, forwarded with plane 1, is released
        // before the copy of plane NS has to wait for its stage
        const int lag = fwd ? NS - 2 : 0;
        int issued = 0;
        bool ok = true;
        for (int i = 0; i < nplanes + lag; ++i) {
            if (i < nplanes) {
                if (lead) {
                    const int I = base + i, s = I % NS;
                    if (I >= NS && !(fwd ? mbar_wait(&empty[s], ((I / NS) - 1) & 1)
                                         : mbar_wait_sleep(&empty[s], ((I / NS) - 1) & 1))) {
                        ok = false;
                    } else if (!(skip && i == 1)) {
                        if (tmap) {
                            mbar_expect_tx(&full[s], (uint32_t)Sh::BOX_BYTES);
                            // one box: padded x from the 16-byte chunk left of the tile (x0 + off
                            // - VX, 16-byte aligned), padded rows y0.., padded plane zc0 + i;
                            // out-of-range parts are zero-filled, never used
                            tma_load_3d(stages + s * STAGE, tmap, x0 + g.off - VX, y0, zc0 + i, &full[s]);
                        } else {
                            // row by row (no tensor map): the box's rows that lie in the buffer
                            const long long row0 = (long long)(x0 + g.off - VX);
                            const int bytes_row = (int)min((long long)SW, (long long)g.pitch - row0) * (int)sizeof(S);
                            const int nrows = min(ROWS, g.ny + 2 - y0);
                            mbar_expect_tx(&full[s], (uint32_t)(bytes_row * nrows));
                            const S *plane = src + (long long)(zc0 + i) * g.plane + (long long)y0 * g.pitch + row0;
                            S *st = stages + s * STAGE;
                            for (int r = 0; r < nrows; ++r)
                                bulk_g2s(st + r * SW, plane + (long long)r * g.pitch, (uint32_t)bytes_row, &full[s]);
                        }
                    }
                    if (ok) ++issued;
                }
                if (fwd) ok = __shfl_sync(0xffffffffu, ok, 0) != 0;
                if (!ok) break;
            }
            if (fwd && i >= lag && !forward(i - lag)) {
                ok = false;
                break;
            }
        }
        if (fwd) issued = __shfl_sync(0xffffffffu, issued, 0);
        if (!lead) return ok;
        if (!ok) atomicOr(err, 1);
        // never leave with copies in flight: wait for each stage's copy (a stage
        // whose wait gives up does not stop the waits for the others)
        if (drain || !ok)
            for (int I = max(0, base + issued - NS); I < base + issued; ++I)
                if (!mbar_wait_sleep(&full[I % NS], (I / NS) & 1)) atomicOr(err, 2);
        return ok;
    }

    // ------------------------------------------------------------- consumers
    constexpr int RPT = Sh::RPT;
    const int tx = tid % TX, ty = (tid / TX) * RPT;   // first of the thread's RPT rows
    const int lane = tid & 31;
    const int gx = x0 + tx * VX;
    const int gy = y0 + ty;
    const S *rbase = stages + (ty + 1) * SW + VX + tx * VX;   // first own row in a stage
    S *obase = dst + cell_index(g, gx, gy, 0);                // plane 0, first own row
    // Periodic images (IMG: all faces periodic, nx a multiple of 2 VX, nx >= 4 VX,
    // ny >= 2): a cell in the first two 16-byte chunks of a row also goes to the
    // sector right of the row (x + nx), one in the last two chunks to the sector
    // left of it (x - nx); the two threads of a sector store it in one request.
    // Rows 0 and ny - 1 also go to the ghost rows across (y -+ ny), with the x
    // image.  The offsets (elements, 0 where a cell has no image) are recomputed
    // where they are used, so that the plane loop keeps only the flag live.
    auto ximg = [&]() { return gx < 2 * VX ? g.nx : (gx >= g.nx - 2 * VX ? -g.nx : 0); };
    auto yimg = [&](int r) {
        return gy + r == 0 ? g.ny * g.pitch : (gy + r == g.ny - 1 ? -g.ny * g.pitch : 0);
    };
    bool img = false;
    if constexpr (IMG) img = gx < 2 * VX || gx >= g.nx - 2 * VX || gy == 0 || gy + RPT >= g.ny;

    bool ok = true;
    auto body = [&](int i, PlaneQ<T, NP> (&m)[RPT], PlaneQ<T, NP> (&z)[RPT],
                    PlaneQ<T, NP> (&p)[RPT]) -> bool {
        const int I = base + i, s = I % NS;
        // warp-uniform: every lane waits (acquire), the warp goes on only if all saw it
        if (!__all_sync(0xffffffffu, mbar_wait(fwd ? &ready[s] : &full[s], (I / NS) & 1))) {
            if (lane == 0) atomicOr(err, 4);
            ok = false;
            return false;
        }
        {
            // rows ty-1 .. ty+RPT of the stage (north halo, own rows, south halo)
            const S *r0 = rbase + s * STAGE - SW;
            P rc[RPT + 2][NP], rw[RPT + 2][NP], re[RPT + 2][NP];
#pragma unroll
            for (int r = 0; r < RPT + 2; ++r) get_row<S, T, VX>(r0 + r * SW, rc[r], rw[r], re[r]);
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
#pragma unroll
            for (int r = 0; r < RPT; ++r) {
#pragma unroll
                for (int q = 0; q < NP; ++q) {
                    const P c = rc[r + 1][q];
                    p[r].c[q] = c;
                    // F' = (W + E + N + S) - 4C, E' = (NW + NE + SW + SE) - 4C
                    const P f = K::fma(PC.m4, c, K::add(K::add(rw[r + 1][q], re[r + 1][q]),
                                                        K::add(rc[r][q], rc[r + 2][q])));
                    // 6 neighbours: h = F' (c1 applied in the update's FMA); 18: g = F'
                    // (c2 applied to the sum of the two planes' g in one FMA)
                    if (STENCIL == 6) {
                        p[r].h[q] = f;
                    } else {
                        const P e = K::fma(PC.m4, c, K::add(K::add(rw[r][q], re[r][q]),
                                                            K::add(rw[r + 2][q], re[r + 2][q])));
                        p[r].h[q] = K::fma(PC.c2, e, K::mul(PC.c1, f));
                        p[r].g[q] = STENCIL == 26 ? K::fma(PC.c3, e, K::mul(PC.c2, f)) : f;
                    }
                }
                if (KIND == 6) {
                    // log-odds at the cells and central differences along x and y.  A
                    // warp holds 32/TX rows: each lane inverts its own cells and
                    // its row's two x-neighbour cells; the rows above and below
                    // come by shuffle from the lanes TX away, except beyond the
                    // warp's first and last rows, where the lane inverts them.
                    static_assert(KIND != 6 || (TX <= 16 && 32 % TX == 0), "TI_n needs two or more rows a warp");
                    const T ep = C.eps;
                    const bool first = lane < TX, last = lane >= 32 - TX;
                    T own[VX], outer[VX];
#pragma unroll
                    for (int q = 0; q < NP; ++q) {
                        const P po = log_odds_pack<T>(rc[r + 1][q], ep);
                        const P pb = log_odds_pack<T>(first ? rc[r][q] : rc[r + 2][q], ep);
                        p[r].psi[q] = po;
                        own[2 * q] = po.x;
                        own[2 * q + 1] = po.y;
                        outer[2 * q] = pb.x;
                        outer[2 * q + 1] = pb.y;
                    }
                    // the two x-neighbour cells of the thread's run
                    const P pwe = log_odds_pack<T>(K::mk(rw[r + 1][0].x, re[r + 1][NP - 1].y), ep);
                    const T pw = pwe.x;   // x - 1
                    const T pe = pwe.y;   // x + VX
#pragma unroll
                    for (int q = 0; q < NP; ++q) {
                        const T w0 = 2 * q == 0 ? pw : own[2 * q - 1];
                        const T e1 = 2 * q + 2 == VX ? pe : own[2 * q + 2];
                        // the log-odds are no products, so equal values differ by exactly
                        // zero and a clamped region keeps the CF fallback (a difference
                        // fused with a multiply would leave that product's rounding
                        // error, enough to pass |g| >= 1e-8 in FP32 with a meaningless normal)
                        p[r].gx[q] = K::sub(K::mk(own[2 * q + 1], e1), K::mk(w0, own[2 * q]));
                        T nb[2], sb[2];
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const T up = __shfl_up_sync(0xffffffffu, own[2 * q + h], TX);
                            const T dn = __shfl_down_sync(0xffffffffu, own[2 * q + h], TX);
                            nb[h] = first ? outer[2 * q + h] : up;   // row j - 1
                            sb[h] = last ? outer[2 * q + h] : dn;    // row j + 1
                        }
                        p[r].gy[q] = K::sub(K::mk(sb[0], sb[1]), K::mk(nb[0], nb[1]));   // psi(j + 1) - psi(j - 1)
                    }
                }
            }
        }
        if (i >= 2) {
            const int oz = zc0 - 2 + i;   // output plane
#pragma unroll
            for (int r = 0; r < RPT; ++r) {
                if (gy + r >= g.ny || gx >= g.nx) continue;
                T outv[VX];
                // padded index of the row's first cell (32-bit, wraps): the cell's
                // part of the stochastic-rounding hash
                const uint32_t sr_row = SR ? (uint32_t)cell_index(g, gx, gy + r, oz) : 0u;
                if constexpr (KIND == 5) {
                    // up to 13 groups counted at run time (in a batch the coefficients
                    // sit in global memory): the running fraction over every pack of
                    // the row per group, so that each (A, beta) pair is read once a row
                    P acc[NP], sg[NP], q1[NP], u[NP], num[NP], den[NP];
                    const typename PackCoef<T>::Pair t0 = PC.pair[0];
#pragma unroll
                    for (int q = 0; q < NP; ++q) {
                        const P ph = z[r].c[q];
                        const P t = K::add(K::sub(m[r].c[q], ph), K::sub(p[r].c[q], ph));
                        // SR: the increment alone, phi is added once in sr_update
                        acc[q] = laplace_update<SR, STENCIL>(PC, t, ph, z[r].h[q], m[r].g[q], p[r].g[q]);
                        sg[q] = K::fma(PC.m2, ph, PC.one);
                        q1[q] = K::mul(ph, K::sub(PC.one, ph));
                        u[q] = K::mul(sg[q], sg[q]);
                        num[q] = t0.nbeta;
                        den[q] = K::fma(t0.nA, u[q], PC.one);
                    }
                    auto group = [&](const typename PackCoef<T>::Pair tk) {
#pragma unroll
                        for (int q = 0; q < NP; ++q) {
                            const P d = K::fma(tk.nA, u[q], PC.one);
                            num[q] = K::fma(num[q], d, K::mul(tk.nbeta, den[q]));
                            den[q] = K::mul(den[q], d);
                        }
                    };
                    if constexpr (ROLL) {
#pragma unroll 1
                        for (int kk = 1; kk < PC.nterms; ++kk) group(PC.pair[kk]);
                    } else {
#pragma unroll
                        for (int kk = 1; kk < NTMAX; ++kk)
                            if (kk < PC.nterms) group(PC.pair[kk]);
                    }
#pragma unroll
                    for (int q = 0; q < NP; ++q) {
                        P o = K::fma(q1[q], K::fma(sg[q], K::div(num[q], den[q]), PC.nkmu), acc[q]);
                        if constexpr (SR) o = sr_update<S>(z[r].c[q], o, sr_hash((sr_row + 2 * q) ^ sr_key));
                        outv[2 * q] = o.x;
                        outv[2 * q + 1] = o.y;
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < NP; ++q) {
                        const P ph = z[r].c[q];
                        const P t = K::add(K::sub(m[r].c[q], ph), K::sub(p[r].c[q], ph));
                        // phi + dt * Laplacian (SR: the increment alone, phi is added in sr_update)
                        const P acc = laplace_update<SR, STENCIL>(PC, t, ph, z[r].h[q], m[r].g[q], p[r].g[q]);
                        const P sg = K::fma(PC.m2, ph, PC.one);               // s = 1 - 2 phi
                        const P q1 = K::mul(ph, K::sub(PC.one, ph));          // q = phi (1 - phi)
                        P w;   // -dt (potential / q + 4 M dF / (lambda Gamma))
                        if (KIND == 0) {
                            // driving term -dt pref dF h'(phi) = q (nkmu f): f = 1 for h3,
                            // 5 q for h5, 1/(3 (1 - 2q)^2) for h_Abel
                            P drive = PC.nkmu;
                            if (C.interp == 1) {
                                drive = K::mul(PC.nkmu, K::mul(K::mk(T(5), T(5)), q1));
                            } else if (C.interp == 2) {
                                const P d = K::fma(K::mk(T(-2), T(-2)), q1, PC.one);
                                drive = K::div(PC.nkmu, K::mul(K::mk(T(3), T(3)), K::mul(d, d)));
                            }
                            w = K::fma(sg, PC.nkap, drive);
                        } else if (KIND == 6) {
                            const P s2 = K::mk(C.psi_grad, C.psi_grad);
                            const P gz = K::mul(K::sub(p[r].psi[q], m[r].psi[q]), s2);
                            w = ti_local_w<T, STENCIL>(C, sg, K::mul(sg, sg), K::mul(z[r].gx[q], s2),
                                                       K::mul(z[r].gy[q], s2), gz);
                        } else {
                            // exactly KIND groups, coefficients from the parameter bank
                            const P u = K::mul(sg, sg);
                            P num = PC.nbeta[0];
                            P den = K::fma(PC.nA[0], u, PC.one);
#pragma unroll
                            for (int kk = 1; kk < NTMAX; ++kk) {
                                const P d = K::fma(PC.nA[kk], u, PC.one);
                                num = K::fma(num, d, K::mul(PC.nbeta[kk], den));
                                den = K::mul(den, d);
                            }
                            w = K::fma(sg, K::div(num, den), PC.nkmu);
                        }
                        P o = K::fma(q1, w, acc);
                        if constexpr (SR) o = sr_update<S>(ph, o, sr_hash((sr_row + 2 * q) ^ sr_key));
                        outv[2 * q] = o.x;
                        outv[2 * q + 1] = o.y;
                    }
                }
                S *optr = obase + (long long)oz * g.plane + (long long)r * g.pitch;
                if (gx + VX <= g.nx) {
                    Io<S, T>::st(optr, outv);
                    if (IMG && img) {
                        const int xo = ximg(), yo = yimg(r);
                        if (xo) Io<S, T>::st(optr + xo, outv);
                        if (yo) {
                            Io<S, T>::st(optr + yo, outv);
                            if (xo) Io<S, T>::st(optr + yo + xo, outv);
                        }
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < VX; ++e)
                        if (gx + e < g.nx) optr[e] = Io<S, T>::cvt_out(outv[e]);
                }
            }
        }
        return i + 1 < nplanes;
    };

    PlaneQ<T, NP> q0[RPT], q1[RPT], q2[RPT];
    for (int i = 0;; i += 3) {
        if (!body(i, q1, q2, q0)) break;
        if (!body(i + 1, q2, q0, q1)) break;
        if (!body(i + 2, q0, q1, q2)) break;
    }
    // Images across the z faces, after the march so that the plane loop stays
    // free of them: the threads of a tile holding plane 0 or nz - 1 read back
    // their own stores of that plane (program order) and copy them.
    if (IMG && ok && gx < g.nx && (zc0 == 0 || zc1 == g.nz)) {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int oz = e == 0 ? 0 : g.nz - 1;
            if (oz < zc0 || oz >= zc1 || (e == 1 && oz == 0)) continue;
#pragma unroll
            for (int r = 0; r < RPT; ++r) {
                if (gy + r >= g.ny) continue;
                const uint4 v = *reinterpret_cast<const uint4 *>(dst + cell_index(g, gx, gy + r, oz));
                store_z_images<S>(g, dst, gx, gy + r, oz, v, ximg(), yimg(r));
            }
        }
    }
    return ok;
}

// Resident CTAs per SM the register budget is sized for: three by default;
// the single-grid FP32 kernels fit four (96 registers, no spills, 20 warps per
// SM: 2 % faster for TI_<120>, 3-6 % for CF at 512^3), while FP64 and BF16
// spill there, and the persistent batch kernel keeps three.
template <class S> struct MinBlocks { static constexpr int value = SPFM_MIN_CTAS; };
template <> struct MinBlocks<float> { static constexpr int value = 4; };
template <class S> struct BatchMinBlocks { static constexpr int value = SPFM_MIN_CTAS; };

// (the stochastic-rounding kernels and the 13-group potential keep three CTAs
// per SM: at four their registers spill, and the 13-group kernel ran 15-18 %
// slower at 192^3)
template <class S, class T, int STENCIL, int KIND, int TX, int TY, int RPT_, bool IMG, bool SR = false>
__global__ void __launch_bounds__(TileShape<S, T, TX, TY, RPT_>::NTHREADS,
                                  RPT_ == 1 ? 2 : ((SR || KIND == 5) ? SPFM_MIN_CTAS : MinBlocks<S>::value))
    spfm_step_kernel(const StepCoef<T> C, const PackCoef<T> PC, const S *__restrict__ src,
                     S *__restrict__ dst, int *__restrict__ err, int zchunk,
                     const __grid_constant__ CUtensorMap tmap, int use_tmap, int mode)
{
    using Sh = TileShape<S, T, TX, TY, RPT_>;
    // a step that writes its own ghost images, or whose grid has no periodic face
    // (no face kernel follows), lets the next step launch at once: every box of
    // that step waits for this grid (kWaitAll) before it reads
    if (IMG || (mode & kEarly)) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    __shared__ __align__(128) S stages[Sh::NS * Sh::STAGE];
    __shared__ __align__(8) uint64_t full[Sh::NS], empty[Sh::NS], ready[Sh::NS];
    if (threadIdx.x == 0) {
        for (int s = 0; s < Sh::NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], Sh::NCONS / 32);
            mbar_init(&ready[s], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int zc0 = blockIdx.z * zchunk;
    const int zc1 = min(zc0 + zchunk, C.g.nz);
    // no periodic face: the producer warp stages the ghosts of the faces
    bool fwd = false;
    if constexpr (!IMG) {
        fwd = true;
#pragma unroll
        for (int f = 0; f < 6; ++f) fwd = fwd && C.g.bc[f] != SPFM_PERIODIC;
    }
    step_tile<S, T, STENCIL, KIND, TX, TY, RPT_, IMG, SR, true>(C, PC, src, dst, err, use_tmap ? &tmap : nullptr,
                                                     blockIdx.x, blockIdx.y, zc0, zc1, stages, full, empty, 0,
                                                     true, mode, C.sr_key, ready, fwd);
}

// ------------------------------------------------------------------- batches

// One grid of a batch as the persistent kernel reads it from device memory.
template <class T>
struct BatchGrid {
    CUtensorMap map[2];     // TMA maps of the two buffers (when has_map)
    StepCoef<T> C;
    PackCoef<T> PC;
    void *field[2];
    int cur;                // buffer holding the field at parity 0
    int has_map;
    CUtensorMap map_sq[2];  // the same for the box of the square tile shape (when has_map_sq)
    int has_map_sq;
};

// Persistent kernel over a packed work-list of items of one tile shape (TX,
// TY): CTA b takes items b, b + gridDim.x, ...  Step `parity` reads buffer
// cur ^ parity.  SQ: the items use the square tile's TMA maps (map_sq).
// SR: stochastic rounding, the step key of grid i from sr_step_key(its seed,
// steps[i] + sub).  fwd: no grid of the batch has a periodic face (the
// producer warp stages the ghosts of the faces; no ghost kernel runs).
template <class S, class T, int STENCIL, int KIND, int TX, int TY, bool SQ, bool SR = false>
__global__ void __launch_bounds__(TileShape<S, T, TX, TY>::NTHREADS, BatchMinBlocks<S>::value)
    spfm_batch_kernel(const BatchGrid<T> *__restrict__ grids, const BatchItem *__restrict__ work,
                      int nwork, int parity, int *__restrict__ err, const long long *__restrict__ steps,
                      int sub, int fwd)
{
    using Sh = TileShape<S, T, TX, TY>;
    __shared__ __align__(128) S stages[Sh::NS * Sh::STAGE];
    __shared__ __align__(8) uint64_t full[Sh::NS], empty[Sh::NS], ready[Sh::NS];
    if (threadIdx.x == 0) {
        for (int s = 0; s < Sh::NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], Sh::NCONS / 32);
            mbar_init(&ready[s], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    int base = 0;
    for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
        const BatchItem it = work[w];
        const BatchGrid<T> &bg = grids[it.grid];
        const int cur = bg.cur ^ parity;
        const CUtensorMap *map = SQ ? (bg.has_map_sq ? &bg.map_sq[cur] : nullptr) : (bg.has_map ? &bg.map[cur] : nullptr);
        if (map && threadIdx.x == Sh::NCONS)
            asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(map) : "memory");
        const bool last = w + (int)gridDim.x >= nwork;
        const uint32_t key = SR ? sr_step_key(bg.C.sr_seed, steps[it.grid] + sub) : 0u;
        if (!step_tile<S, T, STENCIL, KIND, TX, TY, SPFM_ROWS_PER_THREAD, false, SR>(
                bg.C, bg.PC, (const S *)bg.field[cur], (S *)bg.field[cur ^ 1], err, map, it.bx, it.by, it.zc0,
                it.zc1, stages, full, empty, base, last, 0, key, ready, fwd != 0))
            return;
        base += it.zc1 - it.zc0 + 2;
    }
}

// Work-list entries of one grid for the tile shape (TX, TY) of the (S, T)
// kernel, marked with the item shape index `shape`.
template <class S, class T, int TX, int TY>
inline int batch_items_t(const GridGeom &g, int grid_index, int zchunk, BatchItem *out, int shape = 0)
{
    using Sh = TileShape<S, T, TX, TY>;
    const int gxn = (g.nx + Sh::W - 1) / Sh::W, gyn = (g.ny + TY - 1) / TY;
    int n = 0;
    for (int z = 0; z < g.nz; z += zchunk)
        for (int by = 0; by < gyn; ++by)
            for (int bx = 0; bx < gxn; ++bx) {
                if (out) out[n] = BatchItem{grid_index, bx, by, z, min(z + zchunk, g.nz), shape};
                ++n;
            }
    return n;
}

template <class S, class T, int TX, int TY, bool SQ = false, bool SR = false>
cudaError_t launch_batch_t(const void *grids, const BatchItem *work, int nwork, int parity, int *err,
                           int stencil, int kind, cudaStream_t st, const long long *steps = nullptr,
                           int sub = 0, int fwd = 0)
{
    using Sh = TileShape<S, T, TX, TY>;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int ctas = sms * BatchMinBlocks<S>::value;
    if (ctas > nwork) ctas = nwork;
    if (ctas < 1) return cudaSuccess;
    const BatchGrid<T> *bg = (const BatchGrid<T> *)grids;
#define SPFM_BLAUNCH(ST, KD)                                                                               \
    spfm_batch_kernel<S, T, ST, KD, TX, TY, SQ, SR><<<ctas, Sh::NTHREADS, 0, st>>>(bg, work, nwork, parity, err, \
                                                                                 steps, sub, fwd)
#define SPFM_BBY_KIND(ST)                      \
    do {                                       \
        if (kind == 0) SPFM_BLAUNCH(ST, 0);    \
        else SPFM_BLAUNCH(ST, 5);              \
    } while (0)
    if (stencil == 6) SPFM_BBY_KIND(6);
    else if (stencil == 18) SPFM_BBY_KIND(18);
    else SPFM_BBY_KIND(26);
#undef SPFM_BBY_KIND
#undef SPFM_BLAUNCH
    return cudaGetLastError();
}

// IMG: the kernels that write the periodic ghost images (cfg.mode has kImages)
template <class S, class T, int TX, int TY, bool IMG, bool SR = false>
cudaError_t launch_step_t(const StepCoef<T> &c, const S *src, S *dst, int *err, LaunchCfg cfg,
                          const CUtensorMap *tmap, cudaStream_t st)
{
    using Sh = TileShape<S, T, TX, TY>;
    const int gxn = (c.g.nx + Sh::W - 1) / Sh::W, gyn = (c.g.ny + TY - 1) / TY;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int target = 6 * MinBlocks<S>::value * sms;
    // exact group counts 1..4 get their own kernels; 0 groups (all A_k = 0)
    // runs the one-group kernel with beta = 0
    const int kind = is_fd_scheme(cfg.scheme) ? 0
                     : cfg.scheme == SPFM_TI_LOCAL ? 6
                                                   : (c.nterms <= 4 ? (c.nterms < 1 ? 1 : c.nterms) : 5);
    const PackCoef<T> pc = make_pack_coef<T>(c);
    CUtensorMap map;
    if (tmap) map = *tmap;
    else memset(&map, 0, sizeof map);
    const int use = tmap ? 1 : 0;
    constexpr int R = SPFM_ROWS_PER_THREAD;
    constexpr int NT1 = TileShape<S, T, TX, TY, 1>::NTHREADS;
    // programmatic dependent launch: the kernel may begin while the previous
    // kernel in the stream runs; cfg.mode says which boxes wait (griddepcontrol)
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t lc = {};
    lc.dynamicSmemBytes = 0;
    lc.stream = st;
    lc.attrs = attr;
    lc.numAttrs = 1;
    const int mode = cfg.mode;
    // z-chunk: the caller's, else the launch-shape model's for this kernel (a
    // grid dimension stays below 65536 chunks)
    auto go = [&](auto kern, int threads) {
        int zchunk = cfg.zchunk > 0 ? cfg.zchunk : pick_zchunk((const void *)kern, threads, gxn * gyn, c.g.nz, target);
        if (zchunk > c.g.nz) zchunk = c.g.nz;
        if (zchunk < (c.g.nz + 65534) / 65535) zchunk = (c.g.nz + 65534) / 65535;
        if (cfg.zchunk_used) *cfg.zchunk_used = zchunk;
        lc.gridDim = dim3(gxn, gyn, (c.g.nz + zchunk - 1) / zchunk);
        lc.blockDim = dim3(threads);
        return cudaLaunchKernelEx(&lc, kern, c, pc, src, dst, err, zchunk, map, use, mode);
    };
    cudaError_t le = cudaSuccess;
#define SPFM_LAUNCH(ST, KD) le = go(spfm_step_kernel<S, T, ST, KD, TX, TY, R, IMG, SR>, Sh::NTHREADS)
#define SPFM_BY_KIND(ST)                        \
    do {                                        \
        if (kind == 0) SPFM_LAUNCH(ST, 0);      \
        else if (kind == 1) SPFM_LAUNCH(ST, 1); \
        else if (kind == 2) SPFM_LAUNCH(ST, 2); \
        else if (kind == 3) SPFM_LAUNCH(ST, 3); \
        else if (kind == 4) SPFM_LAUNCH(ST, 4); \
        else if (kind == 5) SPFM_LAUNCH(ST, 5); \
        else le = go(spfm_step_kernel<S, T, ST, 6, TX, TY, 1, IMG, SR>, NT1); \
    } while (0)
    if (cfg.stencil == 6) SPFM_BY_KIND(6);
    else if (cfg.stencil == 18) SPFM_BY_KIND(18);
    else SPFM_BY_KIND(26);
#undef SPFM_BY_KIND
#undef SPFM_LAUNCH
    if (le != cudaSuccess) return le;
    return cudaGetLastError();
}

}  // namespace spfm
