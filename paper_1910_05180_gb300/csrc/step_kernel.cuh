// step_kernel.cuh -- z-marching 2.5D stencil kernel of one explicit SPFM / CF step.
//
// One CTA owns an xy tile of TX*VX by TY cells (VX = cells per 16 bytes) and
// marches through a chunk of z planes.  Each arriving plane is staged, with a
// one-cell halo whose ghost cells come from the boundary conditions, in a
// double-buffered shared-memory tile, so one __syncthreads per plane suffices;
// the next plane's 16-byte global loads are issued before the barrier and land
// in registers while this plane is being used.  The x/y ghost mapping of every
// load slot is resolved once per CTA; per plane only the z mapping changes.
//
// From each plane every thread forms, for its cells, three plane quantities:
//   C  = phi at the cell,
//   F' = sum of the 4 in-plane face neighbours minus C (each as a difference),
//   E' = sum of the 4 in-plane diagonal neighbours minus C,
// kept in registers for the planes z-1, z, z+1 (the z loop is unrolled by
// three with rotating register roles, so nothing is copied between planes).
// The shell sums of the 27-point stencil then follow without re-reading:
//   S1 - 6 phi  = F'_z + t,             t = (C_{z-1} - phi) + (C_{z+1} - phi)
//   S2 - 12 phi = E'_z + F'_{z-1} + F'_{z+1} + 4 t
//   S3 - 8 phi  = E'_{z-1} + E'_{z+1} + 4 t
// Every term is a difference of neighbouring values, which keeps FP32 drift far
// below a plain sum of neighbours.
//
// FP32 arithmetic runs on packed f32x2 pairs (FFMA2/FADD2/FMUL2 of sm_100+).  A
// thread's four cells x..x+3 form the packs A = (x, x+2) and B = (x+1, x+3);
// shared memory holds every 16-byte quad in the order (v0, v2, v1, v3), so one
// 128-bit shared load yields both packs in aligned register pairs and the
// x-neighbour packs are W(A) = (x-1, x+1), E(A) = B, W(B) = A, E(B) = (x+2, x+4).
// FP64 runs on scalar doubles with the same structure.
#pragma once

#include "spfm_internal.h"

namespace spfm {

// ------------------------------------------------------------ pack arithmetic

template <class T> struct Pk;

template <> struct Pk<float> {
    using P = float2;
    static __device__ __forceinline__ P mk(float a, float b) { return make_float2(a, b); }
    static __device__ __forceinline__ P add(P a, P b) { return __fadd2_rn(a, b); }
    static __device__ __forceinline__ P mul(P a, P b) { return __fmul2_rn(a, b); }
    static __device__ __forceinline__ P fma(P a, P b, P c) { return __ffma2_rn(a, b, c); }
    static __device__ __forceinline__ P sub(P a, P b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
    static __device__ __forceinline__ P div(P a, P b)
    {
        return make_float2(__fdividef(a.x, b.x), __fdividef(a.y, b.y));
    }
};

struct D2 { double x, y; };

template <> struct Pk<double> {
    using P = D2;
    static __device__ __forceinline__ P mk(double a, double b) { return {a, b}; }
    static __device__ __forceinline__ P add(P a, P b) { return {a.x + b.x, a.y + b.y}; }
    static __device__ __forceinline__ P mul(P a, P b) { return {a.x * b.x, a.y * b.y}; }
    static __device__ __forceinline__ P fma(P a, P b, P c)
    {
        return {__fma_rn(a.x, b.x, c.x), __fma_rn(a.y, b.y, c.y)};
    }
    static __device__ __forceinline__ P sub(P a, P b) { return {a.x - b.x, a.y - b.y}; }
    static __device__ __forceinline__ P div(P a, P b) { return {a.x / b.x, a.y / b.y}; }
};

template <class T> struct PackT;
template <> struct PackT<float> { using P = float2; static P splat(float v) { return make_float2(v, v); } };
template <> struct PackT<double> { using P = D2; static P splat(double v) { return {v, v}; } };

// Step coefficients pre-splatted into packs (kernel parameter space).
template <class T>
struct PackCoef {
    using P = typename PackT<T>::P;
    P one, m2, four, c1, c2, c3, dt, nkmu, kappa;
    P nA[kMaxTerms], beta[kMaxTerms];
    int nterms;
};

template <class T>
inline PackCoef<T> make_pack_coef(const StepCoef<T> &c)
{
    using PT = PackT<T>;
    PackCoef<T> p;
    p.one = PT::splat(T(1));
    p.m2 = PT::splat(T(-2));
    p.four = PT::splat(T(4));
    p.c1 = PT::splat(c.c1);
    p.c2 = PT::splat(c.c2);
    p.c3 = PT::splat(c.c3);
    p.dt = PT::splat(c.dt);
    p.nkmu = PT::splat(-c.kmu);
    p.kappa = PT::splat(c.kappa);
    for (int k = 0; k < kMaxTerms; ++k) {
        p.nA[k] = PT::splat(-c.A[k]);
        p.beta[k] = PT::splat(c.beta[k]);
    }
    p.nterms = c.nterms;
    return p;
}

// ------------------------------------------------------ storage <-> compute

template <class S, class T> struct Io;

template <> struct Io<float, float> {
    static constexpr int VX = 4;
    static __device__ __forceinline__ void ld(const float *p, float *v)
    {
        float4 r = __ldg(reinterpret_cast<const float4 *>(p));
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
    static __device__ __forceinline__ void ld(const double *p, double *v)
    {
        double2 r = __ldg(reinterpret_cast<const double2 *>(p));
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
    static __device__ __forceinline__ void ld(const __nv_bfloat16 *p, float *v)
    {
        uint4 r = __ldg(reinterpret_cast<const uint4 *>(p));
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

// ------------------------------------------------------------- load slots

// One staged load of a plane: a row of VX cells (or one cell) whose x/y ghost
// mapping is fixed for the whole z march.
struct Slot {
    long long row;   // sy * pitch (+ gx when xfull)
    int gx;          // first x of the slot
    int yface;       // contact face of the y mapping, or -1
    int mode;        // 0 inactive (value unused), 1 full vector in range, 2 per element
};

__device__ __forceinline__ Slot make_slot(const GridGeom &g, int gx, int gy, int width)
{
    Slot s;
    s.gx = gx;
    s.yface = -1;
    if (gy < -1 || gy > g.ny || gx > g.nx || gx + width - 1 < -1) {
        s.mode = 0;
        s.row = 0;
        return s;
    }
    const int sy = map_axis(gy, g.ny, g.bc[2], g.bc[3], &s.yface, 2);
    s.row = (long long)sy * g.pitch;
    if (gx >= 0 && gx + width <= g.nx) {
        s.mode = 1;
        s.row += gx;
    } else {
        s.mode = 2;
    }
    return s;
}

// Loads the slot's `width` cells of plane (already z-mapped) `pbase`, applying
// the ghost maps of x (per element), y (per slot) and z (per plane).
template <class S, class T, int WIDTH>
__device__ __forceinline__ void load_slot(const StepCoef<T> &C, const S *__restrict__ pbase,
                                          const Slot &s, int zface, T *out)
{
    if (s.mode == 1) {
        if (WIDTH == 1) out[0] = Io<S, T>::cvt_in(pbase[s.row]);
        else Io<S, T>::ld(pbase + s.row, out);
    } else if (s.mode == 2) {
#pragma unroll
        for (int e = 0; e < WIDTH; ++e) {
            const int gx = s.gx + e;
            T v = T(0);
            if (gx >= -1 && gx <= C.g.nx) {
                int fx;
                const int sx = map_axis(gx, C.g.nx, C.g.bc[0], C.g.bc[1], &fx, 0);
                v = Io<S, T>::cvt_in(pbase[s.row + sx]);
                if (fx >= 0) v = contact_shift<T>(v, C.aface[fx]);
            }
            out[e] = v;
        }
    } else {
#pragma unroll
        for (int e = 0; e < WIDTH; ++e) out[e] = T(0);
    }
    if (s.yface >= 0) {
#pragma unroll
        for (int e = 0; e < WIDTH; ++e) out[e] = contact_shift<T>(out[e], C.aface[s.yface]);
    }
    if (zface >= 0) {
#pragma unroll
        for (int e = 0; e < WIDTH; ++e) out[e] = contact_shift<T>(out[e], C.aface[zface]);
    }
}

// ------------------------------------------------------ shared-memory rows

// Shared rows hold quads of 4 cells in the order (v0, v2, v1, v3) for VX >= 4.
template <class T, int VX>
__device__ __forceinline__ void put_row(T *dst, const T *v)
{
    if constexpr (VX == 2) {
        dst[0] = v[0];
        dst[1] = v[1];
    } else {
#pragma unroll
        for (int q = 0; q < VX / 4; ++q) {
            if constexpr (sizeof(T) == 4) {
                *reinterpret_cast<float4 *>(dst + 4 * q) =
                    make_float4(v[4 * q], v[4 * q + 2], v[4 * q + 1], v[4 * q + 3]);
            } else {
                dst[4 * q] = v[4 * q];
                dst[4 * q + 1] = v[4 * q + 2];
                dst[4 * q + 2] = v[4 * q + 1];
                dst[4 * q + 3] = v[4 * q + 3];
            }
        }
    }
}

// The packs of one shared row around a thread's cells: C[p], W[p], E[p].
template <class T, int VX>
struct RowPacks {
    using P = typename Pk<T>::P;
    static constexpr int NP = VX / 2;
    P c[NP], w[NP], e[NP];
};

template <class T, int VX>
__device__ __forceinline__ void get_row(const T *r, RowPacks<T, VX> &o)
{
    using K = Pk<T>;
    if constexpr (VX == 2) {
        const T l = r[-1], v0 = r[0], v1 = r[1], rr = r[2];
        o.c[0] = K::mk(v0, v1);
        o.w[0] = K::mk(l, v0);
        o.e[0] = K::mk(v1, rr);
    } else {
        constexpr int NQ = VX / 4;
        typename Pk<T>::P a[NQ], b[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            if constexpr (sizeof(T) == 4) {
                const float4 f = *reinterpret_cast<const float4 *>(r + 4 * q);
                a[q] = K::mk(f.x, f.y);   // (v0, v2)
                b[q] = K::mk(f.z, f.w);   // (v1, v3)
            } else {
                a[q] = K::mk(r[4 * q], r[4 * q + 1]);
                b[q] = K::mk(r[4 * q + 2], r[4 * q + 3]);
            }
        }
        const T l = r[-1], rr = r[VX];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            o.c[2 * q] = a[q];
            o.c[2 * q + 1] = b[q];
            o.w[2 * q] = K::mk(q == 0 ? l : b[q - 1].y, b[q].x);          // (x-1, x+1)
            o.e[2 * q] = b[q];                                            // (x+1, x+3)
            o.w[2 * q + 1] = a[q];                                        // (x,   x+2)
            o.e[2 * q + 1] = K::mk(a[q].y, q == NQ - 1 ? rr : a[q + 1].x);  // (x+2, x+4)
        }
    }
}

// cell index (0..VX-1) of lane `lane` of pack p
template <int VX>
__device__ __forceinline__ constexpr int pack_cell(int p, int lane)
{
    return VX == 2 ? p * 2 + lane : (p / 2) * 4 + (p % 2) + 2 * lane;
}

// -------------------------------------------------------------------- tile

template <class S, class T, int TX, int TY>
struct TileShape {
    static constexpr int VX = Io<S, T>::VX;
    static constexpr int NP = VX / 2;
    static constexpr int W = TX * VX;
    static constexpr int SW = W + 2 * VX;   // interior starts at VX (16-byte aligned)
    static constexpr int ROWS = TY + 2;
    static constexpr int SMEM_ELEMS = 2 * ROWS * SW;
};

template <class T, int NP>
struct PlaneQ {
    using P = typename Pk<T>::P;
    P c[NP], f[NP], e[NP];
};

// KIND: 0 = CF potential, 1 = TI global with <= 4 groups, 2 = TI global <= 13 groups
template <class S, class T, int STENCIL, int KIND, int TX, int TY>
__device__ __forceinline__ void step_tile(const StepCoef<T> &C, const PackCoef<T> &PC,
                                          const S *__restrict__ src, S *__restrict__ dst, int bx,
                                          int by, int zc0, int zc1, T *__restrict__ sbuf)
{
    using Sh = TileShape<S, T, TX, TY>;
    using K = Pk<T>;
    using P = typename K::P;
    constexpr int VX = Sh::VX, NP = Sh::NP, W = Sh::W, SW = Sh::SW, ROWS = Sh::ROWS;
    constexpr int NTMAX = KIND == 1 ? 4 : kMaxTerms;

    const GridGeom &g = C.g;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x0 = bx * W, y0 = by * TY;
    const int gx = x0 + tx * VX;
    const int gy = y0 + ty;
    const bool has_extra = ty < 2;
    const int extra_row = ty == 0 ? 0 : ROWS - 1;
    const bool has_side = tid < 2 * ROWS;
    const int side_row = tid >> 1, side_right = tid & 1;
    const bool out_ok = gy < g.ny && gx < g.nx;

    // x/y ghost mapping of the three load slots, fixed for the whole march
    const Slot s_own = make_slot(g, gx, gy, VX);
    const Slot s_extra = has_extra ? make_slot(g, gx, ty == 0 ? y0 - 1 : y0 + TY, VX) : Slot{0, 0, -1, 0};
    const Slot s_side = has_side ? make_slot(g, side_right ? x0 + W : x0 - 1, y0 + side_row - 1, 1)
                                 : Slot{0, 0, -1, 0};
    T *const own_dst0 = sbuf + (ty + 1) * SW + VX + tx * VX;
    T *const extra_dst0 = sbuf + extra_row * SW + VX + tx * VX;
    T *const side_dst0 = sbuf + side_row * SW + (side_right ? VX + W : VX - 1);

    T own[VX], extra[VX], side[1];
    auto fetch = [&](int z) {
        int zf;
        const int sz = map_axis(z, g.nz, g.bc[4], g.bc[5], &zf, 4);
        const S *pb = src + (long long)sz * g.plane;
        load_slot<S, T, VX>(C, pb, s_own, zf, own);
        if (has_extra) load_slot<S, T, VX>(C, pb, s_extra, zf, extra);
        if (has_side) load_slot<S, T, 1>(C, pb, s_side, zf, side);
    };

    S *out_base = dst + (long long)gy * g.pitch + gx;

    // one arriving plane: publish, prefetch the next, reduce to plane quantities,
    // and emit the output plane pz-1 from (m, z, p).  Returns false after the last.
    auto body = [&](int k, PlaneQ<T, NP> &m, PlaneQ<T, NP> &z, PlaneQ<T, NP> &p) -> bool {
        const int pz = zc0 - 1 + k;
        const int boff = (k & 1) * (ROWS * SW);
        put_row<T, VX>(own_dst0 + boff, own);
        if (has_extra) put_row<T, VX>(extra_dst0 + boff, extra);
        if (has_side) side_dst0[boff] = side[0];
        if (pz < zc1) fetch(pz + 1);
        __syncthreads();

        {
            const T *r0 = own_dst0 + boff;
            RowPacks<T, VX> rc, rn, rs;
            get_row<T, VX>(r0, rc);
            get_row<T, VX>(r0 - SW, rn);
            get_row<T, VX>(r0 + SW, rs);
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                const P c = rc.c[q];
                p.c[q] = c;
                p.f[q] = K::add(K::add(K::sub(rc.w[q], c), K::sub(rc.e[q], c)),
                                K::add(K::sub(rn.c[q], c), K::sub(rs.c[q], c)));
                if (STENCIL != 6)
                    p.e[q] = K::add(K::add(K::sub(rn.w[q], c), K::sub(rn.e[q], c)),
                                    K::add(K::sub(rs.w[q], c), K::sub(rs.e[q], c)));
            }
        }

        if (k >= 2 && out_ok) {
            T outv[VX];
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                const P ph = z.c[q];
                const P t = K::add(K::sub(m.c[q], ph), K::sub(p.c[q], ph));
                P lap = K::mul(PC.c1, K::add(z.f[q], t));
                if (STENCIL != 6) {
                    const P s2 = K::fma(PC.four, t, K::add(z.e[q], K::add(m.f[q], p.f[q])));
                    lap = K::fma(PC.c2, s2, lap);
                }
                if (STENCIL == 26) {
                    const P s3 = K::fma(PC.four, t, K::add(m.e[q], p.e[q]));
                    lap = K::fma(PC.c3, s3, lap);
                }
                const P s = K::fma(PC.m2, ph, PC.one);          // 1 - 2 phi
                const P q1 = K::mul(ph, K::sub(PC.one, ph));     // phi (1 - phi)
                const P qs = K::mul(q1, s);
                P pot;
                if (KIND == 0) {
                    pot = K::mul(PC.kappa, qs);
                } else {
                    const P u = K::mul(s, s);
                    P num = PC.beta[0];
                    P den = K::fma(PC.nA[0], u, PC.one);
#pragma unroll
                    for (int kk = 1; kk < NTMAX; ++kk) {
                        if (kk < PC.nterms) {
                            const P d = K::fma(PC.nA[kk], u, PC.one);
                            num = K::fma(num, d, K::mul(PC.beta[kk], den));
                            den = K::mul(den, d);
                        }
                    }
                    pot = K::mul(qs, K::div(num, den));
                }
                P R = K::sub(lap, pot);
                R = K::fma(PC.nkmu, q1, R);
                const P o = K::fma(PC.dt, R, ph);
                outv[pack_cell<VX>(q, 0)] = o.x;
                outv[pack_cell<VX>(q, 1)] = o.y;
            }
            S *optr = out_base + (long long)(pz - 1) * g.plane;
            if (gx + VX <= g.nx) {
                Io<S, T>::st(optr, outv);
            } else {
#pragma unroll
                for (int e = 0; e < VX; ++e)
                    if (gx + e < g.nx) optr[e] = Io<S, T>::cvt_out(outv[e]);
            }
        }
        return pz < zc1;
    };

    PlaneQ<T, NP> q0, q1, q2;
    fetch(zc0 - 1);
    for (int k = 0;; k += 3) {
        if (!body(k, q1, q2, q0)) break;
        if (!body(k + 1, q2, q0, q1)) break;
        if (!body(k + 2, q0, q1, q2)) break;
    }
}

// minimum resident CTAs per SM: caps registers so three 256-thread CTAs fit
template <class T> struct MinBlocks { static constexpr int value = sizeof(T) == 4 ? 3 : 2; };

template <class S, class T, int STENCIL, int KIND, int TX, int TY>
__global__ void __launch_bounds__(TX *TY, MinBlocks<T>::value)
    spfm_step_kernel(const StepCoef<T> C, const PackCoef<T> PC, const S *__restrict__ src,
                     S *__restrict__ dst, int zchunk)
{
    using Sh = TileShape<S, T, TX, TY>;
    __shared__ __align__(16) T sbuf[Sh::SMEM_ELEMS];
    const int zc0 = blockIdx.z * zchunk;
    const int zc1 = min(zc0 + zchunk, C.g.nz);
    step_tile<S, T, STENCIL, KIND, TX, TY>(C, PC, src, dst, blockIdx.x, blockIdx.y, zc0, zc1, sbuf);
}

// z-chunk length so that the launch has enough CTAs for 152 SMs
inline int pick_zchunk(int tiles_xy, int nz)
{
    const int target = 2048;
    int chunks = (target + tiles_xy - 1) / tiles_xy;
    int max_chunks = nz / 16 > 1 ? nz / 16 : 1;
    if (chunks > max_chunks) chunks = max_chunks;
    if (chunks < 1) chunks = 1;
    return (nz + chunks - 1) / chunks;
}

template <class S, class T, int TX, int TY>
cudaError_t launch_step_t(const StepCoef<T> &c, const S *src, S *dst, LaunchCfg cfg, cudaStream_t st)
{
    using Sh = TileShape<S, T, TX, TY>;
    const dim3 block(TX, TY);
    const int gxn = (c.g.nx + Sh::W - 1) / Sh::W, gyn = (c.g.ny + TY - 1) / TY;
    const int zchunk = pick_zchunk(gxn * gyn, c.g.nz);
    const dim3 grid(gxn, gyn, (c.g.nz + zchunk - 1) / zchunk);
    const int kind = cfg.scheme == SPFM_FD ? 0 : (c.nterms <= 4 ? 1 : 2);
    const PackCoef<T> pc = make_pack_coef<T>(c);
#define SPFM_LAUNCH(ST, KD) \
    spfm_step_kernel<S, T, ST, KD, TX, TY><<<grid, block, 0, st>>>(c, pc, src, dst, zchunk)
#define SPFM_BY_KIND(ST)                        \
    do {                                        \
        if (kind == 0) SPFM_LAUNCH(ST, 0);      \
        else if (kind == 1) SPFM_LAUNCH(ST, 1); \
        else SPFM_LAUNCH(ST, 2);                \
    } while (0)
    if (cfg.stencil == 6) SPFM_BY_KIND(6);
    else if (cfg.stencil == 18) SPFM_BY_KIND(18);
    else SPFM_BY_KIND(26);
#undef SPFM_BY_KIND
#undef SPFM_LAUNCH
    return cudaGetLastError();
}

}  // namespace spfm
