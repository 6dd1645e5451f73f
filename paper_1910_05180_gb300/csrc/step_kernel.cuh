// step_kernel.cuh -- z-marching 2.5D stencil kernel of one explicit SPFM / CF step.
//
// One CTA owns an xy tile of TX*VX by TY cells and marches through a chunk of z
// planes.  Each arriving plane is staged (with a one-cell halo whose ghost cells
// come from the boundary conditions) in shared memory, double-buffered so one
// __syncthreads per plane suffices; the next plane's 16-byte global loads are
// issued before the barrier and land in registers while this plane is used.
//
// From each plane every thread forms, for its cells, three plane quantities:
//   C  = phi at the cell,
//   F' = sum of the 4 in-plane face neighbours minus C (each as a difference),
//   E' = sum of the 4 in-plane diagonal neighbours minus C,
// kept in registers for the planes z-1, z, z+1.  The shell sums of the 27-point
// stencil then follow without re-reading neighbours:
//   S1 - 6 phi  = F'_z + t,             t = (C_{z-1} - phi) + (C_{z+1} - phi)
//   S2 - 12 phi = E'_z + F'_{z-1} + F'_{z+1} + 4 t
//   S3 - 8 phi  = E'_{z-1} + E'_{z+1} + 4 t
// Every term is a difference of neighbouring values, which keeps FP32 drift far
// below a plain sum of neighbours.  FP32 arithmetic runs on packed f32x2 pairs
// (FFMA2/FADD2/FMUL2 of sm_100+); FP64 on scalar doubles.
#pragma once

#include "spfm_internal.h"

namespace spfm {

// ------------------------------------------------------------ pack arithmetic

template <class T> struct Pk;

template <> struct Pk<float> {
    using P = float2;
    static __device__ __forceinline__ P mk(float a, float b) { return make_float2(a, b); }
    static __device__ __forceinline__ P splat(float a) { return make_float2(a, a); }
    static __device__ __forceinline__ P add(P a, P b) { return __fadd2_rn(a, b); }
    static __device__ __forceinline__ P mul(P a, P b) { return __fmul2_rn(a, b); }
    static __device__ __forceinline__ P fma(P a, P b, P c) { return __ffma2_rn(a, b, c); }
    static __device__ __forceinline__ P sub(P a, P b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
    static __device__ __forceinline__ P div(P a, P b)
    {
        return make_float2(__fdividef(a.x, b.x), __fdividef(a.y, b.y));
    }
};

template <> struct Pk<double> {
    struct P { double x, y; };
    static __device__ __forceinline__ P mk(double a, double b) { return {a, b}; }
    static __device__ __forceinline__ P splat(double a) { return {a, a}; }
    static __device__ __forceinline__ P add(P a, P b) { return {a.x + b.x, a.y + b.y}; }
    static __device__ __forceinline__ P mul(P a, P b) { return {a.x * b.x, a.y * b.y}; }
    static __device__ __forceinline__ P fma(P a, P b, P c)
    {
        return {__fma_rn(a.x, b.x, c.x), __fma_rn(a.y, b.y, c.y)};
    }
    static __device__ __forceinline__ P sub(P a, P b) { return {a.x - b.x, a.y - b.y}; }
    static __device__ __forceinline__ P div(P a, P b) { return {a.x / b.x, a.y / b.y}; }
};

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

// Element (gx, gy, gz) of the source with ghost cells from the boundary
// conditions; up to one cell outside per axis, 0 beyond (never used as data).
template <class S, class T>
__device__ __forceinline__ T load_elem(const StepCoef<T> &C, const S *__restrict__ src, int gx,
                                       int gy, int gz)
{
    const GridGeom &g = C.g;
    if (gx < -1 || gx > g.nx || gy < -1 || gy > g.ny || gz < -1 || gz > g.nz) return T(0);
    int fx, fy, fz;
    const int sx = map_axis(gx, g.nx, g.bc[0], g.bc[1], &fx, 0);
    const int sy = map_axis(gy, g.ny, g.bc[2], g.bc[3], &fy, 2);
    const int sz = map_axis(gz, g.nz, g.bc[4], g.bc[5], &fz, 4);
    T v = Io<S, T>::cvt_in(src[(long long)sz * g.plane + (long long)sy * g.pitch + sx]);
    // contact shifts compose (they are translations of the ideal profile)
    if (fx >= 0) v = contact_shift<T>(v, C.aface[fx]);
    if (fy >= 0) v = contact_shift<T>(v, C.aface[fy]);
    if (fz >= 0) v = contact_shift<T>(v, C.aface[fz]);
    return v;
}

template <class S, class T>
__device__ __forceinline__ void fetch_vec(const StepCoef<T> &C, const S *__restrict__ src, int gx,
                                          int gy, int gz, T *out)
{
    constexpr int VX = Io<S, T>::VX;
    const GridGeom &g = C.g;
    if (gz >= 0 && gz < g.nz && gy >= 0 && gy < g.ny && gx >= 0 && gx + VX <= g.nx) {
        Io<S, T>::ld(src + (long long)gz * g.plane + (long long)gy * g.pitch + gx, out);
    } else {
#pragma unroll
        for (int e = 0; e < VX; ++e) out[e] = load_elem<S, T>(C, src, gx + e, gy, gz);
    }
}

// cells of pack p (two lanes): for VX = 2 (0,1); otherwise (0,2),(1,3),(4,6),(5,7)
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

// KIND: 0 = CF potential, 1 = TI global with <= 4 groups, 2 = TI global <= 13 groups
template <class S, class T, int STENCIL, int KIND, int TX, int TY>
__device__ __forceinline__ void step_tile(const StepCoef<T> &C, const S *__restrict__ src,
                                          S *__restrict__ dst, int bx, int by, int zc0, int zc1,
                                          T *__restrict__ sbuf)
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
    const int extra_gy = ty == 0 ? y0 - 1 : y0 + TY;
    const bool has_side = tid < 2 * ROWS;
    const int side_row = tid >> 1, side_right = tid & 1;
    const int side_gx = side_right ? x0 + W : x0 - 1;
    const int side_gy = y0 + side_row - 1;
    const bool out_ok = gy < g.ny && gx < g.nx;

    T own[VX], extra[VX], side = T(0);
#pragma unroll
    for (int e = 0; e < VX; ++e) extra[e] = T(0);

    auto fetch = [&](int z) {
        fetch_vec<S, T>(C, src, gx, gy, z, own);
        if (has_extra) fetch_vec<S, T>(C, src, gx, extra_gy, z, extra);
        if (has_side) side = load_elem<S, T>(C, src, side_gx, side_gy, z);
    };

    P Cm[NP], Fm[NP], Em[NP], C0[NP], F0[NP], E0[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        Cm[p] = C0[p] = Fm[p] = F0[p] = Em[p] = E0[p] = K::splat(T(0));
    }

    const P one = K::splat(T(1)), m2 = K::splat(T(-2)), four = K::splat(T(4));
    const P pc1 = K::splat(C.c1), pc2 = K::splat(C.c2), pc3 = K::splat(C.c3);
    const P pdt = K::splat(C.dt), pnkmu = K::splat(-C.kmu), pkap = K::splat(C.kappa);

    fetch(zc0 - 1);
    int it = 0;
    for (int pz = zc0 - 1; pz <= zc1; ++pz, ++it) {
        T *b = sbuf + (it & 1) * (ROWS * SW);
        // publish the staged plane pz
        {
            T *row = b + (ty + 1) * SW + VX + tx * VX;
#pragma unroll
            for (int e = 0; e < VX; ++e) row[e] = own[e];
            if (has_extra) {
                T *er = b + extra_row * SW + VX + tx * VX;
#pragma unroll
                for (int e = 0; e < VX; ++e) er[e] = extra[e];
            }
            if (has_side) b[side_row * SW + (side_right ? VX + W : VX - 1)] = side;
        }
        if (pz < zc1) fetch(pz + 1);
        __syncthreads();

        // plane quantities of plane pz for this thread's cells
        P Cp[NP], Fp[NP], Ep[NP];
        {
            const T *r0 = b + (ty + 1) * SW + VX + tx * VX;
            const T *rn = r0 - SW;
            const T *rs = r0 + SW;
            T v0[VX + 2], vn[VX + 2], vs[VX + 2];
#pragma unroll
            for (int e = -1; e <= VX; ++e) v0[e + 1] = r0[e];
#pragma unroll
            for (int e = 0; e < VX; ++e) { vn[e + 1] = rn[e]; vs[e + 1] = rs[e]; }
            if (STENCIL != 6) {
                vn[0] = rn[-1]; vn[VX + 1] = rn[VX];
                vs[0] = rs[-1]; vs[VX + 1] = rs[VX];
            }
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const int i0 = pack_cell<VX>(p, 0) + 1, i1 = pack_cell<VX>(p, 1) + 1;
                const P c = K::mk(v0[i0], v0[i1]);
                const P w = K::mk(v0[i0 - 1], v0[i1 - 1]);
                const P e = K::mk(v0[i0 + 1], v0[i1 + 1]);
                const P n = K::mk(vn[i0], vn[i1]);
                const P s = K::mk(vs[i0], vs[i1]);
                Cp[p] = c;
                Fp[p] = K::add(K::add(K::sub(w, c), K::sub(e, c)), K::add(K::sub(n, c), K::sub(s, c)));
                if (STENCIL != 6) {
                    const P nw = K::mk(vn[i0 - 1], vn[i1 - 1]), ne = K::mk(vn[i0 + 1], vn[i1 + 1]);
                    const P sw = K::mk(vs[i0 - 1], vs[i1 - 1]), se = K::mk(vs[i0 + 1], vs[i1 + 1]);
                    Ep[p] = K::add(K::add(K::sub(nw, c), K::sub(ne, c)), K::add(K::sub(sw, c), K::sub(se, c)));
                } else {
                    Ep[p] = K::splat(T(0));
                }
            }
        }

        if (pz >= zc0 + 1 && out_ok) {
            T outv[VX];
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const P ph = C0[p];
                const P t = K::add(K::sub(Cm[p], ph), K::sub(Cp[p], ph));
                P lap = K::mul(pc1, K::add(F0[p], t));
                if (STENCIL != 6) {
                    const P s2 = K::fma(four, t, K::add(E0[p], K::add(Fm[p], Fp[p])));
                    lap = K::fma(pc2, s2, lap);
                }
                if (STENCIL == 26) {
                    const P s3 = K::fma(four, t, K::add(Em[p], Ep[p]));
                    lap = K::fma(pc3, s3, lap);
                }
                const P s = K::fma(m2, ph, one);              // 1 - 2 phi
                const P q = K::mul(ph, K::sub(one, ph));       // phi (1 - phi)
                const P qs = K::mul(q, s);
                P pot;
                if (KIND == 0) {
                    pot = K::mul(pkap, qs);
                } else {
                    const P u = K::mul(s, s);
                    P num = K::splat(C.beta[0]);
                    P den = K::fma(K::splat(-C.A[0]), u, one);
#pragma unroll
                    for (int k = 1; k < NTMAX; ++k) {
                        if (k < C.nterms) {
                            const P d = K::fma(K::splat(-C.A[k]), u, one);
                            num = K::fma(num, d, K::mul(K::splat(C.beta[k]), den));
                            den = K::mul(den, d);
                        }
                    }
                    pot = K::mul(qs, K::div(num, den));
                }
                P R = K::sub(lap, pot);
                R = K::fma(pnkmu, q, R);
                const P o = K::fma(pdt, R, ph);
                outv[pack_cell<VX>(p, 0)] = o.x;
                outv[pack_cell<VX>(p, 1)] = o.y;
            }
            const int oz = pz - 1;
            S *optr = dst + (long long)oz * g.plane + (long long)gy * g.pitch + gx;
            if (gx + VX <= g.nx) {
                Io<S, T>::st(optr, outv);
            } else {
#pragma unroll
                for (int e = 0; e < VX; ++e)
                    if (gx + e < g.nx) optr[e] = Io<S, T>::cvt_out(outv[e]);
            }
        }
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            Cm[p] = C0[p]; Fm[p] = F0[p]; Em[p] = E0[p];
            C0[p] = Cp[p]; F0[p] = Fp[p]; E0[p] = Ep[p];
        }
    }
}

template <class S, class T, int STENCIL, int KIND, int TX, int TY>
__global__ void __launch_bounds__(TX *TY)
    spfm_step_kernel(const StepCoef<T> C, const S *__restrict__ src, S *__restrict__ dst, int zchunk)
{
    using Sh = TileShape<S, T, TX, TY>;
    __shared__ __align__(16) T sbuf[Sh::SMEM_ELEMS];
    const int zc0 = blockIdx.z * zchunk;
    const int zc1 = min(zc0 + zchunk, C.g.nz);
    step_tile<S, T, STENCIL, KIND, TX, TY>(C, src, dst, blockIdx.x, blockIdx.y, zc0, zc1, sbuf);
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
#define SPFM_LAUNCH(ST, KD) \
    spfm_step_kernel<S, T, ST, KD, TX, TY><<<grid, block, 0, st>>>(c, src, dst, zchunk)
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
