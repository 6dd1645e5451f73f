// api.cu -- the C ABI of include/spfm.h: grid handles, validation, host-side
// FP64 coefficients (a1), and the launches of the step, init and stats kernels.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "host_internal.h"

using namespace spfm;

namespace {

thread_local std::string t_err;

}  // namespace

namespace spfm_host {

void set_thread_error(const char *msg) { t_err = msg; }

int fail(spfm_grid *g, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (g) g->err = buf;
    t_err = buf;
    return code;
}

int cuda_fail(spfm_grid *g, cudaError_t e, const char *what)
{
    return fail(g, SPFM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

size_t elem_size(int dtype)
{
    return dtype == SPFM_F64 ? 8 : (dtype == SPFM_F32 ? 4 : 2);
}

int n_dirs(int stencil) { return stencil == 6 ? 3 : (stencil == 18 ? 9 : 13); }

void default_gamma(int stencil, const double *given, double *g)
{
    g[0] = given[0]; g[1] = given[1]; g[2] = given[2];
    if (g[0] == 0.0 && g[1] == 0.0 && g[2] == 0.0) {
        if (stencil == 6) { g[0] = 1.0; g[1] = 0.0; g[2] = 0.0; }
        else if (stencil == 18) { g[0] = 1.0 / 3.0; g[1] = 2.0 / 3.0; g[2] = 0.0; }
        else { g[0] = 0.5; g[1] = 1.0 / 3.0; g[2] = 1.0 / 6.0; }
    }
}

// TI_<hkl> coupling direction: the desc's u when given, else its normal n
static const double *coupling_dir(const spfm_grid *g)
{
    const double *u = g->d.u;
    return (u[0] != 0.0 || u[1] != 0.0 || u[2] != 0.0) ? u : g->d.n;
}

int build_model(spfm_grid *g, double M, double Gamma, double lambda, double dx, double dt,
                double dF, int stencil, int scheme, Model &m)
{
    if (!(M > 0.0) || !(Gamma > 0.0) || !(lambda > 0.0) || !(dx > 0.0) || !(dt > 0.0) ||
        !isfinite(M) || !isfinite(Gamma) || !isfinite(lambda) || !isfinite(dx) || !isfinite(dt) ||
        !isfinite(dF))
        return fail(g, SPFM_EINVAL, "spfm_step: M, Gamma, lambda, dx, dt must be finite and > 0");
    if (stencil != 6 && stencil != 18 && stencil != 26)
        return fail(g, SPFM_EINVAL, "spfm_step: stencil %d not in {6, 18, 26}", stencil);
    if (scheme != SPFM_TI_GLOBAL && scheme != SPFM_TI_LOCAL && !is_fd_scheme(scheme))
        return fail(g, SPFM_EINVAL, "spfm_step: unknown scheme %d", scheme);
    m.interp = scheme == SPFM_FD_H5 ? 1 : (scheme == SPFM_FD_HABEL ? 2 : 0);
    const int nd = n_dirs(stencil);
    default_gamma(stencil, g->d.gamma, m.gamma);
    const double nu[3] = {1.0, 0.5, 0.75};   // 3 / m_j, m = (3, 6, 4) directions per shell
    m.Cg = g->d.C_gamma > 0.0 ? g->d.C_gamma : 2.0 / 3.0;
    m.D = 2.0 * M / (3.0 * m.Cg);
    for (int j = 0; j < 3; ++j) {
        const bool active = (j == 0) || (j == 1 && stencil >= 18) || (j == 2 && stencil == 26);
        m.c_shell[j] = active ? m.D * m.gamma[j] * nu[j] / ((j + 1) * dx * dx) : 0.0;
    }
    double wsum = 0.0;
    for (int k = 0; k < kMaxTerms; ++k) {
        const Dir d = grid_dir(k);
        m.w[k] = k < nd ? m.gamma[d.shell - 1] * nu[d.shell - 1] : 0.0;
        m.ck[k] = k < nd ? m.c_shell[d.shell - 1] : 0.0;
        wsum += m.w[k];
        const double *u = coupling_dir(g);
        const double rn = dx * (d.x * u[0] + d.y * u[1] + d.z * u[2]);
        m.a[k] = tanh(2.0 * rn / lambda);   // Eq. 5
    }
    // group equal A_k = a_k^2 of the active directions (TI global)
    m.nterms = 0;
    for (int k = 0; k < nd; ++k) {
        const double A = m.a[k] * m.a[k];
        const double beta = 4.0 * m.ck[k] * A;
        if (!(A > 1e-300) || beta == 0.0) continue;
        int t = 0;
        for (; t < m.nterms; ++t)
            if (fabs(m.A[t] - A) <= 4e-15 * A) break;
        if (t == m.nterms) { m.A[t] = A; m.beta[t] = 0.0; ++m.nterms; }
        m.beta[t] += beta;
    }
    m.kmu = 4.0 * M * dF / (lambda * Gamma);
    m.kappa = m.D / (lambda * lambda) * (16.0 / 3.0) * wsum;
    for (int f = 0; f < 6; ++f) {
        const double sgn = (f % 2 == 0) ? -1.0 : 1.0;
        m.aface[f] = tanh(2.0 * sgn * dx * g->d.n[f / 2] / lambda);
    }
    // Spectral radius of the Laplacian part: its symbol is multilinear in
    // cos(xi_x), cos(xi_y), cos(xi_z), so the maximum sits on xi in {0, pi}^3.
    double lap = 0.0;
    for (int corner = 0; corner < 8; ++corner) {
        const double cx = (corner & 1) ? -1.0 : 1.0, cy = (corner & 2) ? -1.0 : 1.0,
                     cz = (corner & 4) ? -1.0 : 1.0;
        double s = 0.0;
        for (int k = 0; k < nd; ++k) {
            const Dir d = grid_dir(k);
            // cos(xi.d) with xi_i in {0, pi}: product of cos(xi_i)^|d_i|
            double c = 1.0;
            if (d.x) c *= cx;
            if (d.y) c *= cy;
            if (d.z) c *= cz;
            s += m.ck[k] * (2.0 - 2.0 * c);
        }
        lap = std::max(lap, s);
    }
    double pot = 0.0;
    if (is_fd_scheme(scheme)) {
        pot = m.kappa;
    } else {
        for (int k = 0; k < nd; ++k) {
            const Dir d = grid_dir(k);
            // TI_n: the largest coupling any local normal can give this direction
            const double amax = scheme == SPFM_TI_LOCAL
                                    ? tanh(2.0 * dx * sqrt((double)d.shell) / lambda)
                                    : fabs(m.a[k]);
            const double A = amax * amax;
            pot += 4.0 * m.ck[k] * A / (1.0 - A);
        }
    }
    // the driving term's derivative: kmu (d/dphi q)          <= kmu     (h3),
    // 5 kmu (d/dphi q^2) <= 2.5 kmu (h5), kmu/3 (d/dphi q/(1-2q)^2) <= kmu (h_Abel)
    m.bound = lap + pot + (m.interp == 1 ? 2.5 : 1.0) * fabs(m.kmu);
    if (dt * m.bound > 2.0)
        return fail(g, SPFM_EUNSTABLE,
                    "spfm_step: dt = %g exceeds the explicit-Euler bound 2/%g = %g", dt, m.bound,
                    2.0 / m.bound);
    // phase stability (Sec. 3.1): a barrier between the phases.  h3: |dF~| <
    // 8/(3 C lambda~); h_Abel: |dF~| < 8/(C lambda~) (derived; the paper prints
    // 440/(3 C lambda~)); h5: at any dF.
    if (scheme == SPFM_FD || scheme == SPFM_FD_HABEL) {
        const double lam_t = lambda / dx, dF_t = fabs(dF) * dx / Gamma;
        const double limit = (scheme == SPFM_FD ? 8.0 / 3.0 : 8.0) / (m.Cg * lam_t);
        if (dF_t >= limit)
            return fail(g, SPFM_EPHASE,
                        "spfm_step: CF driving force |dF dx/Gamma| = %g is beyond phase stability %g",
                        dF_t, limit);
    }
    return SPFM_OK;
}


cudaStream_t stream_of(const spfm_grid *g) { return (cudaStream_t)g->d.stream; }

// Refill the ghost layer of the current buffer for the given lambda and dx
// (contact faces depend on both), and clear the device error word.
int refresh_ghosts(spfm_grid *g, double lambda, double dx, cudaStream_t st)
{
    double af[6];
    for (int f = 0; f < 6; ++f) {
        const double sgn = (f % 2 == 0) ? -1.0 : 1.0;
        af[f] = tanh(2.0 * sgn * dx * g->d.n[f / 2] / lambda);
    }
    cudaError_t e = launch_fill_ghosts(g->geom, g->d.dtype, af, g->d.field[g->cur], st ? st : stream_of(g), 1);
    if (e != cudaSuccess) return cuda_fail(g, e, "ghost fill");
    g->ghosts_dirty = false;
    g->ghost_lambda = lambda;
    g->ghost_dx = dx;
    return SPFM_OK;
}

// Every face periodic, nx a whole number (>= 2) of 32-byte sectors and ny >= 2:
// the step kernel writes the ghost images of its new cells itself (kImages),
// its x images as whole sectors of the row pads.
bool faces_inline(const spfm_grid *g)
{
    for (int f = 0; f < 6; ++f)
        if (g->d.bc[f] == SPFM_PERIODIC) return false;
    return true;
}

bool writes_own_images(const spfm_grid *g)
{
    for (int f = 0; f < 6; ++f)
        if (g->d.bc[f] != SPFM_PERIODIC) return false;
    const int per32 = (int)(32 / g->elem);
    return g->d.nx % per32 == 0 && g->d.nx >= 2 * per32 && g->d.ny >= 2 && g->geom.off == per32;
}

int *err_word(const spfm_grid *g)
{
    return (int *)((char *)g->d.scratch + scratch_err_offset());
}


// Arguments of the stats pass over grid g (model of its last step or init).
void fill_stats_args(const spfm_grid *g, int flags, StatsArgs &a)
{
    memset(&a, 0, sizeof a);
    a.g = g->geom;
    a.dtype = g->d.dtype;
    for (int i = 0; i < 3; ++i) { a.n[i] = g->d.n[i]; a.ctr[i] = g->d.center[i]; }
    a.lambda = g->lambda;
    a.dx = g->dx;
    a.energy = (flags & SPFM_STATS_ENERGY) && g->scheme != SPFM_TI_LOCAL ? 1 : 0;
    a.scheme = g->scheme;
    a.stencil = g->stencil;
    a.Gamma = g->Gamma;
    a.C_gamma = g->d.C_gamma > 0.0 ? g->d.C_gamma : 2.0 / 3.0;
    double gam[3];
    default_gamma(g->stencil, g->d.gamma, gam);
    const double nu[3] = {1.0, 0.5, 0.75};
    const int nd = n_dirs(g->stencil);
    for (int k = 0; k < kMaxTerms; ++k) {
        const Dir d = grid_dir(k);
        a.w[k] = k < nd ? gam[d.shell - 1] * nu[d.shell - 1] : 0.0;
        const double *u = coupling_dir(g);
        a.a[k] = tanh(2.0 * g->dx * (d.x * u[0] + d.y * u[1] + d.z * u[2]) / g->lambda);
    }
}

// The public stats record from the kNStat reduced doubles of grid g.
void stats_from_reduction(const spfm_grid *g, const double *h, int energy, spfm_stats *out)
{
    out->volume = h[0] * g->dx * g->dx * g->dx;
    out->S_w = h[1];
    out->S_c = h[2];
    out->S_r = h[3];
    out->phi_min = h[4];
    out->phi_max = h[5];
    out->nonfinite = h[6];
    out->position = h[1] > 0.0 ? h[2] / h[1] : NAN;
    out->radius = h[1] > 0.0 ? h[3] / h[1] : NAN;
    out->energy = energy ? h[7] * g->dx * g->dx * g->dx : NAN;
    out->steps = (double)g->steps;
    out->time = g->time;
}

int check_extent(const spfm_grid_desc *d, size_t px, const char *who)
{
    if ((long long)(d->nx + 2) * (d->ny + 2) >= (1LL << 30) || (long long)(d->nx + 2) * d->nz >= (1LL << 30) ||
        (long long)d->ny * d->nz >= (1LL << 30))
        return fail(nullptr, SPFM_EINVAL, "%s: a face of the grid exceeds 2^30 cells", who);
    if ((long long)px * (d->ny + 2) * (long long)(d->nz + 2) >= (1LL << 40))
        return fail(nullptr, SPFM_EINVAL, "%s: grid too large", who);
    return SPFM_OK;
}

}  // namespace spfm_host

using namespace spfm_host;

extern "C" {

const char *spfm_last_error(const spfm_grid *g)
{
    return g ? g->err.c_str() : t_err.c_str();
}

spfm_status spfm_layout(const spfm_grid_desc *d, size_t *pitch_x, size_t *x_offset,
                        size_t *field_bytes, size_t *scratch_bytes)
{
    if (!d) return fail(nullptr, SPFM_EINVAL, "spfm_layout: desc is NULL");
    if (d->nx < 1 || d->ny < 1 || d->nz < 1)
        return fail(nullptr, SPFM_EINVAL, "spfm_layout: sizes must be >= 1");
    if (d->dtype != SPFM_F64 && d->dtype != SPFM_F32 && d->dtype != SPFM_BF16)
        return fail(nullptr, SPFM_EINVAL, "spfm_layout: unknown dtype %d", d->dtype);
    const size_t es = elem_size(d->dtype), per32 = 32 / es;
    const size_t px = (per32 + d->nx + 1 + per32 - 1) / per32 * per32;
    if (pitch_x) *pitch_x = px;
    if (x_offset) *x_offset = per32;
    if (field_bytes) *field_bytes = px * (size_t)(d->ny + 2) * (size_t)(d->nz + 2) * es;
    if (scratch_bytes) *scratch_bytes = grid_scratch_bytes();
    return SPFM_OK;
}

spfm_status spfm_create_grid(const spfm_grid_desc *d, spfm_grid **out)
{
    if (!out) return fail(nullptr, SPFM_EINVAL, "spfm_create_grid: out is NULL");
    *out = nullptr;
    size_t px = 0, off = 0, fb = 0, sb = 0;
    spfm_status st = spfm_layout(d, &px, &off, &fb, &sb);
    if (st != SPFM_OK) return st;
    st = check_extent(d, px, "spfm_create_grid");
    if (st != SPFM_OK) return st;
    for (int f = 0; f < 6; ++f)
        if (d->bc[f] != SPFM_PERIODIC && d->bc[f] != SPFM_NOFLUX && d->bc[f] != SPFM_CONTACT)
            return fail(nullptr, SPFM_EINVAL, "spfm_create_grid: bad boundary kind on face %d", f);
    for (int ax = 0; ax < 3; ++ax)
        if ((d->bc[2 * ax] == SPFM_PERIODIC) != (d->bc[2 * ax + 1] == SPFM_PERIODIC))
            return fail(nullptr, SPFM_EINVAL, "spfm_create_grid: PERIODIC must be set on both faces of axis %d", ax);
    const double nn = d->n[0] * d->n[0] + d->n[1] * d->n[1] + d->n[2] * d->n[2];
    if (!(fabs(nn - 1.0) < 1e-9))
        return fail(nullptr, SPFM_EINVAL, "spfm_create_grid: |n| = %g, must be 1", sqrt(nn));
    const double uu = d->u[0] * d->u[0] + d->u[1] * d->u[1] + d->u[2] * d->u[2];
    if (!(uu == 0.0 || fabs(uu - 1.0) < 1e-9))
        return fail(nullptr, SPFM_EINVAL, "spfm_create_grid: |u| = %g, must be 0 (u = n) or 1", sqrt(uu));
    for (int b = 0; b < 2; ++b)
        if (!d->field[b] || ((uintptr_t)d->field[b] & 15))
            return fail(nullptr, SPFM_EINVAL, "spfm_create_grid: field[%d] NULL or not 16-byte aligned", b);
    if (d->field[0] == d->field[1])
        return fail(nullptr, SPFM_EINVAL, "spfm_create_grid: the two field buffers must differ");
    if (!d->scratch || ((uintptr_t)d->scratch & 15) || d->scratch_bytes < sb)
        return fail(nullptr, SPFM_ENOMEM, "spfm_create_grid: scratch NULL, unaligned or below %zu bytes", sb);
    if (d->C_gamma < 0.0 || d->gamma[0] < 0.0 || d->gamma[1] < 0.0 || d->gamma[2] < 0.0)
        return fail(nullptr, SPFM_EINVAL, "spfm_create_grid: negative gamma or C_gamma");
    spfm_grid *g = new spfm_grid();
    memset(&g->tma, 0, sizeof g->tma);
    g->d = *d;
    g->elem = elem_size(d->dtype);
    g->geom.nx = d->nx;
    g->geom.ny = d->ny;
    g->geom.nz = d->nz;
    g->geom.pitch = (int)px;
    g->geom.off = (int)off;
    g->geom.plane = (long long)px * (d->ny + 2);
    for (int f = 0; f < 6; ++f) g->geom.bc[f] = d->bc[f];
    *out = g;
    return SPFM_OK;
}

spfm_status spfm_destroy_grid(spfm_grid *g)
{
    delete g;
    return SPFM_OK;
}

spfm_status spfm_set_stream(spfm_grid *g, void *stream)
{
    if (!g) return fail(nullptr, SPFM_EINVAL, "spfm_set_stream: grid is NULL");
    g->d.stream = stream;
    return SPFM_OK;
}

spfm_status spfm_debug_skip_copy(spfm_grid *g)
{
    if (!g) return fail(nullptr, SPFM_EINVAL, "spfm_debug_skip_copy: grid is NULL");
    g->skip_copy = true;
    return SPFM_OK;
}

spfm_status spfm_set_rounding(spfm_grid *g, int mode, unsigned long long seed)
{
    if (!g) return fail(nullptr, SPFM_EINVAL, "spfm_set_rounding: grid is NULL");
    if (mode != SPFM_ROUND_NEAREST && mode != SPFM_ROUND_STOCHASTIC)
        return fail(g, SPFM_EINVAL, "spfm_set_rounding: unknown mode %d", mode);
    if (mode == SPFM_ROUND_STOCHASTIC && g->d.dtype == SPFM_F64)
        return fail(g, SPFM_EINVAL, "spfm_set_rounding: stochastic rounding is for FP32 and BF16 storage");
    g->rounding = mode;
    g->sr_seed = sr_seed_mix(seed);
    return SPFM_OK;
}

spfm_status spfm_set_zchunk(spfm_grid *g, int zchunk)
{
    if (!g) return fail(nullptr, SPFM_EINVAL, "spfm_set_zchunk: grid is NULL");
    if (zchunk < 0) return fail(g, SPFM_EINVAL, "spfm_set_zchunk: zchunk %d < 0", zchunk);
    g->zchunk = zchunk;
    return SPFM_OK;
}

int spfm_last_zchunk(const spfm_grid *g) { return g ? g->last_zchunk : -1; }

int spfm_current(const spfm_grid *g) { return g ? g->cur : -1; }

int spfm_kernels_per_step(const spfm_grid *g)
{
    return g ? ((writes_own_images(g) || faces_inline(g)) ? 1 : 2) : -1;
}

static spfm_status init_common(spfm_grid *g, InitArgs &a, double lambda, double dx)
{
    if (!(lambda > 0.0) || !(dx > 0.0))
        return fail(g, SPFM_EINVAL, "spfm_init: lambda and dx must be > 0");
    a.g = g->geom;
    a.dtype = g->d.dtype;
    a.lambda = lambda;
    a.dx = dx;
    g->cur = 0;
    cudaError_t e = launch_init(a, g->d.field[0], stream_of(g));
    if (e == cudaSuccess) e = cudaMemsetAsync(err_word(g), 0, sizeof(int), stream_of(g));
    if (e != cudaSuccess) return cuda_fail(g, e, "spfm_init");
    g->steps = 0;
    g->time = 0.0;
    g->lambda = lambda;
    g->dx = dx;
    return refresh_ghosts(g, lambda, dx);
}

spfm_status spfm_init_planar(spfm_grid *g, double c, double lambda, double dx)
{
    if (!g) return fail(nullptr, SPFM_EINVAL, "spfm_init_planar: grid is NULL");
    InitArgs a;
    memset(&a, 0, sizeof a);
    for (int i = 0; i < 3; ++i) a.n[i] = g->d.n[i];
    a.c = c;
    return init_common(g, a, lambda, dx);
}

spfm_status spfm_init_sphere(spfm_grid *g, const double ctr[3], double R, double lambda, double dx)
{
    if (!g || !ctr) return fail(g, SPFM_EINVAL, "spfm_init_sphere: NULL argument");
    InitArgs a;
    memset(&a, 0, sizeof a);
    a.shape = 1;
    for (int i = 0; i < 3; ++i) { a.ctr[i] = ctr[i]; g->d.center[i] = ctr[i]; }
    a.R = R;
    return init_common(g, a, lambda, dx);
}

spfm_status spfm_init_cube(spfm_grid *g, const double ctr[3], double half, double lambda, double dx)
{
    if (!g || !ctr) return fail(g, SPFM_EINVAL, "spfm_init_cube: NULL argument");
    if (!(half > 0.0)) return fail(g, SPFM_EINVAL, "spfm_init_cube: half side must be > 0");
    InitArgs a;
    memset(&a, 0, sizeof a);
    a.shape = 2;
    for (int i = 0; i < 3; ++i) { a.ctr[i] = ctr[i]; g->d.center[i] = ctr[i]; }
    a.half = half;
    return init_common(g, a, lambda, dx);
}

spfm_status spfm_step(spfm_grid *g, int n_steps, double M, double Gamma, double lambda, double dx,
                      double dt, double dF, int stencil, int scheme)
{
    if (!g) return fail(nullptr, SPFM_EINVAL, "spfm_step: grid is NULL");
    if (n_steps < 0) return fail(g, SPFM_EINVAL, "spfm_step: n_steps < 0");
    Model m;
    spfm_status st = build_model(g, M, Gamma, lambda, dx, dt, dF, stencil, scheme, m);
    if (st != SPFM_OK) return st;
    LaunchCfg cfg{stencil, scheme, 0};
    cfg.zchunk = g->zchunk;
    cfg.zchunk_used = &g->last_zchunk;
    cudaStream_t s = stream_of(g);
    // no periodic face: the step kernel computes the ghosts of the faces as it
    // reads them, and no face kernel runs (the ghost layer in memory is not used)
    const bool inline_faces = faces_inline(g);
    if (n_steps > 0 && !inline_faces && (g->ghosts_dirty || g->ghost_lambda != lambda || g->ghost_dx != dx)) {
        st = refresh_ghosts(g, lambda, dx);
        if (st != SPFM_OK) return st;
    }
    // all faces periodic and rows of whole 32-byte sectors: each step writes the
    // periodic images of its new cells, and no face kernel runs between steps
    const bool images = writes_own_images(g);
    const bool face_kernel = !images && !inline_faces;
    const int skip = g->skip_copy && n_steps > 0 ? kSkipCopy : 0;
    g->skip_copy = g->skip_copy && n_steps == 0;
    auto mode_of = [&](int i) {
        const int m = images ? kWaitAll | kImages : (inline_faces ? kWaitAll | kEarly : (i == 0 ? kWaitAll : kWaitFaces));
        return m | (i == 0 ? skip : 0);
    };
    int *err = err_word(g);
    if (g->d.dtype == SPFM_F64) {
        StepCoef<double> c;
        fill_coef<double>(g, m, dt, stencil, c);
        set_local_coef<double>(c, lambda, dx);
        for (int i = 0; i < n_steps; ++i) {
            cfg.mode = mode_of(i);
            cudaError_t e = launch_step_f64(c, (const double *)g->d.field[g->cur],
                                            (double *)g->d.field[1 - g->cur], err, cfg, &g->tma,
                                            g->cur, s);
            if (e == cudaSuccess && face_kernel)
                e = launch_fill_ghosts(g->geom, g->d.dtype, m.aface, g->d.field[1 - g->cur], s, 1);
            if (e != cudaSuccess) return cuda_fail(g, e, "spfm_step");
            g->cur ^= 1;
        }
    } else {
        StepCoef<float> c;
        fill_coef<float>(g, m, dt, stencil, c);
        set_local_coef<float>(c, lambda, dx);
        cfg.rounding = g->rounding;
        for (int i = 0; i < n_steps; ++i) {
            cfg.mode = mode_of(i);
            // the step's key of the stochastic rounding: seed and the grid's step count
            c.sr_key = sr_step_key(g->sr_seed, g->steps + i);
            cudaError_t e;
            if (g->d.dtype == SPFM_F32)
                e = launch_step_f32(c, (const float *)g->d.field[g->cur], (float *)g->d.field[1 - g->cur],
                                    err, cfg, &g->tma, g->cur, s);
            else
                e = launch_step_bf16(c, (const __nv_bfloat16 *)g->d.field[g->cur],
                                     (__nv_bfloat16 *)g->d.field[1 - g->cur], err, cfg, &g->tma,
                                     g->cur, s);
            if (e == cudaSuccess && face_kernel)
                e = launch_fill_ghosts(g->geom, g->d.dtype, m.aface, g->d.field[1 - g->cur], s, 1);
            if (e != cudaSuccess) return cuda_fail(g, e, "spfm_step");
            g->cur ^= 1;
        }
    }
    if (inline_faces && n_steps > 0) g->ghosts_dirty = true;   // the ghost layer in memory is stale
    g->steps += n_steps;
    g->time += n_steps * dt;
    g->M = M;
    g->Gamma = Gamma;
    g->lambda = lambda;
    g->dx = dx;
    g->dF = dF;
    g->stencil = stencil;
    g->scheme = scheme;
    return SPFM_OK;
}

spfm_status spfm_step_conserving(spfm_grid *g, int n_steps, double M, double Gamma, double lambda, double dx,
                                 double dt, int stencil, int scheme, double *dF_last)
{
    if (!g) return fail(nullptr, SPFM_EINVAL, "spfm_step_conserving: grid is NULL");
    if (n_steps < 0) return fail(g, SPFM_EINVAL, "spfm_step_conserving: n_steps < 0");
    if (scheme == SPFM_FD_H5 || scheme == SPFM_FD_HABEL)
        return fail(g, SPFM_EINVAL, "spfm_step_conserving: the volume correction uses h3 (TI, TI_n or CF + h3)");
    Model m;
    spfm_status st = build_model(g, M, Gamma, lambda, dx, dt, 0.0, stencil, scheme, m);
    if (st != SPFM_OK) return st;
    LaunchCfg cfg{stencil, scheme, 0};
    cfg.zchunk = g->zchunk;
    cfg.zchunk_used = &g->last_zchunk;
    cudaStream_t s = stream_of(g);
    if (n_steps > 0 && (g->ghosts_dirty || g->ghost_lambda != lambda || g->ghost_dx != dx)) {
        st = refresh_ghosts(g, lambda, dx);
        if (st != SPFM_OK) return st;
    }
    int *err = err_word(g);
    double *partials = (double *)g->d.scratch;
    double *alpha = (double *)((char *)g->d.scratch + scratch_final_offset());
    StepCoef<double> cd;
    StepCoef<float> cf;
    if (g->d.dtype == SPFM_F64) {
        fill_coef<double>(g, m, dt, stencil, cd);
        set_local_coef<double>(cd, lambda, dx);
    } else {
        fill_coef<float>(g, m, dt, stencil, cf);
        set_local_coef<float>(cf, lambda, dx);
        cfg.rounding = g->rounding;
    }
    for (int i = 0; i < n_steps; ++i) {
        void *src = g->d.field[g->cur], *dst = g->d.field[1 - g->cur];
        cfg.mode = i == 0 ? kWaitAll : kWaitFaces;   // the face kernel follows the correction
        cf.sr_key = sr_step_key(g->sr_seed, g->steps + i);
        cudaError_t e;
        if (g->d.dtype == SPFM_F64)
            e = launch_step_f64(cd, (const double *)src, (double *)dst, err, cfg, &g->tma, g->cur, s);
        else if (g->d.dtype == SPFM_F32)
            e = launch_step_f32(cf, (const float *)src, (float *)dst, err, cfg, &g->tma, g->cur, s);
        else
            e = launch_step_bf16(cf, (const __nv_bfloat16 *)src, (__nv_bfloat16 *)dst, err, cfg, &g->tma,
                                 g->cur, s);
        if (e == cudaSuccess) e = launch_conserve(g->geom, g->d.dtype, src, dst, partials, alpha, s);
        if (e == cudaSuccess) e = launch_fill_ghosts(g->geom, g->d.dtype, m.aface, dst, s, 1);
        if (e != cudaSuccess) return cuda_fail(g, e, "spfm_step_conserving");
        g->cur ^= 1;
    }
    g->steps += n_steps;
    g->time += n_steps * dt;
    g->M = M;
    g->Gamma = Gamma;
    g->lambda = lambda;
    g->dx = dx;
    g->dF = 0.0;
    g->stencil = stencil;
    g->scheme = scheme;
    if (dF_last) {
        *dF_last = 0.0;
        if (n_steps > 0) {
            double a = 0.0;
            cudaError_t e = cudaMemcpyAsync(&a, alpha, sizeof a, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return cuda_fail(g, e, "spfm_step_conserving");
            *dF_last = a * lambda * Gamma / (4.0 * M * dt);
        }
    }
    return SPFM_OK;
}

spfm_status spfm_interface_stats(spfm_grid *g, int flags, spfm_stats *out)
{
    if (!g || !out) return fail(g, SPFM_EINVAL, "spfm_interface_stats: NULL argument");
    if (!(g->lambda > 0.0)) return fail(g, SPFM_EINVAL, "spfm_interface_stats: no model yet (init or step first)");
    StatsArgs a;
    fill_stats_args(g, flags, a);
    if (a.energy && (g->ghosts_dirty || g->ghost_lambda != g->lambda || g->ghost_dx != g->dx)) {
        spfm_status st = refresh_ghosts(g, g->lambda, g->dx);
        if (st != SPFM_OK) return st;
    }
    double *partials = (double *)g->d.scratch;
    double *fin = (double *)((char *)g->d.scratch + scratch_final_offset());
    cudaStream_t s = stream_of(g);
    cudaError_t e = launch_stats(a, g->d.field[g->cur], partials, fin, s);
    if (e != cudaSuccess) return cuda_fail(g, e, "spfm_interface_stats");
    double h[kNStat + 1];   // the reduction, then the error word
    e = cudaMemcpyAsync(h, fin, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(g, e, "spfm_interface_stats");
    int errw;
    memcpy(&errw, &h[kNStat], sizeof errw);
    stats_from_reduction(g, h, a.energy, out);
    if (errw != 0)
        return fail(g, SPFM_ETIMEOUT, "a bounded wait in the step kernel gave up (code %d)", errw);
    if (h[6] > 0.0) return fail(g, SPFM_ENONFINITE, "field holds %.0f non-finite cells", h[6]);
    return SPFM_OK;
}

static spfm_status copy_field(spfm_grid *g, void *host_or_dev, int on_host, int to_grid)
{
    const size_t es = g->elem;
    cudaMemcpy3DParms p;
    memset(&p, 0, sizeof p);
    const cudaPitchedPtr grid_ptr =
        make_cudaPitchedPtr(g->d.field[g->cur], (size_t)g->geom.pitch * es, (size_t)g->geom.pitch * es,
                            (size_t)g->d.ny + 2);
    const cudaPitchedPtr dense_ptr =
        make_cudaPitchedPtr(host_or_dev, (size_t)g->d.nx * es, (size_t)g->d.nx * es, (size_t)g->d.ny);
    const cudaPos interior = make_cudaPos((size_t)g->geom.off * es, 1, 1);
    p.extent = make_cudaExtent((size_t)g->d.nx * es, (size_t)g->d.ny, (size_t)g->d.nz);
    if (to_grid) {
        p.srcPtr = dense_ptr;
        p.dstPtr = grid_ptr;
        p.dstPos = interior;
        p.kind = on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    } else {
        p.srcPtr = grid_ptr;
        p.srcPos = interior;
        p.dstPtr = dense_ptr;
        p.kind = on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    }
    cudaStream_t s = stream_of(g);
    cudaError_t e = cudaMemcpy3DAsync(&p, s);
    if (e == cudaSuccess && on_host) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(g, e, to_grid ? "spfm_set_field" : "spfm_get_field");
    return SPFM_OK;
}

spfm_status spfm_get_field(spfm_grid *g, void *dst, int dst_on_host)
{
    if (!g || !dst) return fail(g, SPFM_EINVAL, "spfm_get_field: NULL argument");
    return copy_field(g, dst, dst_on_host, 0);
}

spfm_status spfm_shift_x(spfm_grid *g, int cells)
{
    if (!g) return fail(nullptr, SPFM_EINVAL, "spfm_shift_x: grid is NULL");
    if (cells == 0) return SPFM_OK;
    cudaError_t e = launch_shift_x(g->geom, g->d.dtype, g->d.field[g->cur], g->d.field[1 - g->cur], cells,
                                   stream_of(g));
    if (e != cudaSuccess) return cuda_fail(g, e, "spfm_shift_x");
    g->cur ^= 1;
    g->ghosts_dirty = true;
    if (g->lambda > 0.0) return refresh_ghosts(g, g->lambda, g->dx);
    return SPFM_OK;
}

spfm_status spfm_max_dt(spfm_grid *g, double M, double Gamma, double lambda, double dx, double dF, int stencil,
                        int scheme, double *dt_max)
{
    if (!g || !dt_max) return fail(g, SPFM_EINVAL, "spfm_max_dt: NULL argument");
    Model m;
    const spfm_status st = build_model(g, M, Gamma, lambda, dx, 1e-300, dF, stencil, scheme, m);
    if (st != SPFM_OK) return st;
    *dt_max = 2.0 / m.bound;
    return SPFM_OK;
}

spfm_status spfm_set_field(spfm_grid *g, const void *src, int src_on_host)
{
    if (!g || !src) return fail(g, SPFM_EINVAL, "spfm_set_field: NULL argument");
    spfm_status st = copy_field(g, const_cast<void *>(src), src_on_host, 1);
    if (st != SPFM_OK) return st;
    g->steps = 0;
    g->time = 0.0;
    g->ghosts_dirty = true;   // refilled by the next step, or now when lambda is known
    cudaError_t e = cudaMemsetAsync(err_word(g), 0, sizeof(int), stream_of(g));
    if (e != cudaSuccess) return cuda_fail(g, e, "spfm_set_field");
    if (g->lambda > 0.0) return refresh_ghosts(g, g->lambda, g->dx);
    return SPFM_OK;
}

}  // extern "C"
