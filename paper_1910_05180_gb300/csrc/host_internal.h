// host_internal.h -- host-side state shared by the C ABI translation units
// (api.cu: single grids, batch.cu: batches): the grid handle, the FP64 model
// coefficients (a1) and the helpers that report errors.
#pragma once

#include <string>

#include "spfm_internal.h"

struct spfm_grid {
    spfm_grid_desc d;
    spfm::GridGeom geom;
    size_t elem;           // bytes per element
    int cur = 0;           // buffer holding the current field
    bool ghosts_dirty = true;          // ghost layer of the current buffer needs a refill
    double ghost_lambda = 0.0, ghost_dx = 0.0;   // model the ghosts were filled with
    spfm::TmaCache tma;                // tensor maps of the two buffers
    long long steps = 0;
    double time = 0.0;
    // model of the last step (stats: energy, estimator)
    double M = 1.0, Gamma = 1.0, lambda = 0.0, dx = 1.0, dF = 0.0;
    int stencil = 26, scheme = SPFM_TI_GLOBAL;
    // rounding of the update (spfm_set_rounding) and the mixed seed of SPFM_ROUND_STOCHASTIC
    int rounding = SPFM_ROUND_NEAREST;
    uint32_t sr_seed = 0;
    bool skip_copy = false;   // spfm_debug_skip_copy: the next step launch skips one copy
    int zchunk = 0;           // spfm_set_zchunk: planes per CTA of the step launches (0: chosen per launch)
    int last_zchunk = 0;      // planes per CTA of the last step launch
    std::string err;
};

namespace spfm_host {

int fail(spfm_grid *g, int code, const char *fmt, ...);
int cuda_fail(spfm_grid *g, cudaError_t e, const char *what);
void set_thread_error(const char *msg);
size_t elem_size(int dtype);
// Extent limits of a grid (every face below 2^30 cells, the padded field below
// 2^40 elements): 0 when they hold, else SPFM_EINVAL with the thread's message
// set (prefixed by `who`).
int check_extent(const spfm_grid_desc *d, size_t pitch_x, const char *who);

// Model coefficients in FP64 (a1).  gamma defaults, nu_j = 3/m_j, c_j, A_k
// grouped by value, stability and phase checks.
struct Model {
    double gamma[3], w[spfm::kMaxTerms], c_shell[3], ck[spfm::kMaxTerms];
    double a[spfm::kMaxTerms];
    int nterms;
    double beta[spfm::kMaxTerms], A[spfm::kMaxTerms];
    double kmu, kappa, D, Cg;
    int interp;     // CF driving term: 0 h3, 1 h5, 2 h_Abel
    double aface[6];
    double bound;   // upper bound of the spectral radius of the Euler Jacobian
};

int n_dirs(int stencil);
void default_gamma(int stencil, const double *given, double *g);
int build_model(spfm_grid *g, double M, double Gamma, double lambda, double dx, double dt,
                double dF, int stencil, int scheme, Model &m);
cudaStream_t stream_of(const spfm_grid *g);
// ghost layer of the current buffer from the interior (face kernel), on st or
// the grid's stream
int refresh_ghosts(spfm_grid *g, double lambda, double dx, cudaStream_t st = nullptr);
int *err_word(const spfm_grid *g);
bool writes_own_images(const spfm_grid *g);
// no periodic face: the step kernels compute the ghosts as they read them, and
// no face kernel runs between steps (the ghost layer in memory goes stale)
bool faces_inline(const spfm_grid *g);
void fill_stats_args(const spfm_grid *g, int flags, spfm::StatsArgs &a);
void stats_from_reduction(const spfm_grid *g, const double *h, int energy, spfm_stats *out);

template <class T>
void fill_coef(const spfm_grid *g, const Model &m, double dt, int stencil, spfm::StepCoef<T> &c)
{
    memset(&c, 0, sizeof c);
    c.g = g->geom;
    for (int f = 0; f < 6; ++f) c.aface[f] = (T)m.aface[f];
    c.c1 = (T)m.c_shell[0];
    c.c2 = (T)m.c_shell[1];
    c.c3 = (T)m.c_shell[2];
    c.dt = (T)dt;
    c.kmu = (T)m.kmu;
    c.kappa = (T)m.kappa;
    c.nterms = m.nterms;
    for (int t = 0; t < spfm::kMaxTerms; ++t) {
        c.beta[t] = t < m.nterms ? (T)m.beta[t] : T(0);
        c.A[t] = t < m.nterms ? (T)m.A[t] : T(0);
        c.ck[t] = (T)m.ck[t];
        c.nbetadt[t] = t < m.nterms ? (T)(-m.beta[t] * dt) : T(0);
    }
    // S1 = F'_z + t, S2 = E'_z + F'_{z-1} + F'_{z+1} + 4t, S3 = E'_{z-1} + E'_{z+1} + 4t
    double ct = m.c_shell[0];
    if (stencil >= 18) ct += 4.0 * m.c_shell[1];
    if (stencil == 26) ct += 4.0 * m.c_shell[2];
    c.c1dt = (T)(m.c_shell[0] * dt);
    c.c2dt = (T)(m.c_shell[1] * dt);
    c.c3dt = (T)(m.c_shell[2] * dt);
    c.ctdt = (T)(ct * dt);
    c.nkmudt = (T)(-m.kmu * dt);
    c.nkapdt = (T)(-m.kappa * dt);
    c.interp = m.interp;
    c.sr_seed = g->sr_seed;
}

// TI_n constants of the step kernels: the gradient scale of the log-odds
// (psi = (lambda/4) ln((1 - phi)/phi); the FP32 kernels take log2), 2 dx/lambda
// and the clamp of phi before the profile inversion (1e-6)
template <class T>
void set_local_coef(spfm::StepCoef<T> &c, double lambda, double dx)
{
    c.psi_grad = (T)(0.25 * lambda * (sizeof(T) == 4 ? 0.69314718055994530942 : 1.0) / (2.0 * dx));
    c.two_dx_over_lam = (T)(2.0 * dx / lambda);
    c.eps = (T)1e-6;
}

}  // namespace spfm_host
