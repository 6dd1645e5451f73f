/*
 * spfm_oracle.c -- FP64 CPU oracle of the sharp phase-field method.
 *
 * TEST INFRASTRUCTURE ONLY (see spfm_oracle.h): the test suite, the smoke
 * check and the benchmark's CPU-baseline leg are its only users.  Everything
 * here is written straight from the paper's definitions, cell by cell and
 * direction by direction, with no blocking, grouping or reordering:
 *
 *   Eq. 1  discrete free-energy density
 *          f_p = Gamma/(C_Gamma lambda) sum_k gamma_j nu_j
 *                ( lambda^2/2 (d+_k phi_p)^2 + g_k(phi_p) ) + dF h(phi_p)
 *   Eq. 2  3 lambda Gamma dphi/dt = -2 M dF/dphi   (Allen-Cahn relaxation)
 *          with dF/dphi_p = df/dphi_p - sum_k d-_k (df/d(d+_k phi))
 *   Eq. 3  ideal profile phi = (1 - tanh(2 (p.n - c)/lambda))/2
 *   Eq. 5  grid coupling a_k(n) = tanh(2 r_k.n / lambda)
 *   Eq. 6  TI potential g_k r_k^2/lambda^2 = q + (1-a^2)/(4a^2) ln((1-a^2)/(1-a^2 s^2))
 *   Eq. 7  contact-angle boundary value (1-a) phi_s / (1 - a (2 phi_s - 1))
 *   Sec. 2.3  nonlinear contour interpolation (Eqs. 8-10)
 *
 * with q = phi(1-phi) and s = 1 - 2 phi.  Readings where the paper is silent
 * or garbled (each is pinned by a test):
 *   - the backward difference of Eq. 2 is taken as the true variational
 *     derivative of F = sum_p f_p dx^3, which yields +Laplacian - g'
 *     (the form of the equilibrium condition, Eq. 4);
 *   - nu_j = 3/m_j with m_j the number of directions of shell j (3, 6, 4);
 *   - the CF potential is 8 phi^2 (1-phi)^2 / 3 per direction (Tab. 2);
 *   - default ponderations gamma = (1,0,0), (1/3,2/3,0), (1/2,1/3,1/6) for 6, 18,
 *     26 neighbours (fourth-order isotropy of the discrete Laplacian), and
 *     C_Gamma = 2/3 (interface energy Gamma in the continuum limit);
 *   - forward Euler in time; the driving term uses h3 = phi^2 (3 - 2 phi),
 *     or, for the CF variants of Tab. 2, h5 or h_Abel;
 *   - NOFLUX ghost = copy of the adjacent interior cell; CONTACT ghost by
 *     Eq. 7 with the signed a = tanh(2 (x_ghost - x_source).n / lambda);
 *   - TI_n: n = grad psi / |grad psi| with psi = (lambda/2) artanh(1 - 2 phi),
 *     phi clamped to [eps, 1-eps], central differences; where |grad psi| <
 *     1e-8 the cell falls back to the CF potential.
 */
#include "spfm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Tab. 1: one grid vector per +/- pair, k = 0..12, shells 1..3. */
static const int DIRS[13][3] = {
    {1, 0, 0},  {0, 1, 0},  {0, 0, 1},                               /* shell 1 */
    {1, 1, 0},  {0, 1, 1},  {1, 0, 1},  {1, -1, 0}, {0, 1, -1}, {1, 0, -1},  /* shell 2 */
    {1, 1, 1},  {-1, 1, 1}, {1, -1, 1}, {1, 1, -1}                   /* shell 3 */
};
static const int SHELL[13] = {1, 1, 1, 2, 2, 2, 2, 2, 2, 3, 3, 3, 3};

int oracle_directions(int *out_d, int *out_shell)
{
    for (int k = 0; k < 13; ++k) {
        for (int c = 0; c < 3; ++c) out_d[3 * k + c] = DIRS[k][c];
        out_shell[k] = SHELL[k];
    }
    return 13;
}

static int n_dirs(int stencil)
{
    return stencil == 6 ? 3 : stencil == 18 ? 9 : 13;
}

static double c_gamma_of(const orc_params *p)
{
    return p->C_gamma > 0.0 ? p->C_gamma : 2.0 / 3.0;
}

int oracle_weights(const orc_params *p, double *w, double *gam)
{
    double g[3] = {p->gamma[0], p->gamma[1], p->gamma[2]};
    if (g[0] == 0.0 && g[1] == 0.0 && g[2] == 0.0) {
        if (p->stencil == 6) { g[0] = 1.0; }
        else if (p->stencil == 18) { g[0] = 1.0 / 3.0; g[1] = 2.0 / 3.0; }
        else { g[0] = 0.5; g[1] = 1.0 / 3.0; g[2] = 1.0 / 6.0; }
    }
    /* nu_j = 3 / m_j, m_j = number of directions in shell j */
    const double nu[3] = {3.0 / 3.0, 3.0 / 6.0, 3.0 / 4.0};
    int nd = n_dirs(p->stencil);
    for (int k = 0; k < 13; ++k) {
        int j = SHELL[k] - 1;
        w[k] = (k < nd) ? g[j] * nu[j] : 0.0;
    }
    if (gam) { gam[0] = g[0]; gam[1] = g[1]; gam[2] = g[2]; }
    return nd;
}

void oracle_coupling(const double u[3], double lambda, double dx, double *a)
{
    for (int k = 0; k < 13; ++k) {
        double rdotu = dx * (DIRS[k][0] * u[0] + DIRS[k][1] * u[1] + DIRS[k][2] * u[2]);
        a[k] = tanh(2.0 * rdotu / lambda);
    }
}

void oracle_init_planar(double *phi, int nx, int ny, int nz, const double n[3],
                        double c, double lambda, double dx)
{
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double pn = dx * (i * n[0] + j * n[1] + k * n[2]);
                phi[((size_t)k * ny + j) * nx + i] = 0.5 * (1.0 - tanh(2.0 * (pn - c) / lambda));
            }
}

void oracle_init_sphere(double *phi, int nx, int ny, int nz, const double ctr[3],
                        double R, double lambda, double dx)
{
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double x = dx * i - ctr[0], y = dx * j - ctr[1], z = dx * k - ctr[2];
                double r = sqrt(x * x + y * y + z * z);
                phi[((size_t)k * ny + j) * nx + i] = 0.5 * (1.0 - tanh(2.0 * (R - r) / lambda));
            }
}

void oracle_init_cube(double *phi, int nx, int ny, int nz, const double ctr[3], double half,
                      double lambda, double dx)
{
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const double d[3] = {dx * i - ctr[0], dx * j - ctr[1], dx * k - ctr[2]};
                double inside = 1.0;   /* product of the three 1D particle fractions */
                for (int a = 0; a < 3; ++a)
                    inside *= 0.5 * (1.0 - tanh(2.0 * (fabs(d[a]) - half) / lambda));
                phi[((size_t)k * ny + j) * nx + i] = 1.0 - inside;
            }
}

void oracle_shift_x(double *phi, int nx, int ny, int nz, int cells)
{
    double *row = (double *)malloc(sizeof(double) * (size_t)nx);
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j) {
            double *r = phi + ((size_t)k * ny + j) * nx;
            for (int i = 0; i < nx; ++i) {
                int src = i + cells;
                if (src < 0) src = 0;
                if (src > nx - 1) src = nx - 1;
                row[i] = r[src];
            }
            memcpy(r, row, sizeof(double) * (size_t)nx);
        }
    free(row);
}

/* ---------------------------------------------------------------- ghosts */

#define PADX(p) ((p)->nx + 2)
#define PADY(p) ((p)->ny + 2)
#define PIDX(p, i, j, k) ((((size_t)(k) + 1) * PADY(p) + ((j) + 1)) * PADX(p) + ((i) + 1))

/* Eq. 7 with a signed coupling: value at a ghost displaced by delta (a grid
 * vector) from its source cell. */
static double contact_value(double phi_s, const double n[3], const double delta[3],
                            double lambda)
{
    double a = tanh(2.0 * (delta[0] * n[0] + delta[1] * n[1] + delta[2] * n[2]) / lambda);
    return (1.0 - a) * phi_s / (1.0 - a * (2.0 * phi_s - 1.0));
}

/* ghost value on face `face` (0..5) given the source value and kind */
static double ghost_from(const orc_params *p, int face, double src_val)
{
    int axis = face / 2;
    double delta[3] = {0.0, 0.0, 0.0};
    delta[axis] = (face % 2 == 0) ? -p->dx : p->dx;
    if (p->bc[face] == ORC_CONTACT) return contact_value(src_val, p->n, delta, p->lambda);
    return src_val;
}

void oracle_fill_ghosts(const orc_params *p, const double *phi, double *pad)
{
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i)
                pad[PIDX(p, i, j, k)] = phi[((size_t)k * ny + j) * nx + i];
    /* x faces over interior y, z */
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j) {
            int s_lo = (p->bc[0] == ORC_PERIODIC) ? nx - 1 : 0;
            int s_hi = (p->bc[1] == ORC_PERIODIC) ? 0 : nx - 1;
            pad[PIDX(p, -1, j, k)] = ghost_from(p, 0, pad[PIDX(p, s_lo, j, k)]);
            pad[PIDX(p, nx, j, k)] = ghost_from(p, 1, pad[PIDX(p, s_hi, j, k)]);
        }
    /* y faces over x in [-1, nx], interior z */
    for (int k = 0; k < nz; ++k)
        for (int i = -1; i <= nx; ++i) {
            int s_lo = (p->bc[2] == ORC_PERIODIC) ? ny - 1 : 0;
            int s_hi = (p->bc[3] == ORC_PERIODIC) ? 0 : ny - 1;
            pad[PIDX(p, i, -1, k)] = ghost_from(p, 2, pad[PIDX(p, i, s_lo, k)]);
            pad[PIDX(p, i, ny, k)] = ghost_from(p, 3, pad[PIDX(p, i, s_hi, k)]);
        }
    /* z faces over x in [-1, nx], y in [-1, ny] */
    for (int j = -1; j <= ny; ++j)
        for (int i = -1; i <= nx; ++i) {
            int s_lo = (p->bc[4] == ORC_PERIODIC) ? nz - 1 : 0;
            int s_hi = (p->bc[5] == ORC_PERIODIC) ? 0 : nz - 1;
            pad[PIDX(p, i, j, -1)] = ghost_from(p, 4, pad[PIDX(p, i, j, s_lo)]);
            pad[PIDX(p, i, j, nz)] = ghost_from(p, 5, pad[PIDX(p, i, j, s_hi)]);
        }
}

/* ------------------------------------------------------------- model terms */

/* the TI_<hkl> coupling direction u of Eq. 5: p->u when set, else the normal */
static const double *coupling_u(const orc_params *p)
{
    return (p->u[0] != 0.0 || p->u[1] != 0.0 || p->u[2] != 0.0) ? p->u : p->n;
}

/* derivative of h3 = phi^2 (3 - 2 phi) (Sec. 2.1, natural interpolation) */
static double h3_prime(double phi)
{
    return 6.0 * phi * (1.0 - phi);
}

/* Tab. 2: h5 = phi^3 (10 - 15 phi + 6 phi^2) and
 * h_Abel = phi^2 / (phi^2 + (1 - phi)^2), differentiated by hand */
static double h5_prime(double phi)
{
    return 30.0 * phi * phi * (1.0 - phi) * (1.0 - phi);
}

static double habel_prime(double phi)
{
    const double d = phi * phi + (1.0 - phi) * (1.0 - phi);
    return 2.0 * phi * (1.0 - phi) / (d * d);
}

/* the interpolation function of the scheme: h5 and h_Abel belong to CF models
 * only (Tab. 2); every other scheme uses h3 */
static double h_prime(const orc_params *p, double phi)
{
    if (p->scheme == ORC_CF_H5) return h5_prime(phi);
    if (p->scheme == ORC_CF_HABEL) return habel_prime(phi);
    return h3_prime(phi);
}

static int is_cf(const orc_params *p)
{
    return p->scheme == ORC_CF || p->scheme == ORC_CF_H5 || p->scheme == ORC_CF_HABEL;
}

/* derivative of the TI potential of Eq. 6 w.r.t. phi, multiplied out:
 * g'_k = (lambda^2/r^2) 4 a^2 q s / (1 - a^2 s^2).  *bad set when the
 * denominator is not positive. */
static double g_ti_prime(double phi, double a, double lam2_over_r2, int *bad)
{
    double q = phi * (1.0 - phi), s = 1.0 - 2.0 * phi;
    double den = 1.0 - a * a * s * s;
    if (!(den > 0.0)) { *bad = 1; return NAN; }
    return lam2_over_r2 * 4.0 * a * a * q * s / den;
}

/* Eq. 6 itself (energy diagnostics); series 2 a^2 q^2 for tiny a */
static double g_ti(double phi, double a, double lam2_over_r2)
{
    double q = phi * (1.0 - phi), s = 1.0 - 2.0 * phi, A = a * a;
    if (A < 1e-8) return lam2_over_r2 * 2.0 * A * q * q;
    return lam2_over_r2 * (q + (1.0 - A) / (4.0 * A) * log((1.0 - A) / (1.0 - A * s * s)));
}

/* CF quartic double well per direction, 8 phi^2 (1-phi)^2 / 3 (Tab. 2) */
static double g_cf(double phi)
{
    return 8.0 * phi * phi * (1.0 - phi) * (1.0 - phi) / 3.0;
}

static double g_cf_prime(double phi)
{
    return 16.0 * phi * (1.0 - phi) * (1.0 - 2.0 * phi) / 3.0;
}

static double eps_of(const orc_params *p)
{
    return p->eps_local > 0.0 ? p->eps_local : 1e-6;
}

/* TI_n: local coupling parameters at padded index c.  Returns 0 and fills a[]
 * when the normal is defined, 1 when the cell falls back to CF. */
static int local_coupling(const orc_params *p, const double *pad, size_t c, double *a)
{
    const double eps = eps_of(p);
    const size_t sx = 1, sy = PADX(p), sz = (size_t)PADX(p) * PADY(p);
    const size_t off[3] = {sx, sy, sz};
    double g[3];
    for (int ax = 0; ax < 3; ++ax) {
        double pp = pad[c + off[ax]], pm = pad[c - off[ax]];
        pp = pp < eps ? eps : (pp > 1.0 - eps ? 1.0 - eps : pp);
        pm = pm < eps ? eps : (pm > 1.0 - eps ? 1.0 - eps : pm);
        double psi_p = 0.5 * p->lambda * atanh(1.0 - 2.0 * pp);
        double psi_m = 0.5 * p->lambda * atanh(1.0 - 2.0 * pm);
        g[ax] = (psi_p - psi_m) / (2.0 * p->dx);
    }
    double norm = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    if (!(norm >= 1e-8)) return 1;
    double n[3] = {g[0] / norm, g[1] / norm, g[2] / norm};
    oracle_coupling(n, p->lambda, p->dx, a);
    return 0;
}

/* ------------------------------------------------------------------- RHS */

long oracle_rhs(const orc_params *p, const double *phi, double *R)
{
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    double w[13];
    int nd = oracle_weights(p, w, NULL);
    const double Cg = c_gamma_of(p);
    const double lam = p->lambda, dx = p->dx;
    double a_glob[13];
    oracle_coupling(coupling_u(p), lam, dx, a_glob);

    double *pad = (double *)malloc(sizeof(double) * (size_t)PADX(p) * PADY(p) * (nz + 2));
    oracle_fill_ghosts(p, phi, pad);

    /* Eq. 2 with Eq. 1: dphi/dt = -(2M/(3 lambda Gamma)) dF/dphi, where
     * dF/dphi = Gamma/(C_Gamma lambda) sum_k w_k [ g'_k - lambda^2/r^2 lap_k ] + dF h' */
    const double pref = 2.0 * p->M / (3.0 * lam * p->Gamma);
    const double pref_int = p->Gamma / (Cg * lam);
    long nbad = 0;

#pragma omp parallel for reduction(+ : nbad) schedule(static)
    for (int k = 0; k < nz; ++k) {
        double a_loc[13];
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t c = PIDX(p, i, j, k);
                double ph = pad[c];
                const double *a = a_glob;
                int use_cf = is_cf(p);
                if (p->scheme == ORC_TI_LOCAL) {
                    use_cf = local_coupling(p, pad, c, a_loc);
                    a = a_loc;
                }
                double dFdphi_int = 0.0;
                int bad = 0;
                for (int kk = 0; kk < nd; ++kk) {
                    long off = (long)DIRS[kk][0] + (long)DIRS[kk][1] * PADX(p) +
                               (long)DIRS[kk][2] * (long)PADX(p) * PADY(p);
                    double r2 = (double)SHELL[kk] * dx * dx;
                    double lap = pad[c + off] + pad[c - off] - 2.0 * ph;
                    double gp = use_cf ? g_cf_prime(ph) : g_ti_prime(ph, a[kk], lam * lam / r2, &bad);
                    dFdphi_int += w[kk] * (gp - lam * lam / r2 * lap);
                }
                double dFdphi = pref_int * dFdphi_int + p->dF * h_prime(p, ph);
                R[((size_t)k * ny + j) * nx + i] = -pref * dFdphi;
                nbad += bad;
            }
    }
    free(pad);
    return nbad;
}

long oracle_step(const orc_params *p, double *phi, int n_steps)
{
    size_t n = (size_t)p->nx * p->ny * p->nz;
    double *R = (double *)malloc(sizeof(double) * n);
    long nbad = 0;
    for (int s = 0; s < n_steps; ++s) {
        nbad += oracle_rhs(p, phi, R);
        for (size_t c = 0; c < n; ++c) phi[c] += p->dt * R[c];
    }
    free(R);
    return nbad;
}

long oracle_step_conserving(const orc_params *p, double *phi, int n_steps, double *dF_out)
{
    size_t n = (size_t)p->nx * p->ny * p->nz;
    double *R = (double *)malloc(sizeof(double) * n);
    orc_params p0 = *p;
    p0.dF = 0.0;
    /* Eq. 2 with Eq. 1: the driving term of dphi/dt is -(2M/(3 lambda Gamma)) dF h3'(phi) */
    const double pref = 2.0 * p->M / (3.0 * p->lambda * p->Gamma);
    long nbad = 0;
    for (int s = 0; s < n_steps; ++s) {
        nbad += oracle_rhs(&p0, phi, R);
        double sum_r = 0.0, sum_h = 0.0;
        for (size_t c = 0; c < n; ++c) {
            sum_r += R[c];
            sum_h += h_prime(p, phi[c]);
        }
        /* the homogeneous dF for which sum_p (R_p - pref dF h3'(phi_p)) = 0 */
        const double dF = sum_h != 0.0 ? sum_r / (pref * sum_h) : 0.0;
        for (size_t c = 0; c < n; ++c) phi[c] += p->dt * (R[c] - pref * dF * h_prime(p, phi[c]));
        if (dF_out) dF_out[s] = dF;
    }
    free(R);
    return nbad;
}

/* ------------------------------------------------------------ diagnostics */

void oracle_stats(const orc_params *p, const double *phi, const double ctr[3], double *out)
{
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    const double dx = p->dx, lam = p->lambda;
    double vol = 0.0, sw = 0.0, sc = 0.0, sr = 0.0, mn = INFINITY, mx = -INFINITY, bad = 0.0;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double ph = phi[((size_t)k * ny + j) * nx + i];
                if (!isfinite(ph)) { bad += 1.0; continue; }
                vol += ph;
                if (ph < mn) mn = ph;
                if (ph > mx) mx = ph;
                if (ph > 1e-6 && ph < 1.0 - 1e-6) {
                    double q = ph * (1.0 - ph);
                    double psi = 0.5 * lam * atanh(1.0 - 2.0 * ph);
                    double px = dx * i, py = dx * j, pz = dx * k;
                    double pn = px * p->n[0] + py * p->n[1] + pz * p->n[2];
                    double rx = px - ctr[0], ry = py - ctr[1], rz = pz - ctr[2];
                    double r = sqrt(rx * rx + ry * ry + rz * rz);
                    sw += q;
                    sc += q * (pn - psi);
                    sr += q * (r + psi);
                }
            }
    out[0] = vol * dx * dx * dx;
    out[1] = sw;
    out[2] = sc;
    out[3] = sr;
    out[4] = mn;
    out[5] = mx;
    out[6] = bad;
    out[7] = sw > 0.0 ? sc / sw : NAN;
    out[8] = sw > 0.0 ? sr / sw : NAN;
}

double oracle_energy(const orc_params *p, const double *phi)
{
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    double w[13];
    int nd = oracle_weights(p, w, NULL);
    const double lam = p->lambda, dx = p->dx;
    double a_glob[13];
    oracle_coupling(coupling_u(p), lam, dx, a_glob);
    double *pad = (double *)malloc(sizeof(double) * (size_t)PADX(p) * PADY(p) * (nz + 2));
    oracle_fill_ghosts(p, phi, pad);
    double total = 0.0;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t c = PIDX(p, i, j, k);
                double ph = pad[c];
                const double *a = a_glob;
                double a_loc[13];
                int use_cf = is_cf(p);
                if (p->scheme == ORC_TI_LOCAL) {
                    use_cf = local_coupling(p, pad, c, a_loc);
                    a = a_loc;
                }
                double f = 0.0;
                for (int kk = 0; kk < nd; ++kk) {
                    long off = (long)DIRS[kk][0] + (long)DIRS[kk][1] * PADX(p) +
                               (long)DIRS[kk][2] * (long)PADX(p) * PADY(p);
                    double r2 = (double)SHELL[kk] * dx * dx;
                    double dplus = (pad[c + off] - ph) / sqrt(r2);
                    double g = use_cf ? g_cf(ph) : g_ti(ph, a[kk], lam * lam / r2);
                    f += w[kk] * (0.5 * lam * lam * dplus * dplus + g);
                }
                total += p->Gamma / (c_gamma_of(p) * lam) * f;
            }
    free(pad);
    return total * dx * dx * dx;
}

/* |artanh((l - phi)/(2 l phi - phi - l))| of Eqs. 8-10 */
static double contour_arg(double phi, double l)
{
    double x = (l - phi) / (2.0 * l * phi - phi - l);
    return fabs(atanh(x));
}

long oracle_contour(const orc_params *p, const double *phi, double l, double *pts, long max_pts)
{
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    const double dx = p->dx;
    long np = 0;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double pa = phi[((size_t)k * ny + j) * nx + i];
                for (int ax = 0; ax < 3; ++ax) {
                    int ii = i + (ax == 0), jj = j + (ax == 1), kq = k + (ax == 2);
                    if (ii >= nx || jj >= ny || kq >= nz) continue;
                    double pb = phi[((size_t)kq * ny + jj) * nx + ii];
                    if ((pa < l) == (pb < l)) continue;
                    /* Eq. 10 gives the directional width that makes the two
                     * positions of Eqs. 8 and 9 coincide; both then sit at the
                     * fraction A_a/(A_a + A_b) of the edge from a to b. */
                    double Aa = contour_arg(pa, l), Ab = contour_arg(pb, l);
                    double lam_hat = 2.0 * dx / (Aa + Ab);
                    double xa = dx * (ax == 0 ? i : ax == 1 ? j : k) + 0.5 * lam_hat * Aa;
                    double xb = dx * (ax == 0 ? ii : ax == 1 ? jj : kq) - 0.5 * lam_hat * Ab;
                    if (isinf(Aa) && !isinf(Ab)) { xa = xb = dx * (ax == 0 ? ii : ax == 1 ? jj : kq); }
                    if (isinf(Ab) && !isinf(Aa)) { xa = xb = dx * (ax == 0 ? i : ax == 1 ? j : k); }
                    if (!(Aa + Ab > 0.0)) xa = xb = dx * ((ax == 0 ? i : ax == 1 ? j : k) + 0.5);
                    /* the linear blend of Sec. 2.3, with its division restored */
                    double x = (pb != pa) ? (xb * (l - pa) + xa * (pb - l)) / (pb - pa) : xa;
                    if (np < max_pts) {
                        pts[3 * np + 0] = ax == 0 ? x : dx * i;
                        pts[3 * np + 1] = ax == 1 ? x : dx * j;
                        pts[3 * np + 2] = ax == 2 ? x : dx * k;
                    }
                    ++np;
                }
            }
    return np;
}
