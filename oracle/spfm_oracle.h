/*
 * spfm_oracle.h -- FP64 CPU oracle of the sharp phase-field method (SPFM).
 *
 * TEST INFRASTRUCTURE ONLY.  This header and spfm_oracle.c are a plain, slow,
 * double-precision restatement of the discrete phase-field equations of
 * Fleck, Schleifer, Zimbrod, "Frictionless motion of diffuse interfaces by
 * sharp phase-field modeling" (arXiv:1910.05180).  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  The
 * CUDA library shares no code, header, table or helper with it.
 *
 * Field layout: phi[(k*ny + j)*nx + i], cell centre p = dx*(i, j, k).
 * Padded (ghost) layout: pad[((k+1)*(ny+2) + (j+1))*(nx+2) + (i+1)],
 * i in [-1, nx], j in [-1, ny], k in [-1, nz].
 *
 * Parity status per function (what pins it, see tests/test_oracle_pins.py):
 *   oracle_init_planar      closed form of the tanh profile (Sec. 2.1, Eq. 3)
 *   oracle_fill_ghosts      contact-angle BC exact on the ideal profile (Eq. 7)
 *   oracle_rhs  TI / CF     energy gradient of Eq. 1 (autograd, 4^3 grid),
 *                           fixed point (Eq. 4), exact translation, v_th
 *   oracle_rhs  TI_n        parity unpinned against the paper beyond the
 *                           planar case: the local-normal procedure is only
 *                           referenced, not given (Sec. 2.1, TI_n model)
 *   oracle_stats            exact on the ideal planar and radial profiles
 *   oracle_energy           shift invariance under TI, continuum limit
 *   oracle_contour          exact on planar ideal profiles (Sec. 2.3)
 *   oracle_init_cube        closed form at face centres; a reading (the paper
 *                           gives no cube profile)
 *   oracle_step_conserving  sum phi invariant, zero dF on flat slabs,
 *                           Gibbs-Thomson dF = 2 Gamma / R on a sphere
 */
#ifndef SPFM_ORACLE_H
#define SPFM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* boundary kinds, per face (x-, x+, y-, y+, z-, z+) */
enum { ORC_PERIODIC = 0, ORC_NOFLUX = 1, ORC_CONTACT = 2 };
/* schemes: TI with one global coupling direction, TI with the local normal,
 * conventional continuum-field finite differences (CF + h3) */
enum { ORC_TI_GLOBAL = 0, ORC_TI_LOCAL = 1, ORC_CF = 2,
       /* CF with the interpolation functions h5 and h_Abel of Tab. 2 */
       ORC_CF_H5 = 3, ORC_CF_HABEL = 4 };

/* Shift the field along x by `cells` (phi_i <- phi_{i+cells}), filling the
 * vacated cells with the value of the row's last (first) cell: the moving
 * frame of the 1D friction study (Sec. 3.1), which moves the system back by
 * one grid point whenever the favoured phase fills half of it. */
void oracle_shift_x(double *phi, int nx, int ny, int nz, int cells);

typedef struct {
    int nx, ny, nz;
    int bc[6];
    double n[3];        /* interface normal: contact BC and, unless u is set, the TI coupling direction */
    double gamma[3];    /* shell ponderations; all zero selects the defaults */
    double C_gamma;     /* interface energy calibration; 0 selects 2/3 */
    double M, Gamma, lambda, dx, dt, dF;
    int stencil;        /* 6, 18 or 26 neighbours */
    int scheme;         /* ORC_TI_GLOBAL, ORC_TI_LOCAL, ORC_CF */
    double eps_local;   /* TI_n clamp of phi before inverting the profile; 0 -> 1e-6 */
    double u[3];        /* TI_<hkl> coupling direction (Tab. 2: u || <hkl>); all 0 -> n */
} orc_params;

/* Direction table of Tab. 1: out_d[3*k + c] (integers) and out_shell[k]
 * for k = 0..12.  Returns 13. */
int oracle_directions(int *out_d, int *out_shell);

/* Per-direction weights w_k = gamma_j * nu_j (nu_j = 3/m_j) for the active
 * directions of the stencil (others 0), and the gamma actually used. */
int oracle_weights(const orc_params *p, double *out_w13, double *out_gamma3);

/* Grid coupling parameters a_k(u) = tanh(2 r_k.u / lambda), Eq. 5. */
void oracle_coupling(const double u[3], double lambda, double dx, double *out_a13);

/* Ideal profile phi = (1 - tanh(2 (p.n - c)/lambda))/2 at the cell centres. */
void oracle_init_planar(double *phi, int nx, int ny, int nz, const double n[3],
                        double c, double lambda, double dx);
/* Radial ideal profile of a grain with phi = 0 inside radius R around ctr:
 * phi = (1 - tanh(2 (R - |p - ctr|)/lambda))/2. */
void oracle_init_sphere(double *phi, int nx, int ny, int nz, const double ctr[3],
                        double R, double lambda, double dx);

/* Cubic particle (phi = 0 inside) of half side `half` around ctr, the product
 * of three 1D ideal profiles: phi = 1 - prod_a (1 - tanh(2 (|p_a - ctr_a| - half)/lambda))/2.
 * The paper starts its shape relaxation (Sec. 3.3) from a cube without giving
 * the profile; this product is exact across every face away from edges. */
void oracle_init_cube(double *phi, int nx, int ny, int nz, const double ctr[3], double half,
                      double lambda, double dx);

/* Copy phi into the padded array and fill the one-cell ghost layer,
 * faces x, then y, then z (so edges and corners compose). */
void oracle_fill_ghosts(const orc_params *p, const double *phi, double *pad);

/* Right-hand side dphi/dt of the discrete Allen-Cahn equation (Eq. 2 with the
 * functional derivative of Eq. 1) at every interior cell.  Returns the number
 * of cells where 1 - a_k^2 (1-2phi)^2 <= 0 (the TI potential is undefined). */
long oracle_rhs(const orc_params *p, const double *phi, double *R);

/* n_steps explicit Euler steps phi <- phi + dt R (in place). */
long oracle_step(const orc_params *p, double *phi, int n_steps);

/* Constant-volume steps (Sec. 3.3: a homogeneous, time-dependent driving force
 * keeps the particle volume fixed).  Each step takes R at dF = 0, then the one
 * homogeneous dF for which the step leaves sum_p phi_p unchanged,
 * dF = sum_p R_p / (2M/(3 lambda Gamma) sum_p h3'(phi_p)), and applies
 * phi <- phi + dt (R - 2M/(3 lambda Gamma) dF h3'(phi)).  p->dF is ignored;
 * dF_out (NULL or n_steps doubles) receives each step's dF. */
long oracle_step_conserving(const orc_params *p, double *phi, int n_steps, double *dF_out);

/* FP64 interface diagnostics (Sec. 2.3 inversion of the ideal profile):
 * out[0] volume sum(phi) dx^3, out[1] S_w = sum q, out[2] S_c, out[3] S_r,
 * out[4] min phi, out[5] max phi, out[6] count of non-finite cells,
 * out[7] planar position c = S_c/S_w, out[8] radius R = S_r/S_w.
 * q = phi(1-phi); sums over cells with 1e-6 < phi < 1 - 1e-6;
 * S_c = sum q (p.n - (lambda/2) artanh(1 - 2 phi)),
 * S_r = sum q (|p - ctr| + (lambda/2) artanh(1 - 2 phi)). */
void oracle_stats(const orc_params *p, const double *phi, const double ctr[3],
                  double *out9);

/* Interface energy F_int = sum_p f_p(dF = 0) dx^3 of Eq. 1. */
double oracle_energy(const orc_params *p, const double *phi);

/* phi = l contour points on the grid edges along x, y, z by the nonlinear
 * profile interpolation of Sec. 2.3.  Writes up to max_pts points (xyz) and
 * returns the number found. */
long oracle_contour(const orc_params *p, const double *phi, double l,
                    double *pts, long max_pts);

#ifdef __cplusplus
}
#endif
#endif
