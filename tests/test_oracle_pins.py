"""Pins of the FP64 oracle to what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the paper's
closed forms (ideal profile Eq. 3, v_th = -M dF/Gamma, phase-stability bound of
Sec. 3.1), its printed table (Tab. 1), invariants (discrete equilibrium Eq. 4,
shift invariance of the TI energy), brute force (autograd of the energy Eq. 1
on a 4^3 grid) and textbook limits.  A dropped term, a wrong sign or index, or
a transposed operand in the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
import torch

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _unit(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v)


def _rand_normals(seed, k):
    rng = np.random.default_rng(seed)
    return [_unit(rng.normal(size=3)) for _ in range(k)]


# ----------------------------------------------------------------- Tab. 1


def test_tab1_coupling_multisets():
    """Tab. 1: |arctanh a_k| for u || [120], per shell, in units 1/(sqrt5 lambda)."""
    rows = [tuple(int(x) for x in ln.split()) for ln in open(os.path.join(GOLDEN, "tab1_120_arctanh.txt"))
            if ln.strip() and not ln.startswith("#")]
    lam = 3.0
    a = O.coupling(_unit([1, 2, 0]), lam, 1.0)
    got = np.abs(np.arctanh(a)) * math.sqrt(5.0) * lam
    d, shell = O.directions()
    for s in (1, 2, 3):
        want = sorted(v for (sh, k, v) in rows if sh == s)
        have = sorted(got[shell == s].tolist())
        assert np.allclose(have, want, atol=1e-12), (s, have, want)
    # the table's grid vectors: 3, 6, 4 directions with |r|^2 = 1, 2, 3
    assert [int((shell == s).sum()) for s in (1, 2, 3)] == [3, 6, 4]
    assert np.all((d ** 2).sum(axis=1) == shell)
    # one vector per +/- pair: no two directions parallel
    for i in range(13):
        for j in range(i + 1, 13):
            assert np.linalg.norm(np.cross(d[i], d[j])) > 0


# ------------------------------------------------- weights (nu_j, gamma_j)


@pytest.mark.parametrize("stencil", [6, 18, 26])
def test_shell_sums_reproduce_square_gradient(stencil):
    """Sec. 2.1: each shell sum nu_j sum_k (e_k.g)^2 approximates |g|^2; with
    nu_j = 3/m_j (m_j = directions per shell) it is exact for linear fields."""
    p = O.Params(4, 4, 4, stencil=stencil)
    w, gam = O.weights(p)
    assert abs(gam.sum() - 1.0) < 1e-15
    d, shell = O.directions()
    rng = np.random.default_rng(1)
    for _ in range(5):
        g = rng.normal(size=3)
        tot = sum(w[k] * (d[k] @ g) ** 2 / shell[k] for k in range(13))
        assert abs(tot - g @ g) < 1e-12 * (g @ g)


@pytest.mark.parametrize("stencil", [18, 26])
def test_default_gamma_gives_isotropic_laplacian(stencil):
    """Reading r4: the default ponderations cancel the anisotropic fourth-order
    truncation term of sum_k w_k/|r_k|^2 (phi(x+r)+phi(x-r)-2phi) (Taylor)."""
    import sympy as sp
    p = O.Params(4, 4, 4, stencil=stencil)
    w, _ = O.weights(p)
    d, shell = O.directions()
    kx, ky, kz = sp.symbols("kx ky kz")
    # Fourier symbol of the stencil to fourth order in k: sum w/|r|^2 * (-(k.r)^2 + (k.r)^4/12)
    sym2 = 0
    sym4 = 0
    for k in range(13):
        if w[k] == 0:
            continue
        kr = kx * int(d[k][0]) + ky * int(d[k][1]) + kz * int(d[k][2])
        wk = sp.Rational(w[k]).limit_denominator(1000) / int(shell[k])
        sym2 += -wk * kr ** 2
        sym4 += wk * kr ** 4 / 12
    k2 = kx ** 2 + ky ** 2 + kz ** 2
    assert sp.expand(sym2 + k2) == 0          # consistent Laplacian
    ratio = sp.simplify(sym4 / k2 ** 2)       # isotropic iff proportional to |k|^4
    assert ratio.free_symbols == set(), ratio


# ----------------------------------------------------- profile and coupling


def test_addition_property_and_contact_bc_exact():
    """Eq. 7 with the signed coupling reproduces the ideal profile (Eq. 3) in the
    ghost layer on all faces, edges and corners."""
    for n in _rand_normals(2, 4):
        for lam in (0.7, 2.0, 4.0):
            p = O.Params(7, 6, 5, bc=(O.CONTACT,) * 6, n=tuple(n), lam=lam)
            c = 0.4 + float(n @ [3, 2.5, 2])
            pad = O.fill_ghosts(p, O.init_planar(p, c))
            k, j, i = np.meshgrid(np.arange(-1, 6), np.arange(-1, 7), np.arange(-1, 8), indexing="ij")
            pn = i * n[0] + j * n[1] + k * n[2]
            ideal = 0.5 * (1 - np.tanh(2 * (pn - c) / lam))
            assert np.abs(pad - ideal).max() < 2e-14   # a few ulps after three compositions


def test_periodic_and_noflux_ghosts():
    p = O.Params(5, 4, 3, bc=(O.PERIODIC, O.PERIODIC, O.NOFLUX, O.NOFLUX, O.PERIODIC, O.NOFLUX))
    phi = np.random.default_rng(3).random(p.shape)
    pad = O.fill_ghosts(p, phi)
    core = pad[1:-1, 1:-1, 1:-1]
    assert np.array_equal(core, phi)
    assert np.array_equal(pad[1:-1, 1:-1, 0], phi[:, :, -1])
    assert np.array_equal(pad[1:-1, 1:-1, -1], phi[:, :, 0])
    assert np.array_equal(pad[1:-1, 0, 1:-1], phi[:, 0, :])
    assert np.array_equal(pad[1:-1, -1, 1:-1], phi[:, -1, :])
    assert np.array_equal(pad[0, 1:-1, 1:-1], phi[-1])
    assert np.array_equal(pad[-1, 1:-1, 1:-1], phi[-1])
    # corner: z- periodic of (y- noflux of (x- periodic))
    assert pad[0, 0, 0] == phi[-1, 0, -1]


# ------------------------------------------------- discrete equilibrium (Eq. 4)


@pytest.mark.parametrize("stencil", [6, 18, 26])
def test_fixed_point_any_orientation(stencil):
    """Eq. 4 with the TI potential (Eq. 6): the ideal profile is a stationary
    discrete solution for any n, every cell including the boundary cells
    (contact BCs); the CF potential violates it."""
    for n in _rand_normals(10 + stencil, 3):
        for lam in (1.0, 2.0, 4.0):
            p = O.Params(9, 8, 7, bc=(O.CONTACT,) * 6, n=tuple(n), lam=lam, stencil=stencil)
            phi = O.init_planar(p, c=float(n @ [4, 3.5, 3]) + 0.21)
            R, nbad = O.rhs(p, phi)
            assert nbad == 0
            assert np.abs(R).max() < 1e-13
            pc = O.Params(**{**p.__dict__, "scheme": O.CF})
            Rc, _ = O.rhs(pc, phi)
            if lam <= 2.0:
                assert np.abs(Rc).max() > 1e-2


@pytest.mark.parametrize("stencil", [6, 26])
def test_exact_translation_velocity(stencil):
    """With h3 the ideal profile translates at v_th = -M dF / Gamma (Sec. 2.1):
    R_p = dphi/dt of the moving profile = (4 v/lambda) q_p, pointwise."""
    for n in _rand_normals(20, 2):
        for (M, G, dF, lam) in ((1.0, 1.0, 0.05, 4.0), (0.7, 1.3, -0.08, 2.5)):
            p = O.Params(8, 7, 6, bc=(O.CONTACT,) * 6, n=tuple(n), lam=lam, stencil=stencil,
                         M=M, Gamma=G, dF=dF, C_gamma=0.55)
            phi = O.init_planar(p, c=float(n @ [3.5, 3, 2.5]))
            R, _ = O.rhs(p, phi)
            v = -M * dF / G
            assert np.abs(R - 4 * v / lam * phi * (1 - phi)).max() < 1e-13


# ------------------------------------------------- brute force: autograd of Eq. 1


def _h_torch(phi, interp):
    """The interpolation functions of Tab. 2, typed from the table."""
    if interp == "h5":
        return phi ** 3 * (10 - 15 * phi + 6 * phi ** 2)
    if interp == "abel":
        return phi ** 2 / (phi ** 2 + (1 - phi) ** 2)
    return phi ** 2 * (3 - 2 * phi)


def _energy_torch(phi, w, d, shell, lam, dx, Gamma, Cg, dF, a=None, interp="h3"):
    """Eq. 1 typed from the paper (periodic forward differences), with Eq. 6 or
    the CF potential and the interpolation function of Tab. 2; F = sum_p f_p dx^3."""
    q = phi * (1 - phi)
    s = 1 - 2 * phi
    f = torch.zeros_like(phi)
    for k in range(13):
        if w[k] == 0:
            continue
        r = math.sqrt(shell[k]) * dx
        shifted = torch.roll(phi, shifts=(-int(d[k][2]), -int(d[k][1]), -int(d[k][0])), dims=(0, 1, 2))
        dplus = (shifted - phi) / r
        if a is None:
            g = 8 * phi ** 2 * (1 - phi) ** 2 / 3
        else:
            A = a[k] ** 2
            if A == 0:
                g = torch.zeros_like(phi)
            else:
                g = lam ** 2 / r ** 2 * (q + (1 - A) / (4 * A) * torch.log((1 - A) / (1 - A * s ** 2)))
        f = f + w[k] * (lam ** 2 / 2 * dplus ** 2 + g)
    f = Gamma / (Cg * lam) * f + dF * _h_torch(phi, interp)
    return f.sum() * dx ** 3


@pytest.mark.parametrize("stencil", [6, 18, 26])
@pytest.mark.parametrize("scheme", [O.TI_GLOBAL, O.CF, O.CF_H5, O.CF_HABEL])
def test_rhs_is_energy_gradient_4cubed(stencil, scheme):
    """Eq. 2: 3 lambda Gamma dphi/dt = -2 M dF/dphi.  Autograd of Eq. 1 on a
    periodic 4^3 random field reproduces the oracle's right-hand side."""
    rng = np.random.default_rng(100 + stencil)
    phi = 0.05 + 0.9 * rng.random((4, 4, 4))
    n = _unit(rng.normal(size=3))
    lam, dx, M, G, Cg, dF = 1.7, 0.9, 0.8, 1.2, 0.6, 0.03
    p = O.Params(4, 4, 4, bc=(O.PERIODIC,) * 6, n=tuple(n), lam=lam, dx=dx, M=M, Gamma=G,
                 C_gamma=Cg, dF=dF, stencil=stencil, scheme=scheme)
    R, nbad = O.rhs(p, phi)
    assert nbad == 0
    w, _ = O.weights(p)
    d, shell = O.directions()
    a = None if scheme in (O.CF, O.CF_H5, O.CF_HABEL) else np.tanh(2 * dx * (d @ n) / lam)
    interp = {O.CF_H5: "h5", O.CF_HABEL: "abel"}.get(scheme, "h3")
    t = torch.tensor(phi, dtype=torch.float64, requires_grad=True)
    F = _energy_torch(t, w, d, shell, lam, dx, G, Cg, dF, a, interp)
    (grad,) = torch.autograd.grad(F, t)
    dFdphi = grad.numpy() / dx ** 3
    R_ref = -2 * M / (3 * lam * G) * dFdphi
    assert np.abs(R - R_ref).max() < 1e-12 * max(1.0, np.abs(R_ref).max())
    # the oracle's own energy equals Eq. 1 typed here (dF = 0 part)
    p0 = O.Params(**{**p.__dict__, "dF": 0.0})
    F0 = _energy_torch(t.detach(), w, d, shell, lam, dx, G, Cg, 0.0, a, interp).item()
    assert abs(O.energy(p0, phi) - F0) < 1e-12 * abs(F0)


# ------------------------------------------------------- time integration


def _velocity_1d(scheme, lam, dF, dt, t_end=200.0, t_start=50.0, nx=72, stencil=6):
    """Planar [100] interface on nx x 1 x 1 (no-flux in x): mean velocity of the
    inverted-profile position between t_start and t_end."""
    p = O.Params(nx, 1, 1, bc=(O.NOFLUX, O.NOFLUX, O.PERIODIC, O.PERIODIC, O.PERIODIC, O.PERIODIC),
                 n=(1.0, 0.0, 0.0), lam=lam, dt=dt, dF=dF, stencil=stencil, scheme=scheme)
    c0 = nx / 2 + 12.0 if dF > 0 else nx / 2 - 12.0   # v_th = -M dF/Gamma
    phi = O.init_planar(p, c0)
    n1 = int(round(t_start / dt))
    n2 = int(round(t_end / dt))
    phi = O.step(p, phi, n1)
    c1 = O.stats(p, phi)["position"]
    phi = O.step(p, phi, n2 - n1)
    c2 = O.stats(p, phi)["position"]
    return (c2 - c1) / ((n2 - n1) * dt)


def test_velocity_first_order_in_dt_and_cf_friction():
    """SPFM velocity error is at time-discretisation level and first order in dt
    (Sec. 3.1); CF keeps an O(1e-2) error at lambda~=4 as dt -> 0 (Sec. 3.1:
    about 2e-2)."""
    dF = 0.05
    vth = -dF
    e1 = _velocity_1d(O.TI_GLOBAL, 4.0, dF, 0.1) / vth - 1
    e2 = _velocity_1d(O.TI_GLOBAL, 4.0, dF, 0.05) / vth - 1
    assert abs(e1) < 2e-4 and abs(e2) < 1e-4
    assert 1.7 < e1 / e2 < 2.3
    f1 = _velocity_1d(O.CF, 4.0, dF, 0.1) / vth - 1
    f2 = _velocity_1d(O.CF, 4.0, dF, 0.05) / vth - 1
    assert 1e-2 < abs(f1) < 5e-2
    assert abs(f1 - f2) < 0.1 * abs(f1)


def test_cf_pinned_ti_not():
    """Fig. 1 / Sec. 3.1: CF is pinned (v = 0) at lambda~=2, dF~=0.1; TI moves at v_th."""
    dF = 0.1
    v_cf = _velocity_1d(O.CF, 2.0, dF, 0.1, t_end=300.0, t_start=100.0)
    v_ti = _velocity_1d(O.TI_GLOBAL, 2.0, dF, 0.1, t_end=150.0, t_start=50.0)
    assert abs(v_cf) < 1e-6
    assert abs(v_ti / -dF - 1) < 1e-3


def test_phase_stability_bound_cf():
    """Sec. 3.1: CF+h3 keeps a barrier between the phases iff
    |dF~| < 8 / (3 C_Gamma lambda~).  The uniform-field RHS has an interior zero
    exactly then."""
    lam, dx, Cg = 3.0, 1.0, 2.0 / 3.0
    bound = 8.0 / (3 * Cg * lam / dx)
    phis = np.linspace(1e-4, 1 - 1e-4, 4001)
    for frac, expect in ((0.97, True), (1.03, False)):
        dF = frac * bound
        p = O.Params(1, 1, 1, lam=lam, dx=dx, C_gamma=Cg, dF=dF, scheme=O.CF, stencil=26)
        vals = np.array([O.rhs(p, np.full((1, 1, 1), x))[0][0, 0, 0] for x in phis])
        has_zero = bool(np.any(np.sign(vals[1:]) != np.sign(vals[:-1])))
        assert has_zero == expect


@pytest.mark.parametrize("scheme,bound", [(O.CF_HABEL, 8.0), (O.CF_H5, None)])
def test_phase_stability_of_the_other_interpolations(scheme, bound):
    """The barrier criterion of Sec. 3.1 for the Tab. 2 interpolations, from
    the uniform-field RHS (brute force over phi).  h5: a barrier at any dF
    (h5' vanishes to second order at both phases).  h_Abel: h' = 8 q / (1 + s^2)^2,
    so df/dphi = q (16 s / (C lambda~) + 8 dF~ / (1 + s^2)^2) (Gamma, dx units)
    changes sign inside (0, 1) iff |dF~| < 8 / (C_Gamma lambda~) (reading r20:
    the paper prints 440 / (3 C_Gamma lambda~))."""
    lam, dx, Cg = 3.0, 1.0, 2.0 / 3.0
    phis = np.linspace(1e-4, 1 - 1e-4, 4001)
    cases = ((0.97, True), (1.03, False)) if bound else ((1.0, True), (30.0, True), (300.0, True))
    for frac, expect in cases:
        dF = frac * (bound / (Cg * lam / dx) if bound else 8.0 / (3 * Cg * lam / dx))
        p = O.Params(1, 1, 1, lam=lam, dx=dx, C_gamma=Cg, dF=dF, scheme=scheme, stencil=26)
        vals = np.array([O.rhs(p, np.full((1, 1, 1), x))[0][0, 0, 0] for x in phis])
        has_zero = bool(np.any(np.sign(vals[1:]) != np.sign(vals[:-1])))
        assert has_zero == expect, (frac, dF)


def test_moving_frame_shift():
    """The 1D study's moving frame: phi_i <- phi_{i+1} with the end cell
    repeated; on the ideal profile a shift by one cell equals the profile
    moved by -dx (away from the last cell)."""
    p = O.Params(40, 2, 3, lam=3.0)
    phi = O.init_planar(p, 20.3)
    got = O.shift_x(p, phi, 1)
    assert np.abs(got[..., :-1] - O.init_planar(p, 19.3)[..., :-1]).max() < 1e-15
    assert np.all(got[..., -1] == phi[..., -1])
    assert np.all(O.shift_x(p, phi, -2)[..., :2] == phi[..., :1])


# ---------------------------------------------------------------- energy


def test_ti_energy_shift_invariant_cf_not():
    """Fig. 1b: the TI interface energy does not depend on the sub-grid position
    of the ideal profile; the CF energy oscillates with it."""
    lam = 2.0
    p = O.Params(64, 1, 1, bc=(O.NOFLUX, O.NOFLUX) + (O.PERIODIC,) * 4, lam=lam)
    pc = O.Params(**{**p.__dict__, "scheme": O.CF})
    e_ti, e_cf = [], []
    for c in np.linspace(30.0, 31.0, 9):
        phi = O.init_planar(p, c)
        e_ti.append(O.energy(p, phi))
        e_cf.append(O.energy(pc, phi))
    assert np.ptp(e_ti) < 1e-12 * np.mean(e_ti)
    assert np.ptp(e_cf) > 1e-4 * np.mean(e_cf)


def test_energy_continuum_limit_is_gamma():
    """Reading r5: with C_Gamma = 2/3 the energy per unit area of the ideal
    profile tends to Gamma as lambda~ grows (continuum integral 2 Gamma/(3 C_Gamma)),
    with a second-order discretisation error."""
    errs = []
    for lam in (8.0, 16.0, 32.0):
        nx = int(12 * lam)
        p = O.Params(nx, 1, 1, bc=(O.NOFLUX, O.NOFLUX) + (O.PERIODIC,) * 4, lam=lam, Gamma=1.3,
                     stencil=26)
        phi = O.init_planar(p, nx / 2 + 0.3)
        errs.append(abs(O.energy(p, phi) / 1.3 - 1))
    assert errs[2] < 1e-3
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


# ----------------------------------------------------------- diagnostics


def test_position_and_radius_estimators_exact():
    """Sec. 2.3 inversion: the q-weighted artanh estimate returns the exact c of
    any ideal planar profile and the exact R of the ideal radial profile."""
    for n in _rand_normals(30, 3):
        p = O.Params(10, 9, 8, n=tuple(n), lam=1.3)
        c = float(n @ [4.5, 4, 3.5]) + 0.37
        st = O.stats(p, O.init_planar(p, c))
        assert abs(st["position"] - c) < 1e-12
        assert st["nonfinite"] == 0
    p = O.Params(24, 24, 24, lam=3.0)
    ctr = (11.5, 11.2, 11.7)
    st = O.stats(p, O.init_sphere(p, ctr, 7.3), ctr)
    assert abs(st["radius"] - 7.3) < 1e-12


def test_contour_points_on_plane():
    """Sec. 2.3: the nonlinear interpolation puts the phi = 1/2 contour points of
    an ideal planar profile exactly on the plane p.n = c."""
    for n in _rand_normals(31, 3):
        p = O.Params(10, 10, 10, n=tuple(n), lam=0.8)
        c = float(n @ [4.5, 4.5, 4.5]) + 0.13
        pts = O.contour(p, O.init_planar(p, c))
        assert len(pts) > 20
        assert np.abs(pts @ n - c).max() < 1e-12


def test_sphericity_of_ideal_sphere_small():
    p = O.Params(32, 32, 32, lam=3.0)
    s = O.sphericity(p, O.init_sphere(p, (15.5, 15.5, 15.5), 9.0))
    assert abs(s["R_mean"] - 9.0) < 0.05
    assert s["eps_eff"] < 5e-3


def test_sphericity_barycentre_is_the_particles():
    """Sec. 3.3: the radii are taken from the particle's barycentre.  An
    off-centre sphere in a box that is not a cube separates the particle-weighted
    barycentre (the sphere's centre) from the matrix-weighted one (near the box
    centre), so weighting by the wrong phase fails here; the particle may be
    either phase."""
    shape, ctr, R, lam = (40, 32, 28), np.array([10.3, 14.1, 12.7]), 6.0, 2.0
    p = O.Params(*shape, lam=lam)
    grain0 = O.init_sphere(p, ctr, R)            # phi = 0 inside
    for phi, inside in ((grain0, 0), (1.0 - grain0, 1)):
        s = O.sphericity(p, phi, inside_phase=inside)
        # the profile is radial about ctr: its grid-sampled centroid sits on ctr
        # up to the aliasing of the sampled profile (2.5e-5 cells at lambda = 2)
        assert np.abs(np.array(s["barycentre"]) - ctr).max() < 1e-4, s["barycentre"]
        assert abs(s["R_mean"] - R) < 0.03 and s["eps_eff"] < 5e-3
        assert s["n_points"] > 300
    # the matrix weighting would put the centre far from the sphere
    wrong = O.sphericity(p, grain0, inside_phase=1)
    assert np.abs(np.array(wrong["barycentre"]) - ctr).max() > 2.0
    assert wrong["eps_eff"] > 0.2


def test_sphericity_of_a_cube_start():
    """The cube start of Sec. 3.3 (half side h, centre on a grid point, off the
    box centre): its barycentre is the cube's centre by symmetry, the smallest
    radius is h exactly (contour points at the face centres, where the profile
    is the 1D profile of Eq. 3 and the nonlinear interpolation is exact), and the
    largest is that of the corner of the phi = 1/2 level set, below sqrt(3) h."""
    ctr, h, lam = np.array([12.0, 11.0, 10.0]), 5.5, 1.0
    p = O.Params(30, 26, 24, lam=lam)
    s = O.sphericity(p, O.init_cube(p, ctr, h), inside_phase=0)
    assert np.abs(np.array(s["barycentre"]) - ctr).max() < 1e-9
    assert abs(s["R_min"] - h) < 1e-8
    # on the body diagonal the three 1D fractions are equal: ((1 - t)/2)^3 = 1/2
    t = 1.0 - 2.0 * 2.0 ** (-1.0 / 3.0)
    d_corner = h + 0.5 * lam * math.atanh(t)
    assert math.sqrt(3.0) * d_corner - 0.5 < s["R_max"] < math.sqrt(3.0) * h
    assert s["eps_eff"] == pytest.approx((s["R_max"] - s["R_min"]) / (2.0 * s["R_mean"]), rel=1e-12)
    assert s["eps_eff"] > 0.1


# ------------------------------------------------------------- reductions


def test_100_interface_reduces_to_1d_and_axis_permutation():
    p = O.Params(16, 5, 4, bc=(O.NOFLUX, O.NOFLUX) + (O.PERIODIC,) * 4, n=(1.0, 0, 0), lam=2.0,
                 dF=0.04, stencil=26)
    phi = O.step(p, O.init_planar(p, 7.3), 20)
    assert np.abs(phi - phi[:1, :1, :]).max() == 0.0
    p1 = O.Params(16, 1, 1, bc=p.bc, n=(1.0, 0, 0), lam=2.0, dF=0.04, stencil=26)
    phi1 = O.step(p1, O.init_planar(p1, 7.3), 20)
    assert np.abs(phi[0, 0] - phi1[0, 0]).max() < 1e-15
    # permuting axes of field and normal permutes the result
    rng = np.random.default_rng(5)
    n = _unit(rng.normal(size=3))
    q = O.Params(6, 5, 4, bc=(O.CONTACT,) * 6, n=tuple(n), lam=1.5, dF=0.02, stencil=26)
    f = O.init_planar(q, float(n @ [2.5, 2, 1.5])) + 1e-3 * rng.random(q.shape)
    r = O.step(q, f, 5)
    qt = O.Params(4, 5, 6, bc=(O.CONTACT,) * 6, n=(n[2], n[1], n[0]), lam=1.5, dF=0.02, stencil=26)
    rt = O.step(qt, f.transpose(2, 1, 0).copy(), 5)
    assert np.abs(rt.transpose(2, 1, 0) - r).max() < 1e-14


def _signed_perm_apply(f, perm, sign):
    """The field under the lattice symmetry x'_a = sign_a x_perm(a) of an N^3
    periodic grid (a reflection maps index i to N - 1 - i); arrays are (z, y, x)."""
    N = f.shape[0]
    c = np.indices(f.shape)[::-1]              # c[0] = x', c[1] = y', c[2] = z'
    old = [None, None, None]
    for a in range(3):
        old[perm[a]] = c[a] if sign[a] > 0 else N - 1 - c[a]
    return f[old[2], old[1], old[0]]


@pytest.mark.parametrize("scheme", [O.TI_LOCAL, O.TI_GLOBAL, O.CF])
def test_rhs_is_equivariant_under_the_cube_group(scheme):
    """The discrete equation has the symmetry of the cubic lattice: moving the
    field by a rotation or reflection of the grid (and the TI direction u with
    it) moves the right-hand side the same way.  For TI_n this pins the axis
    consistency of the local normal estimate: a neighbour offset or a grid
    spacing wrong on one axis breaks it.  (Sign flips or permutations of the
    normal's components cannot show: the potential depends only on the multiset
    of A_k of each shell.)  6^3 periodic, 27-point, a random field in (0, 1)
    near a tilted profile."""
    import itertools
    rng = np.random.default_rng(11)
    u = _unit(rng.normal(size=3))
    N = 6
    p = O.Params(N, N, N, bc=(O.PERIODIC,) * 6, n=tuple(u), lam=2.0, dF=0.03, stencil=26, scheme=scheme)
    f = np.clip(O.init_planar(p, float(u @ [2.5, 2.5, 2.5])) + 0.05 * (rng.random(p.shape) - 0.5), 1e-3, 1 - 1e-3)
    R, _ = O.rhs(p, f)
    assert np.isfinite(R).all() and np.abs(R).max() > 1e-3
    elems = list(itertools.product(itertools.permutations(range(3)), itertools.product((1, -1), repeat=3)))
    for k in rng.choice(len(elems), 8, replace=False):
        perm, sign = elems[k]
        up = np.zeros(3)
        for a in range(3):
            up[a] = sign[a] * u[perm[a]]
        q = O.Params(N, N, N, bc=(O.PERIODIC,) * 6, n=tuple(up), lam=2.0, dF=0.03, stencil=26, scheme=scheme)
        Rq, _ = O.rhs(q, _signed_perm_apply(f, perm, sign))
        assert np.abs(Rq - _signed_perm_apply(R, perm, sign)).max() < 1e-12, (perm, sign)


def test_ti_minus_cf_vanishes_with_resolution():
    """P6: the TI and CF right-hand sides converge as lambda~ grows (O(lambda~^-2))."""
    diffs = []
    for lam in (4.0, 8.0, 16.0):
        n = _unit([1.0, 0.4, 0.2])
        p = O.Params(12, 12, 12, bc=(O.CONTACT,) * 6, n=tuple(n), lam=lam, stencil=26)
        phi = O.init_planar(p, float(n @ [5.5, 5.5, 5.5]))
        R_ti, _ = O.rhs(p, phi)
        R_cf, _ = O.rhs(O.Params(**{**p.__dict__, "scheme": O.CF}), phi)
        diffs.append(np.abs(R_ti - R_cf).max() * lam ** 2)
    # scaled differences stay bounded and approach a constant
    assert diffs[2] < 1.5 * diffs[1] and diffs[1] < 1.5 * diffs[0]


# ------------------------------------------------------------------ TI_n


def test_local_normal_equals_global_on_planar_profile():
    """Reading r14: on an ideal planar profile psi is linear, the central
    differences give n exactly, and TI_n equals TI with that global n wherever
    the clamp is inactive; elsewhere the RHS stays at the clamp level."""
    for n in _rand_normals(40, 3):
        p = O.Params(30, 11, 10, bc=(O.CONTACT,) * 6, n=tuple(n), lam=1.5, dF=0.03, stencil=26)
        phi = O.init_planar(p, float(n @ [14.5, 5, 4.5]) + 0.2)
        Rg, _ = O.rhs(p, phi)
        Rl, _ = O.rhs(O.Params(**{**p.__dict__, "scheme": O.TI_LOCAL}), phi)
        pad = O.fill_ghosts(p, phi)
        eps = 1e-6
        ok = np.ones(p.shape, dtype=bool)
        for ax in range(3):
            for sgn in (-1, 1):
                sl = [slice(1, -1)] * 3
                sl[2 - ax] = slice(1 + sgn, pad.shape[2 - ax] - 1 + sgn)
                nb = pad[tuple(sl)]
                ok &= (nb > eps) & (nb < 1 - eps)
        assert ok.sum() > 50
        assert np.abs(Rl - Rg)[ok].max() < 1e-11
        if (~ok).any():
            assert np.abs(Rl - Rg)[~ok].max() < 1e-4


def test_local_normal_fallback_is_the_cf_potential():
    """Reading r14, cells with no normal: where |grad psi| < 1e-8 (a uniform
    field, or a cell whose six face neighbours sit in the clamp on the same
    side) the cell takes the CF potential.  A uniform phi = 0.3 field then moves
    at the closed-form CF rate R = -(16 D / lambda^2) q s - (4 M dF/(lambda Gamma)) q
    with D = 2M/(3 C_Gamma); the other reading, a_k = 0, would leave only the
    driving term."""
    for stencil in (6, 18, 26):
        M, Gamma, lam, dF, Cg = 0.7, 1.3, 2.5, 0.04, 2.0 / 3.0
        p = O.Params(6, 5, 4, lam=lam, M=M, Gamma=Gamma, dF=dF, stencil=stencil, scheme=O.TI_LOCAL,
                     n=tuple(_unit([1.0, 2.0, 3.0])))
        phi0 = 0.3
        R, _ = O.rhs(p, np.full(p.shape, phi0))
        q, s, D = phi0 * (1 - phi0), 1 - 2 * phi0, 2 * M / (3 * Cg)
        expect = -(16.0 * D / lam ** 2) * q * s - 4 * M * dF / (lam * Gamma) * q
        assert np.abs(R - expect).max() < 1e-14
        assert abs(expect + 4 * M * dF / (lam * Gamma) * q) > 0.1     # a_k = 0 differs


def test_local_normal_fallback_cells_in_the_clamp():
    """A planar profile with a bulk perturbation: cells whose psi differences are
    exactly zero on all three axes (all face neighbours in the same clamp) take
    the CF right-hand side, every other cell the TI right-hand side with the
    normal estimated from psi; the mask is rebuilt here from the clamp rule."""
    n = _unit([1.0, 0.3, 0.0])
    p = O.Params(40, 8, 6, bc=(O.NOFLUX, O.NOFLUX) + (O.PERIODIC,) * 4, n=tuple(n), lam=2.0, dF=0.02,
                 stencil=26, scheme=O.TI_LOCAL)
    phi = O.init_planar(p, float(n @ [19.5, 3.5, 2.5]))
    # bulk cells perturbed inside the clamp (phi < 1e-6 and 1 - phi < 1e-6)
    rng = np.random.default_rng(9)
    lo, hi = phi < 1e-9, phi > 1 - 1e-9
    phi[lo] = 1e-7 * rng.random(lo.sum())
    phi[hi] = 1 - 1e-7 * rng.random(hi.sum())
    Rl, _ = O.rhs(p, phi)
    Rcf, _ = O.rhs(O.Params(**{**p.__dict__, "scheme": O.CF}), phi)
    pad = O.fill_ghosts(p, phi)
    psi = 0.5 * p.lam * np.arctanh(1 - 2 * np.clip(pad, 1e-6, 1 - 1e-6))
    g2 = np.zeros(p.shape)
    for ax in range(3):
        sp, sm = [slice(1, -1)] * 3, [slice(1, -1)] * 3
        sp[2 - ax], sm[2 - ax] = slice(2, None), slice(0, -2)
        g2 += ((psi[tuple(sp)] - psi[tuple(sm)]) / (2 * p.dx)) ** 2
    fb = ~(np.sqrt(g2) >= 1e-8)
    assert fb.sum() > 100 and (~fb).sum() > 100
    assert np.array_equal(Rl[fb], Rcf[fb])
    assert (lo & fb).sum() > 10 and (hi & fb).sum() > 10
    # elsewhere the RHS is not the CF one: the interface cells see the TI potential
    band = (phi > 0.05) & (phi < 0.95)
    assert np.abs(Rl - Rcf)[band].max() > 1e-3


# ------------------------------------------------ constant-volume relaxation


def test_cube_profile_is_the_1d_profile_across_each_face():
    """The cube start: far from edges the product of the three 1D fractions is
    the 1D ideal profile (Eq. 3) across the face; the cube has its symmetries."""
    N, lam, half = 40, 3.0, 10.0
    p = O.Params(N, N, N, lam=lam)
    ctr = ((N - 1) / 2.0,) * 3
    phi = O.init_cube(p, ctr, half)
    j = k = N // 2   # the line through the face centres along x (|dy|, |dz| = 0.5)
    x = np.arange(N) - ctr[0]
    inner = (1 - np.tanh(2 * (0.5 - half) / lam)) / 2   # the other two factors
    want = 1 - inner ** 2 * (1 - np.tanh(2 * (np.abs(x) - half) / lam)) / 2
    assert np.abs(phi[k, j, :] - want).max() < 1e-14
    assert np.abs(phi - phi.transpose(0, 2, 1)).max() < 1e-14
    assert np.abs(phi - phi[::-1, :, :]).max() < 1e-14


@pytest.mark.parametrize("scheme", [O.CF, O.TI_LOCAL, O.TI_GLOBAL])
def test_conserving_step_keeps_sum_phi(scheme):
    """Sec. 3.3: the homogeneous driving force holds the particle volume, so
    sum(phi) is invariant step after step (rounding only), while the field
    itself does change."""
    N = 24
    p = O.Params(N, N, N, n=tuple(_unit([1, 2, 0])), lam=2.5, dt=0.05, stencil=26, scheme=scheme)
    rng = np.random.default_rng(3)
    phi0 = O.init_cube(p, ((N - 1) / 2.0,) * 3, 6.0) + 0.01 * rng.random(p.shape)
    phi, dF = O.step_conserving(p, phi0, 30)
    assert abs(phi.sum() - phi0.sum()) <= 1e-12 * phi0.sum()
    assert np.abs(phi - phi0).max() > 1e-3 and np.all(np.isfinite(dF))


def test_conserving_step_needs_no_force_on_an_exact_plane():
    """An ideal planar interface under TI with contact faces is a fixed point
    (Eq. 4) at dF = 0, so the volume-holding dF is zero and nothing moves."""
    n = _unit([1, 2, 2])
    p = O.Params(24, 20, 18, bc=(O.CONTACT,) * 6, n=tuple(n), lam=3.0, dt=0.05, stencil=26)
    phi0 = O.init_planar(p, float(n @ [11.5, 9.5, 8.5]))
    phi, dF = O.step_conserving(p, phi0, 20)
    assert np.abs(dF).max() < 1e-13
    assert np.abs(phi - phi0).max() < 1e-13


def test_conserving_force_on_a_sphere_is_gibbs_thomson():
    """Sharp-interface limit: the force that holds a sphere of radius R is the
    curvature force 2 Gamma / R, independent of the mobility M, with an error
    of order (lambda/R)^2 (it falls about fourfold when R doubles)."""
    errs = []
    for R, N in ((12.0, 40), (24.0, 64)):
        for M, G in ((1.0, 1.0), (3.0, 2.0)):
            p = O.Params(N, N, N, lam=3.0, dt=0.02, stencil=26, n=(1.0, 0.0, 0.0), M=M, Gamma=G)
            _, dF = O.step_conserving(p, O.init_sphere(p, ((N - 1) / 2.0,) * 3, R), 1)
            errs.append(abs(dF[0] / (2 * G / R) - 1))
    assert abs(errs[0] - errs[1]) < 1e-12 and abs(errs[2] - errs[3]) < 1e-12
    assert errs[0] < 0.015 and errs[2] < 0.004 and errs[0] > 3.0 * errs[2]


def test_ti_hkl_restores_ti_for_the_whole_family():
    """Tab. 2: with couplings a_k(u), u || <hkl>, TI holds for every interface
    normal of the <hkl> family (the potential's sum over directions depends only
    on the multiset of (w_k, |a_k|), which the cubic symmetries of the stencil
    preserve), not for other normals."""
    u = _unit([1, 2, 0])
    for n, fixed in ((_unit([2, 0, 1]), True), (_unit([0, -1, 2]), True), (_unit([1, 1, 0]), False)):
        p = O.Params(26, 18, 16, bc=(O.CONTACT,) * 6, n=tuple(n), u=tuple(u), lam=2.0, stencil=26)
        phi = O.init_planar(p, float(n @ [12.5, 8.5, 7.5]))
        R, _ = O.rhs(p, phi)
        assert (np.abs(R).max() < 1e-12) == fixed, (n, np.abs(R).max())
