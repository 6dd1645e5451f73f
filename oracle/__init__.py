"""FP64 CPU oracle of the sharp phase-field method (arXiv:1910.05180).

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only code allowed to import this
package.  The CUDA library never imports, links or calls it.

The arithmetic lives in ``spfm_oracle.c`` (plain C, double precision, one cell
and one grid direction at a time, written from Eqs. 1-10 of the paper).  This
module compiles it with gcc on first use and marshals numpy arrays of shape
``(nz, ny, nx)`` (x fastest) through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spfm_oracle.c")
_HDR = os.path.join(_HERE, "spfm_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libspfm_oracle.so")
_lock = threading.Lock()
_lib = None

PERIODIC, NOFLUX, CONTACT = 0, 1, 2
TI_GLOBAL, TI_LOCAL, CF = 0, 1, 2
CF_H5, CF_HABEL = 3, 4   # CF with the interpolation functions h5 and h_Abel (Tab. 2)


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/libspfm_oracle.so (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("bc", ctypes.c_int * 6),
        ("n", ctypes.c_double * 3),
        ("gamma", ctypes.c_double * 3),
        ("C_gamma", ctypes.c_double),
        ("M", ctypes.c_double), ("Gamma", ctypes.c_double),
        ("lam", ctypes.c_double), ("dx", ctypes.c_double),
        ("dt", ctypes.c_double), ("dF", ctypes.c_double),
        ("stencil", ctypes.c_int), ("scheme", ctypes.c_int),
        ("eps_local", ctypes.c_double),
        ("u", ctypes.c_double * 3),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER(_Params)
            dp = ctypes.POINTER(ctypes.c_double)
            lib.oracle_directions.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
            lib.oracle_weights.argtypes = [P, dp, dp]
            lib.oracle_coupling.argtypes = [dp, ctypes.c_double, ctypes.c_double, dp]
            lib.oracle_init_planar.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp,
                                               ctypes.c_double, ctypes.c_double, ctypes.c_double]
            lib.oracle_init_sphere.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp,
                                               ctypes.c_double, ctypes.c_double, ctypes.c_double]
            lib.oracle_fill_ghosts.argtypes = [P, dp, dp]
            lib.oracle_rhs.argtypes = [P, dp, dp]
            lib.oracle_rhs.restype = ctypes.c_long
            lib.oracle_step.argtypes = [P, dp, ctypes.c_int]
            lib.oracle_step.restype = ctypes.c_long
            lib.oracle_step_conserving.argtypes = [P, dp, ctypes.c_int, dp]
            lib.oracle_shift_x.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            lib.oracle_step_conserving.restype = ctypes.c_long
            lib.oracle_init_cube.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_double]
            lib.oracle_stats.argtypes = [P, dp, dp, dp]
            lib.oracle_energy.argtypes = [P, dp]
            lib.oracle_energy.restype = ctypes.c_double
            lib.oracle_contour.argtypes = [P, dp, ctypes.c_double, dp, ctypes.c_long]
            lib.oracle_contour.restype = ctypes.c_long
            _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass
class Params:
    """Grid, boundary kinds and model parameters of one oracle run."""
    nx: int
    ny: int
    nz: int
    bc: tuple = (PERIODIC,) * 6
    n: tuple = (1.0, 0.0, 0.0)
    gamma: tuple = (0.0, 0.0, 0.0)
    C_gamma: float = 0.0
    M: float = 1.0
    Gamma: float = 1.0
    lam: float = 4.0
    dx: float = 1.0
    dt: float = 0.1
    dF: float = 0.0
    stencil: int = 6
    scheme: int = TI_GLOBAL
    eps_local: float = 0.0
    u: tuple = (0.0, 0.0, 0.0)   # TI_<hkl> coupling direction; all zero: n
    extra: dict = field(default_factory=dict)

    def c(self) -> _Params:
        p = _Params()
        p.nx, p.ny, p.nz = self.nx, self.ny, self.nz
        for i in range(6):
            p.bc[i] = int(self.bc[i])
        for i in range(3):
            p.n[i] = float(self.n[i])
            p.gamma[i] = float(self.gamma[i])
        p.C_gamma = self.C_gamma
        p.M, p.Gamma, p.lam, p.dx = self.M, self.Gamma, self.lam, self.dx
        p.dt, p.dF = self.dt, self.dF
        p.stencil, p.scheme = self.stencil, self.scheme
        p.eps_local = self.eps_local
        for i in range(3):
            p.u[i] = float(self.u[i])
        return p

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)


def directions():
    """(13, 3) integer grid vectors of Tab. 1 and their shell numbers."""
    lib = _load()
    d = (ctypes.c_int * 39)()
    s = (ctypes.c_int * 13)()
    lib.oracle_directions(d, s)
    return np.array(list(d), dtype=np.int64).reshape(13, 3), np.array(list(s), dtype=np.int64)


def weights(p: Params):
    """w_k = gamma_j nu_j for the 13 directions (0 where inactive) and gamma used."""
    lib = _load()
    w = np.zeros(13)
    g = np.zeros(3)
    pc = p.c()
    lib.oracle_weights(ctypes.byref(pc), _dp(w), _dp(g))
    return w, g


def coupling(u, lam: float, dx: float) -> np.ndarray:
    """a_k(u) = tanh(2 r_k.u/lambda) for k = 0..12 (Eq. 5)."""
    lib = _load()
    uu = np.ascontiguousarray(u, dtype=np.float64)
    a = np.zeros(13)
    lib.oracle_coupling(_dp(uu), lam, dx, _dp(a))
    return a


def init_planar(p: Params, c: float) -> np.ndarray:
    lib = _load()
    phi = np.zeros(p.shape)
    n = np.ascontiguousarray(p.n, dtype=np.float64)
    lib.oracle_init_planar(_dp(phi), p.nx, p.ny, p.nz, _dp(n), c, p.lam, p.dx)
    return phi


def init_sphere(p: Params, ctr, R: float) -> np.ndarray:
    lib = _load()
    phi = np.zeros(p.shape)
    cc = np.ascontiguousarray(ctr, dtype=np.float64)
    lib.oracle_init_sphere(_dp(phi), p.nx, p.ny, p.nz, _dp(cc), R, p.lam, p.dx)
    return phi


def init_cube(p: Params, ctr, half: float) -> np.ndarray:
    """Cubic particle (phi = 0 inside) of half side `half`: the product of three
    1D ideal profiles (the cube start of the Sec. 3.3 shape relaxation)."""
    lib = _load()
    phi = np.zeros(p.shape)
    cc = np.ascontiguousarray(ctr, dtype=np.float64)
    lib.oracle_init_cube(_dp(phi), p.nx, p.ny, p.nz, _dp(cc), half, p.lam, p.dx)
    return phi


def _field(p: Params, phi) -> np.ndarray:
    a = np.ascontiguousarray(phi, dtype=np.float64)
    assert a.shape == p.shape, (a.shape, p.shape)
    return a


def fill_ghosts(p: Params, phi) -> np.ndarray:
    lib = _load()
    a = _field(p, phi)
    pad = np.zeros((p.nz + 2, p.ny + 2, p.nx + 2))
    pc = p.c()
    lib.oracle_fill_ghosts(ctypes.byref(pc), _dp(a), _dp(pad))
    return pad


def rhs(p: Params, phi):
    """dphi/dt at every cell; returns (R, number of cells with undefined potential)."""
    lib = _load()
    a = _field(p, phi)
    R = np.zeros(p.shape)
    pc = p.c()
    nbad = lib.oracle_rhs(ctypes.byref(pc), _dp(a), _dp(R))
    return R, int(nbad)


def step_conserving(p: Params, phi, n_steps: int):
    """n_steps constant-volume steps (Sec. 3.3): each step's homogeneous dF is
    the one that leaves sum(phi) unchanged.  Returns (field, dF per step)."""
    lib = _load()
    a = _field(p, phi).copy()
    dF = np.zeros(max(int(n_steps), 1))
    pc = p.c()
    lib.oracle_step_conserving(ctypes.byref(pc), _dp(a), int(n_steps), _dp(dF))
    return a, dF[:int(n_steps)]


def shift_x(p: Params, phi, cells: int) -> np.ndarray:
    """The moving frame of the 1D friction study: phi_i <- phi_{i+cells}, the
    vacated cells taking the value of the row's end cell."""
    lib = _load()
    a = _field(p, phi).copy()
    lib.oracle_shift_x(_dp(a), p.nx, p.ny, p.nz, int(cells))
    return a


def step(p: Params, phi, n_steps: int) -> np.ndarray:
    """n_steps forward-Euler steps; returns the new field (input untouched)."""
    lib = _load()
    a = _field(p, phi).copy()
    pc = p.c()
    lib.oracle_step(ctypes.byref(pc), _dp(a), int(n_steps))
    return a


STATS_KEYS = ("volume", "S_w", "S_c", "S_r", "phi_min", "phi_max", "nonfinite",
              "position", "radius")


def stats(p: Params, phi, ctr=(0.0, 0.0, 0.0)) -> dict:
    lib = _load()
    a = _field(p, phi)
    out = np.zeros(9)
    cc = np.ascontiguousarray(ctr, dtype=np.float64)
    pc = p.c()
    lib.oracle_stats(ctypes.byref(pc), _dp(a), _dp(cc), _dp(out))
    return dict(zip(STATS_KEYS, out.tolist()))


def energy(p: Params, phi) -> float:
    lib = _load()
    a = _field(p, phi)
    pc = p.c()
    return float(lib.oracle_energy(ctypes.byref(pc), _dp(a)))


def contour(p: Params, phi, level: float = 0.5) -> np.ndarray:
    """phi = level contour points (N, 3) by the nonlinear interpolation of Sec. 2.3."""
    lib = _load()
    a = _field(p, phi)
    pc = p.c()
    n = lib.oracle_contour(ctypes.byref(pc), _dp(a), level, None, 0)
    pts = np.zeros((max(n, 1), 3))
    lib.oracle_contour(ctypes.byref(pc), _dp(a), level, _dp(pts), n)
    return pts[:n]


def sphericity(p: Params, phi, inside_phase: int = 0) -> dict:
    """eps_eff = (R_max - R_min) / (2 R_mean) of the phi = 1/2 contour points around
    the particle's barycentre (Sec. 3.3); the particle is the phase
    ``inside_phase`` and its barycentre is weighted by its phase fraction."""
    a = _field(p, phi)
    pts = contour(p, a, 0.5)
    wgt = (1.0 - a) if inside_phase == 0 else a
    k, j, i = np.meshgrid(np.arange(p.nz), np.arange(p.ny), np.arange(p.nx), indexing="ij")
    tot = wgt.sum()
    bary = np.array([(wgt * i).sum(), (wgt * j).sum(), (wgt * k).sum()]) * p.dx / tot
    R = np.sqrt(((pts - bary) ** 2).sum(axis=1))
    return {"eps_eff": float((R.max() - R.min()) / (2.0 * R.mean())),
            "R_mean": float(R.mean()), "R_min": float(R.min()), "R_max": float(R.max()),
            "n_points": int(len(R)), "barycentre": bary.tolist()}
