"""Thin Python binding of the C ABI in include/spfm.h.

Argument marshalling only: every step of the computation runs in the CUDA
library ``_build/libspfm_gb300.so``.  PyTorch supplies device memory and the
CUDA stream.  Importing this module does not build anything; loading the
library fails loudly when it has not been built (there is no CPU fallback).

The functions keep the C names (``spfm_create_grid``, ``spfm_step``,
``spfm_interface_stats`` ...).  ``Grid`` bundles a handle with the torch
buffers it borrows so they stay alive as long as the handle.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
# SPFM_LIBRARY may point at another build of the same library (same ABI)
LIB_PATH = os.environ.get("SPFM_LIBRARY") or os.path.join(HERE, "_build", "libspfm_gb300.so")

SPFM_OK, SPFM_EINVAL, SPFM_EUNSTABLE, SPFM_EPHASE = 0, -1, -2, -3
SPFM_ECUDA, SPFM_ENONFINITE, SPFM_ETIMEOUT, SPFM_ENOMEM = -4, -5, -6, -7
SPFM_F64, SPFM_F32, SPFM_BF16 = 0, 1, 2
SPFM_PERIODIC, SPFM_NOFLUX, SPFM_CONTACT = 0, 1, 2
SPFM_TI_GLOBAL, SPFM_TI_LOCAL, SPFM_FD = 0, 1, 2
SPFM_FD_H5, SPFM_FD_HABEL = 3, 4   # CF with the interpolation functions h5 and h_Abel (Tab. 2)
SPFM_STATS_ENERGY = 1
SPFM_TILES_WIDE, SPFM_TILES_SQUARE, SPFM_TILES_FIT = 0, 1, 2   # batch tile policies
SPFM_ROUND_NEAREST, SPFM_ROUND_STOCHASTIC = 0, 1                 # rounding of the update

TORCH_DTYPE = {SPFM_F64: torch.float64, SPFM_F32: torch.float32, SPFM_BF16: torch.bfloat16}
STATUS_NAME = {0: "SPFM_OK", -1: "SPFM_EINVAL", -2: "SPFM_EUNSTABLE", -3: "SPFM_EPHASE",
               -4: "SPFM_ECUDA", -5: "SPFM_ENONFINITE", -6: "SPFM_ETIMEOUT", -7: "SPFM_ENOMEM"}


class SpfmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAME.get(status, status)}: {msg}")
        self.status = status


class GridDesc(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("dtype", ctypes.c_int),
        ("bc", ctypes.c_int * 6),
        ("n", ctypes.c_double * 3),
        ("gamma", ctypes.c_double * 3),
        ("C_gamma", ctypes.c_double),
        ("center", ctypes.c_double * 3),
        ("field", ctypes.c_void_p * 2),
        ("scratch", ctypes.c_void_p),
        ("scratch_bytes", ctypes.c_size_t),
        ("stream", ctypes.c_void_p),
        ("u", ctypes.c_double * 3),
    ]


class Stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in (
        "volume", "S_w", "S_c", "S_r", "phi_min", "phi_max", "nonfinite", "position",
        "radius", "energy", "steps", "time")]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class StepArgs(ctypes.Structure):
    _fields_ = [("M", ctypes.c_double), ("Gamma", ctypes.c_double), ("lam", ctypes.c_double),
                ("dx", ctypes.c_double), ("dt", ctypes.c_double), ("dF", ctypes.c_double),
                ("stencil", ctypes.c_int), ("scheme", ctypes.c_int)]


_lib = None
_lock = threading.Lock()

# (name, restype, argtypes) of every exported entry point of include/spfm.h
_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
SIGNATURES = [
    ("spfm_layout", _I, [ctypes.POINTER(GridDesc), ctypes.POINTER(ctypes.c_size_t),
                         ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t),
                         ctypes.POINTER(ctypes.c_size_t)]),
    ("spfm_create_grid", _I, [ctypes.POINTER(GridDesc), ctypes.POINTER(_P)]),
    ("spfm_destroy_grid", _I, [_P]),
    ("spfm_set_stream", _I, [_P, _P]),
    ("spfm_init_planar", _I, [_P, _D, _D, _D]),
    ("spfm_init_sphere", _I, [_P, ctypes.POINTER(_D), _D, _D, _D]),
    ("spfm_init_cube", _I, [_P, ctypes.POINTER(_D), _D, _D, _D]),
    ("spfm_step", _I, [_P, _I, _D, _D, _D, _D, _D, _D, _I, _I]),
    ("spfm_step_conserving", _I, [_P, _I, _D, _D, _D, _D, _D, _I, _I, ctypes.POINTER(_D)]),
    ("spfm_set_rounding", _I, [_P, _I, ctypes.c_ulonglong]),
    ("spfm_debug_skip_copy", _I, [_P]),
    ("spfm_set_zchunk", _I, [_P, _I]),
    ("spfm_last_zchunk", _I, [_P]),
    ("spfm_debug_pick_zchunk", _I, [_I, _I, _I, _I, _I]),
    ("spfm_shift_x", _I, [_P, _I]),
    ("spfm_max_dt", _I, [_P, _D, _D, _D, _D, _D, _I, _I, ctypes.POINTER(_D)]),
    ("spfm_interface_stats", _I, [_P, _I, ctypes.POINTER(Stats)]),
    ("spfm_interface_stats_static", _I, [ctypes.POINTER(GridDesc), _P, _D, _D, ctypes.POINTER(Stats)]),
    ("spfm_sphericity", _I, [_P, _I, ctypes.POINTER(_D)]),
    ("spfm_get_field", _I, [_P, _P, _I]),
    ("spfm_set_field", _I, [_P, _P, _I]),
    ("spfm_current", _I, [_P]),
    ("spfm_kernels_per_step", _I, [_P]),
    ("spfm_last_error", ctypes.c_char_p, [_P]),
    ("spfm_batch_scratch_bytes", _I, [ctypes.POINTER(_P), _I, ctypes.POINTER(ctypes.c_size_t)]),
    ("spfm_batch_create", _I, [ctypes.POINTER(_P), _I, _P, ctypes.c_size_t, _P, ctypes.POINTER(_P)]),
    ("spfm_batch_step", _I, [_P, _I, ctypes.POINTER(StepArgs)]),
    ("spfm_batch_autotune", _I, [_P, ctypes.POINTER(StepArgs), _I, ctypes.POINTER(ctypes.c_int),
                                 ctypes.POINTER(ctypes.c_double)]),
    ("spfm_batch_set_tiles", _I, [_P, _I]),
    ("spfm_batch_tiles", _I, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    ("spfm_batch_stats", _I, [_P, _I, ctypes.POINTER(Stats)]),
    ("spfm_batch_destroy", _I, [_P]),
]


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(
                    f"SPFM CUDA library not built ({path}); run paper_1910_05180_gb300.build.build()")
            lib = ctypes.CDLL(path)
            for name, res, args in SIGNATURES:
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(status: int, handle=None):
    if status != SPFM_OK:
        msg = load().spfm_last_error(handle)
        raise SpfmError(status, msg.decode() if msg else "")
    return status


# ------------------------------------------------------------- C-named calls

def spfm_layout(desc: GridDesc):
    """(pitch_x, x_off, field_bytes, scratch_bytes) of a grid."""
    px, xo, fb, sb = (ctypes.c_size_t() for _ in range(4))
    _check(load().spfm_layout(ctypes.byref(desc), ctypes.byref(px), ctypes.byref(xo),
                              ctypes.byref(fb), ctypes.byref(sb)))
    return px.value, xo.value, fb.value, sb.value


def spfm_create_grid(desc: GridDesc):
    h = ctypes.c_void_p()
    _check(load().spfm_create_grid(ctypes.byref(desc), ctypes.byref(h)))
    return h


def spfm_destroy_grid(h):
    _check(load().spfm_destroy_grid(h))


def spfm_set_stream(h, stream):
    _check(load().spfm_set_stream(h, stream), h)


def spfm_set_rounding(h, mode, seed=0):
    _check(load().spfm_set_rounding(h, int(mode), int(seed) & 0xFFFFFFFFFFFFFFFF), h)


def spfm_debug_skip_copy(h):
    _check(load().spfm_debug_skip_copy(h), h)


def spfm_set_zchunk(h, zchunk):
    _check(load().spfm_set_zchunk(h, int(zchunk)), h)


def spfm_init_planar(h, c, lam, dx):
    _check(load().spfm_init_planar(h, c, lam, dx), h)


def spfm_init_sphere(h, ctr, R, lam, dx):
    arr = (ctypes.c_double * 3)(*ctr)
    _check(load().spfm_init_sphere(h, arr, R, lam, dx), h)


def spfm_init_cube(h, ctr, half, lam, dx):
    arr = (ctypes.c_double * 3)(*ctr)
    _check(load().spfm_init_cube(h, arr, half, lam, dx), h)


def spfm_step(h, n_steps, M, Gamma, lam, dx, dt, dF, stencil, scheme):
    _check(load().spfm_step(h, int(n_steps), M, Gamma, lam, dx, dt, dF, int(stencil), int(scheme)), h)


def spfm_shift_x(h, cells):
    _check(load().spfm_shift_x(h, int(cells)), h)


def spfm_max_dt(h, M, Gamma, lam, dx, dF, stencil, scheme):
    out = ctypes.c_double(0.0)
    _check(load().spfm_max_dt(h, M, Gamma, lam, dx, dF, int(stencil), int(scheme), ctypes.byref(out)), h)
    return out.value


def spfm_step_conserving(h, n_steps, M, Gamma, lam, dx, dt, stencil, scheme):
    dF = ctypes.c_double(0.0)
    _check(load().spfm_step_conserving(h, int(n_steps), M, Gamma, lam, dx, dt, int(stencil), int(scheme),
                                       ctypes.byref(dF)), h)
    return dF.value


def spfm_interface_stats(h, flags=0, allow_nonfinite=False) -> dict:
    st = Stats()
    s = load().spfm_interface_stats(h, int(flags), ctypes.byref(st))
    if not (allow_nonfinite and s == SPFM_ENONFINITE):
        _check(s, h)
    return st.as_dict()


def spfm_interface_stats_static(desc, field_ptr, lam, dx, allow_nonfinite=False) -> dict:
    """Diagnostics of a borrowed field buffer without any device allocation."""
    st = Stats()
    s = load().spfm_interface_stats_static(ctypes.byref(desc), field_ptr, lam, dx, ctypes.byref(st))
    if not (allow_nonfinite and s == SPFM_ENONFINITE):
        _check(s)
    return st.as_dict()


def spfm_sphericity(h, inside_phase=0) -> dict:
    out = (ctypes.c_double * 8)()
    _check(load().spfm_sphericity(h, int(inside_phase), out), h)
    return {"eps_eff": out[0], "R_mean": out[1], "R_min": out[2], "R_max": out[3],
            "n_points": int(out[4]), "barycentre": [out[5], out[6], out[7]]}


def spfm_get_field(h, ptr, on_host):
    _check(load().spfm_get_field(h, ptr, int(on_host)), h)


def spfm_set_field(h, ptr, on_host):
    _check(load().spfm_set_field(h, ptr, int(on_host)), h)


def spfm_current(h) -> int:
    return load().spfm_current(h)


def spfm_kernels_per_step(h) -> int:
    return load().spfm_kernels_per_step(h)


def spfm_last_error(h=None) -> str:
    m = load().spfm_last_error(h)
    return m.decode() if m else ""


# ------------------------------------------------------------------ helpers

class Grid:
    """One grid: a handle plus the torch buffers (two fields, scratch) it borrows."""

    def __init__(self, nx, ny, nz, dtype=SPFM_F32, bc=(SPFM_PERIODIC,) * 6, n=(1.0, 0.0, 0.0),
                 gamma=(0.0, 0.0, 0.0), C_gamma=0.0, center=(0.0, 0.0, 0.0), device="cuda",
                 stream=None, u=(0.0, 0.0, 0.0)):
        d = GridDesc()
        d.nx, d.ny, d.nz, d.dtype = int(nx), int(ny), int(nz), int(dtype)
        for i in range(6):
            d.bc[i] = int(bc[i])
        for i in range(3):
            d.n[i], d.gamma[i], d.center[i] = float(n[i]), float(gamma[i]), float(center[i])
            d.u[i] = float(u[i])
        d.C_gamma = float(C_gamma)
        pitch, xoff, fbytes, sbytes = spfm_layout(d)
        self.pitch, self.x_off, self.field_bytes, self.scratch_bytes = pitch, xoff, fbytes, sbytes
        tdt = TORCH_DTYPE[dtype]
        self.shape = (int(nz), int(ny), int(nx))
        # ghosted buffers: (nz + 2, ny + 2, pitch), interior at [1:-1, 1:-1, x_off:x_off+nx]
        self.fields = [torch.zeros((nz + 2, ny + 2, pitch), dtype=tdt, device=device) for _ in range(2)]
        self.scratch = torch.empty(max(sbytes, 16), dtype=torch.uint8, device=device)
        for b in range(2):
            d.field[b] = self.fields[b].data_ptr()
        d.scratch = self.scratch.data_ptr()
        d.scratch_bytes = self.scratch.numel()
        st = stream if stream is not None else torch.cuda.current_stream()
        self.stream = st
        d.stream = st.cuda_stream
        self.desc = d
        self.dtype = dtype
        self.handle = spfm_create_grid(d)

    def close(self):
        if getattr(self, "handle", None) is not None:
            spfm_destroy_grid(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # marshalling wrappers
    def init_planar(self, c, lam, dx=1.0):
        spfm_init_planar(self.handle, c, lam, dx)

    def init_sphere(self, ctr, R, lam, dx=1.0):
        spfm_init_sphere(self.handle, ctr, R, lam, dx)

    def init_cube(self, ctr, half, lam, dx=1.0):
        spfm_init_cube(self.handle, ctr, half, lam, dx)

    def step(self, n_steps, M=1.0, Gamma=1.0, lam=4.0, dx=1.0, dt=0.1, dF=0.0, stencil=26,
             scheme=SPFM_TI_GLOBAL):
        spfm_step(self.handle, n_steps, M, Gamma, lam, dx, dt, dF, stencil, scheme)

    def set_rounding(self, mode, seed=0):
        """SPFM_ROUND_NEAREST or SPFM_ROUND_STOCHASTIC (FP32/BF16) for the following steps."""
        spfm_set_rounding(self.handle, mode, seed)

    def set_zchunk(self, zchunk):
        """Planes per CTA of the step launches (0: chosen per launch); the field is the same for any."""
        spfm_set_zchunk(self.handle, zchunk)

    def last_zchunk(self):
        """Planes per CTA of the last step launch (0 before the first step)."""
        return int(load().spfm_last_zchunk(self.handle))

    def shift_x(self, cells):
        """Moving frame: phi_i <- phi_{i+cells} (end cells repeated)."""
        spfm_shift_x(self.handle, cells)

    def max_dt(self, M=1.0, Gamma=1.0, lam=4.0, dx=1.0, dF=0.0, stencil=26, scheme=SPFM_TI_GLOBAL):
        return spfm_max_dt(self.handle, M, Gamma, lam, dx, dF, stencil, scheme)

    def step_conserving(self, n_steps, M=1.0, Gamma=1.0, lam=4.0, dx=1.0, dt=0.1, stencil=26,
                        scheme=SPFM_TI_GLOBAL):
        """Constant-volume steps (Sec. 3.3); returns the last step's dF."""
        return spfm_step_conserving(self.handle, n_steps, M, Gamma, lam, dx, dt, stencil, scheme)

    def stats(self, flags=0, allow_nonfinite=False) -> dict:
        return spfm_interface_stats(self.handle, flags, allow_nonfinite)

    def sphericity(self, inside_phase=0) -> dict:
        return spfm_sphericity(self.handle, inside_phase)

    def kernels_per_step(self) -> int:
        """1 when the step kernel writes the periodic ghost images itself, else 2."""
        return spfm_kernels_per_step(self.handle)

    def current(self) -> torch.Tensor:
        """View (nz, ny, nx) of the interior of the buffer holding the current field."""
        buf = self.fields[spfm_current(self.handle)]
        return buf[1:-1, 1:-1, self.x_off: self.x_off + self.shape[2]]

    def current_with_ghosts(self) -> torch.Tensor:
        """View (nz+2, ny+2, nx+2) of the current buffer including the ghost layer."""
        buf = self.fields[spfm_current(self.handle)]
        return buf[:, :, self.x_off - 1: self.x_off + self.shape[2] + 1]

    def get_field(self, to_host=True) -> torch.Tensor:
        """Dense copy of the current field through spfm_get_field."""
        tdt = TORCH_DTYPE[self.dtype]
        if to_host:
            out = torch.empty(self.shape, dtype=tdt, pin_memory=True)
        else:
            out = torch.empty(self.shape, dtype=tdt, device=self.fields[0].device)
        spfm_get_field(self.handle, out.data_ptr(), 1 if to_host else 0)
        return out

    def set_field(self, src: torch.Tensor):
        src = src.contiguous()
        assert tuple(src.shape) == self.shape and src.dtype == TORCH_DTYPE[self.dtype]
        spfm_set_field(self.handle, src.data_ptr(), 0 if src.is_cuda else 1)


# ------------------------------------------------------------------ batches

def spfm_batch_scratch_bytes(handles) -> int:
    arr = (ctypes.c_void_p * len(handles))(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    n = ctypes.c_size_t()
    _check(load().spfm_batch_scratch_bytes(arr, len(handles), ctypes.byref(n)))
    return n.value


def spfm_batch_create(handles, scratch_ptr, scratch_bytes, stream):
    arr = (ctypes.c_void_p * len(handles))(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    b = ctypes.c_void_p()
    _check(load().spfm_batch_create(arr, len(handles), scratch_ptr, scratch_bytes, stream, ctypes.byref(b)))
    return b


def spfm_batch_step(b, n_steps, args):
    arr = (StepArgs * len(args))(*args)
    _check(load().spfm_batch_step(b, int(n_steps), arr))


BATCH_DEPTHS = (8, 12, 16, 24, 32, 48, 64)   # z-march depths the autotuner tries


def spfm_batch_set_tiles(b, policy):
    _check(load().spfm_batch_set_tiles(b, int(policy)))


def spfm_batch_tiles(b):
    policy, depth = ctypes.c_int(0), ctypes.c_int(0)
    _check(load().spfm_batch_tiles(b, ctypes.byref(policy), ctypes.byref(depth)))
    return policy.value, depth.value


def spfm_batch_autotune(b, args, steps_per_trial=32):
    arr = (StepArgs * len(args))(*args)
    depth = ctypes.c_int(0)
    ms = (ctypes.c_double * len(BATCH_DEPTHS))()
    _check(load().spfm_batch_autotune(b, arr, int(steps_per_trial), ctypes.byref(depth), ms))
    return depth.value, dict(zip(BATCH_DEPTHS, list(ms)))


def spfm_batch_stats(b, n, flags=0, allow_nonfinite=False):
    arr = (Stats * n)()
    s = load().spfm_batch_stats(b, int(flags), arr)
    if not (allow_nonfinite and s == SPFM_ENONFINITE):
        _check(s)
    return [st.as_dict() for st in arr]


def spfm_batch_destroy(b):
    _check(load().spfm_batch_destroy(b))


def step_args(M=1.0, Gamma=1.0, lam=4.0, dx=1.0, dt=0.1, dF=0.0, stencil=26,
              scheme=SPFM_TI_GLOBAL) -> StepArgs:
    a = StepArgs()
    a.M, a.Gamma, a.lam, a.dx, a.dt, a.dF = M, Gamma, lam, dx, dt, dF
    a.stencil, a.scheme = int(stencil), int(scheme)
    return a


class Batch:
    """Grids of one dtype stepped together (one persistent launch per step)."""

    def __init__(self, grids, stream=None):
        self.grids = list(grids)
        handles = [g.handle for g in self.grids]
        nbytes = spfm_batch_scratch_bytes(handles)
        dev = self.grids[0].fields[0].device
        self.scratch = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=dev)
        st = stream if stream is not None else self.grids[0].stream
        self.stream = st
        self.handle = spfm_batch_create(handles, self.scratch.data_ptr(), self.scratch.numel(), st.cuda_stream)

    def step(self, n_steps, args):
        spfm_batch_step(self.handle, n_steps, args)

    def autotune(self, args, steps_per_trial=32):
        """Pick the tile policy (FP32) and then the work-list depth by timing each
        candidate on real steps (the grids advance by (3 + len(BATCH_DEPTHS)) *
        (16 + steps_per_trial) steps for FP32).  Returns (depth, {depth: ms per
        step}); tiles() gives the policy kept."""
        return spfm_batch_autotune(self.handle, args, steps_per_trial)

    def set_tiles(self, policy):
        """SPFM_TILES_WIDE, SPFM_TILES_SQUARE or SPFM_TILES_FIT (the fields do not depend on it)."""
        spfm_batch_set_tiles(self.handle, policy)

    def tiles(self):
        """(tile policy, z-march depth) of the work-list."""
        return spfm_batch_tiles(self.handle)

    def stats(self, flags=0, allow_nonfinite=False):
        return spfm_batch_stats(self.handle, len(self.grids), flags, allow_nonfinite)

    def close(self):
        if getattr(self, "handle", None) is not None:
            spfm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
