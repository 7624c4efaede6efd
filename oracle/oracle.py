"""ctypes wrapper of the plain FP64 CPU oracle (``lbve_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the CPU
baseline of the benchmark may import this module; the product path never
does.  It imports nothing from the CUDA package and the CUDA package
imports nothing from here.

Fields are numpy float64 arrays laid out [component][y][x] (row-major, x
fastest), the same convention the oracle's C code uses.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbve_oracle.c")
_LIB = os.path.join(_HERE, "liblbve_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction)."""
    with _lock:
        stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
        if force or stale:
            tmp = _LIB + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
                   "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("periodic_y", ctypes.c_int32), ("open_x", ctypes.c_int32),
                ("beta", ctypes.c_double), ("Wi", ctypes.c_double), ("Re", ctypes.c_double),
                ("Sc", ctypes.c_double), ("Ma", ctypes.c_double), ("Lc", ctypes.c_double),
                ("Lambda_s", ctypes.c_double), ("Lambda_p", ctypes.c_double),
                ("Fx", ctypes.c_double), ("Fy", ctypes.c_double),
                ("model", ctypes.c_int32), ("gtilde", ctypes.c_int32), ("L2", ctypes.c_double)]


class Coeffs(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in
                ("Uc", "nu0", "nus", "mup", "tau_s1", "tau_s2", "kappa", "tau_p1",
                 "tau_p2", "lambda_")]


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.orc_create.restype = ctypes.c_void_p
        L.orc_create.argtypes = [ctypes.POINTER(Params), _dp, _dp]
        L.orc_destroy.argtypes = [ctypes.c_void_p]
        L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_int64]
        L.orc_fields.argtypes = [ctypes.c_void_p, _dp]
        L.orc_totals.argtypes = [ctypes.c_void_p, _dp]
        L.orc_get_source.argtypes = [ctypes.c_void_p, _dp]
        L.orc_get_state.argtypes = [ctypes.c_void_p, _dp, _dp]
        L.orc_set_state.argtypes = [ctypes.c_void_p, _dp, _dp]
        L.orc_get_coeffs.argtypes = [ctypes.c_void_p, ctypes.POINTER(Coeffs)]
        L.orc_set_inlet.restype = ctypes.c_int
        L.orc_set_inlet.argtypes = [ctypes.c_void_p, _dp]
        L.orc_set_mask.restype = ctypes.c_int
        L.orc_set_mask.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint8), _dp]
        L.orc_time.restype = ctypes.c_int64
        L.orc_time.argtypes = [ctypes.c_void_p]
        L.orc_derive.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(Coeffs)]
        L.orc_feq.argtypes = [ctypes.c_double] * 3 + [_dp]
        L.orc_geq.argtypes = [ctypes.c_double] * 3 + [_dp]
        L.orc_hydro_moments.argtypes = [_dp, ctypes.c_double, ctypes.c_double, _dp, _dp, _dp]
        L.orc_hydro_collide.argtypes = [_dp, ctypes.c_double, ctypes.c_double, _dp, _dp,
                                        ctypes.c_double, ctypes.c_double, _dp]
        L.orc_cde_collide.argtypes = ([_dp] + [ctypes.c_double] * 11 + [_dp])
        L.orc_source.argtypes = [_dp, _dp, ctypes.c_double, _dp]
        L.orc_source_model.argtypes = [_dp, _dp, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                       _dp]
        L.orc_model_F.argtypes = [_dp, ctypes.c_int, ctypes.c_double, _dp]
        L.orc_zou_he.argtypes = [_dp, ctypes.c_double, ctypes.c_double, ctypes.c_int]
        L.orc_cnebb.argtypes = [_dp, _dp, _ip, ctypes.c_double, ctypes.c_double, _dp, _dp]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def make_params(nx, ny, periodic_y=True, beta=0.5, Wi=1.0, Re=1.0, Sc=1e5, Ma=0.1, Lc=None,
                Lambda_s=0.25, Lambda_p=1e-6, Fx=0.0, Fy=0.0, open_x=False, model=0, gtilde=0,
                L2=0.0) -> Params:
    if Lc is None:
        Lc = float(ny - 1) if not periodic_y else float(nx) / (2 * np.pi)
    return Params(nx, ny, 1 if periodic_y else 0, 1 if open_x else 0, beta, Wi, Re, Sc, Ma, Lc, Lambda_s,
                  Lambda_p, Fx, Fy, model, gtilde, L2)


def derive(p: Params) -> dict:
    c = Coeffs()
    lib().orc_derive(ctypes.byref(p), ctypes.byref(c))
    d = {k: getattr(c, k) for k, _ in Coeffs._fields_}
    d["lambda"] = d.pop("lambda_")
    return d


class Sim:
    """One oracle simulation (see ``lbve_oracle.c`` for the algorithm)."""

    def __init__(self, p: Params, force: np.ndarray | None = None,
                 init: np.ndarray | None = None):
        self.p = p
        self.nx, self.ny = p.nx, p.ny
        n = p.nx * p.ny
        self._force = None if force is None else np.ascontiguousarray(force, np.float64).reshape(2, n)
        self._init = None if init is None else np.ascontiguousarray(init, np.float64).reshape(6, n)
        h = lib().orc_create(ctypes.byref(p),
                             _ptr(self._force) if self._force is not None else None,
                             _ptr(self._init) if self._init is not None else None)
        if not h:
            raise ValueError("oracle rejected the parameters")
        self._h = ctypes.c_void_p(h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().orc_destroy(h)
            self._h = None

    def step(self, n: int = 1) -> None:
        lib().orc_step(self._h, int(n))

    @property
    def t(self) -> int:
        return int(lib().orc_time(self._h))

    def fields(self) -> np.ndarray:
        out = np.empty((6, self.ny, self.nx))
        lib().orc_fields(self._h, _ptr(out))
        return out

    def totals(self) -> np.ndarray:
        """[0:3] sum rho, rho ux, rho uy; [3:6] sum phi; [6:9] / [9:12] CNEBB wall
        in / out per lattice; [12:14] force on the solid mask (last step)."""
        out = np.empty(14)
        lib().orc_totals(self._h, _ptr(out))
        return out

    def set_inlet(self, inlet: np.ndarray) -> None:
        """Inlet profile [5][ny] = u_x, u_y, A_xx, A_xy, A_yy (open channels)."""
        a = np.ascontiguousarray(inlet, np.float64).reshape(5, self.ny)
        if lib().orc_set_inlet(self._h, _ptr(a)) != 0:
            raise ValueError("the domain is not open in x")

    def set_mask(self, solid: np.ndarray, q: np.ndarray | None = None) -> None:
        """Solid mask [ny][nx] (nonzero = solid) and optional link fractions
        q [9][ny][nx]; before the first step."""
        m = np.ascontiguousarray(solid, dtype=np.uint8).reshape(self.ny * self.nx)
        qq = None if q is None else np.ascontiguousarray(q, np.float64).reshape(9, -1)
        rc = lib().orc_set_mask(self._h, m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                _ptr(qq) if qq is not None else None)
        if rc != 0:
            raise ValueError(f"oracle rejected the mask ({rc})")

    def source(self) -> np.ndarray:
        out = np.empty((3, self.ny, self.nx))
        lib().orc_get_source(self._h, _ptr(out))
        return out

    def state(self):
        f = np.empty((9, self.ny, self.nx))
        g = np.empty((3, 9, self.ny, self.nx))
        lib().orc_get_state(self._h, _ptr(f), _ptr(g))
        return f, g

    def set_state(self, f, g) -> None:
        f = np.ascontiguousarray(f, np.float64)
        g = np.ascontiguousarray(g, np.float64)
        lib().orc_set_state(self._h, _ptr(f), _ptr(g))

    def coeffs(self) -> dict:
        c = Coeffs()
        lib().orc_get_coeffs(self._h, ctypes.byref(c))
        d = {k: getattr(c, k) for k, _ in Coeffs._fields_}
        d["lambda"] = d.pop("lambda_")
        return d


# ---- node-level entry points (for the moment-identity pins) ---------------

def feq(rho, ux, uy) -> np.ndarray:
    out = np.empty(9)
    lib().orc_feq(rho, ux, uy, _ptr(out))
    return out


def geq(phi, ux, uy) -> np.ndarray:
    out = np.empty(9)
    lib().orc_geq(phi, ux, uy, _ptr(out))
    return out


def hydro_moments(f, Fx, Fy):
    f = np.ascontiguousarray(f, np.float64)
    r, ux, uy = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lib().orc_hydro_moments(_ptr(f), Fx, Fy, ctypes.byref(r), ctypes.byref(ux), ctypes.byref(uy))
    return r.value, ux.value, uy.value


def hydro_collide(f, Fx, Fy, tau, dPhi, tau_s1, tau_s2) -> np.ndarray:
    f = np.ascontiguousarray(f, np.float64)
    tau = np.ascontiguousarray(tau, np.float64)
    dPhi = np.ascontiguousarray(dPhi, np.float64)
    out = np.empty(9)
    lib().orc_hydro_collide(_ptr(f), Fx, Fy, _ptr(tau), _ptr(dPhi), tau_s1, tau_s2, _ptr(out))
    return out


def cde_collide(g, rho, ux, uy, Fx, Fy, S, S_old, uxo, uyo, tau_p1, tau_p2) -> np.ndarray:
    g = np.ascontiguousarray(g, np.float64)
    out = np.empty(9)
    lib().orc_cde_collide(_ptr(g), rho, ux, uy, Fx, Fy, S, S_old, uxo, uyo, tau_p1, tau_p2,
                          _ptr(out))
    return out


def source(A, grad, lam, model=0, L2=0.0) -> np.ndarray:
    A = np.ascontiguousarray(A, np.float64)
    grad = np.ascontiguousarray(grad, np.float64)
    out = np.empty(3)
    if model == 0:
        lib().orc_source(_ptr(A), _ptr(grad), lam, _ptr(out))
    else:
        lib().orc_source_model(_ptr(A), _ptr(grad), lam, int(model), float(L2), _ptr(out))
    return out


def model_F(A, model, L2) -> np.ndarray:
    """Constitutive function F(A) of model 0 (Oldroyd-B), 1 (FENE-P), 2 (FENE-CR)."""
    A = np.ascontiguousarray(A, np.float64)
    out = np.empty(3)
    lib().orc_model_F(_ptr(A), int(model), float(L2), _ptr(out))
    return out


def zou_he(f, Fx, Fy, side) -> np.ndarray:
    f = np.array(f, np.float64)
    lib().orc_zou_he(_ptr(f), Fx, Fy, side)
    return f


def cnebb(g, gpost, known, ux, uy):
    g = np.array(g, np.float64)
    gpost = np.ascontiguousarray(gpost, np.float64)
    known = np.ascontiguousarray(known, np.int32)
    win, wout = ctypes.c_double(), ctypes.c_double()
    lib().orc_cnebb(_ptr(g), _ptr(gpost), known.ctypes.data_as(_ip), ux, uy,
                    ctypes.byref(win), ctypes.byref(wout))
    return g, win.value, wout.value
