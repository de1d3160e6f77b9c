"""ctypes binding of ``hydro_oracle.cpp`` (test infrastructure only).

The shared object is built by :func:`build` with g++ (``-ffp-contract=off`` so
that every ``a*b + c`` in the oracle is two rounded operations, as written).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hydro_oracle.cpp")
_SO = os.path.join(_HERE, "_liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle shared object next to its source; returns its path."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
               "-o", _SO + ".tmp", _SRC]
        subprocess.run(cmd, check=True)
        os.replace(_SO + ".tmp", _SO)
    return _SO


class _P(C.Structure):
    _fields_ = [("gamma", C.c_double), ("omega", C.c_double), ("eta1", C.c_double), ("eta2", C.c_double),
                ("N", C.c_int), ("G", C.c_int), ("nf", C.c_int), ("face_points", C.c_int), ("contact", C.c_int),
                ("spin", C.c_int)]


@dataclass
class OracleParams:
    """Physical and layout parameters.  eta1/eta2 are the dual-energy
    thresholds of Bryan et al. (1995) (selection and tracer resync)."""
    gamma: float = 5.0 / 3.0
    omega: float = 0.0
    eta1: float = 1e-3
    eta2: float = 0.1
    N: int = 8
    G: int = 3
    nf: int = 10
    face_points: int = 9  # 1: flux at the face centres only (the old hydro module, Sec. III-B)
    contact: int = 0  # 1: PPM contact steepening of density and species (optional in Sec. III-B)
    spin: int = 0  # 1: a cell's spin feeds back into the velocity at its quadrature points (parity unpinned)

    def c(self) -> _P:
        return _P(self.gamma, self.omega, self.eta1, self.eta2, self.N, self.G, self.nf, self.face_points,
                  self.contact, self.spin)


_lib = None


def lib():
    global _lib
    if _lib is None:
        l = C.CDLL(build())
        dp = C.POINTER(C.c_double)
        l.orc_step.argtypes = [C.POINTER(_P), C.c_int, dp, dp, dp, dp, dp, dp, C.POINTER(C.c_uint8), dp, C.c_int]
        l.orc_step.restype = C.c_int
        l.orc_step_masked.argtypes = [C.POINTER(_P), C.c_int, dp, dp, dp, dp, dp, dp, C.POINTER(C.c_uint8), C.c_int]
        l.orc_step_masked.restype = C.c_int
        l.orc_update.argtypes = [C.POINTER(_P), C.c_int, dp, dp, dp, C.c_double, C.c_int]
        l.orc_update.restype = C.c_int
        l.orc_primitives.argtypes = [C.POINTER(_P), dp, dp]
        l.orc_ppm_line.argtypes = [dp, dp, dp]
        l.orc_ppm_line.restype = C.c_int
        l.orc_ppm_line_eta.argtypes = [dp, C.c_double, dp, dp]
        l.orc_ppm_line_eta.restype = None
        l.orc_contact_eta.argtypes = [C.POINTER(_P), dp, dp, dp]
        l.orc_contact_eta.restype = C.c_double
        l.orc_spin_velocity.argtypes = [C.POINTER(_P), C.c_double, C.c_double, dp, C.c_double, dp, dp]
        l.orc_spin_velocity.restype = None
        l.orc_point_flux.argtypes = [C.POINTER(_P), dp, dp, C.c_int, dp, dp, dp]
        l.orc_count_ops.argtypes = [C.POINTER(_P), dp, dp, C.c_double, C.POINTER(C.c_long)]
        ip = C.POINTER(C.c_int)
        l.orc_face_values.argtypes = [C.POINTER(_P), dp, C.c_int, ip, ip, dp, ip]
        _lib = l
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def step(P: OracleParams, U: np.ndarray, origin: np.ndarray, h: np.ndarray, g: np.ndarray | None = None,
         want_flags: bool = False, nthreads: int = 0, faces: bool = False):
    """One stage of the semi-discrete operator on a batch of sub-grids.

    U [n_sub][nf][S][S][S] (ghosts filled) -> (dUdt [n_sub][nf][N][N][N], amax [n_sub],
    limflag [n_sub][N][N][N] or None); with faces=True a fourth result, the
    boundary-face sums [n_sub][6][nf+3][N][N]."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    n = U.shape[0]
    N = P.N
    origin = np.ascontiguousarray(np.broadcast_to(origin, (n, 3)), dtype=np.float64)
    h = np.ascontiguousarray(np.broadcast_to(h, (n,)), dtype=np.float64)
    dU = np.zeros((n, P.nf, N, N, N))
    am = np.zeros(n)
    fl = np.zeros((n, N, N, N), dtype=np.uint8) if want_flags else None
    gp = _dp(np.ascontiguousarray(g, dtype=np.float64)) if g is not None else None
    if g is not None:
        g = np.ascontiguousarray(g, dtype=np.float64)
        gp = _dp(g)
    ff = np.zeros((n, 6, P.nf + 3, N, N)) if faces else None
    rc = lib().orc_step(C.byref(P.c()), n, _dp(U), _dp(origin), _dp(h), gp, _dp(dU), _dp(am),
                        fl.ctypes.data_as(C.POINTER(C.c_uint8)) if fl is not None else None,
                        _dp(ff) if ff is not None else None, nthreads)
    if rc != 0:
        raise ValueError("orc_step rejected its arguments")
    if faces:
        return dU, am, fl, ff
    return dU, am, fl


def step_masked(P: OracleParams, U: np.ndarray, origin, h, smooth: np.ndarray, g=None, nthreads: int = 0):
    """step() where cells with smooth[s][z][y][x] != 0 (padded S^3 layout) use the
    unlimited 4-point interface formula on their lines."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    n = U.shape[0]
    N = P.N
    origin = np.ascontiguousarray(np.broadcast_to(origin, (n, 3)), dtype=np.float64)
    h = np.ascontiguousarray(np.broadcast_to(h, (n,)), dtype=np.float64)
    sm = np.ascontiguousarray(smooth, dtype=np.uint8)
    assert sm.size == n * (N + 2 * P.G) ** 3
    dU = np.zeros((n, P.nf, N, N, N))
    am = np.zeros(n)
    gp = None
    if g is not None:
        g = np.ascontiguousarray(g, dtype=np.float64)
        gp = _dp(g)
    rc = lib().orc_step_masked(C.byref(P.c()), n, _dp(U), _dp(origin), _dp(h), gp, _dp(dU), _dp(am),
                               sm.ctypes.data_as(C.POINTER(C.c_uint8)), nthreads)
    if rc != 0:
        raise ValueError("orc_step_masked rejected its arguments")
    return dU, am


def update(P: OracleParams, U: np.ndarray, U0: np.ndarray, dUdt: np.ndarray, dt: float, stage: int) -> np.ndarray:
    """RK3 stage update of the interior (returns a new padded array)."""
    out = np.array(U, dtype=np.float64, order="C", copy=True)
    U0 = np.ascontiguousarray(U0, dtype=np.float64)
    dUdt = np.ascontiguousarray(dUdt, dtype=np.float64)
    rc = lib().orc_update(C.byref(P.c()), out.shape[0], _dp(out), _dp(U0), _dp(dUdt), float(dt), int(stage))
    if rc != 0:
        raise ValueError("orc_update rejected its arguments")
    return out


def primitives(P: OracleParams, u: np.ndarray) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.float64)
    q = np.zeros(P.nf)
    lib().orc_primitives(C.byref(P.c()), _dp(u), _dp(q))
    return q


def ppm_line(s5) -> tuple[float, float, int]:
    s = np.ascontiguousarray(s5, dtype=np.float64)
    qp = C.c_double()
    qm = C.c_double()
    f = lib().orc_ppm_line(_dp(s), C.byref(qp), C.byref(qm))
    return qp.value, qm.value, f


def ppm_line_eta(s5, eta: float) -> tuple[float, float]:
    """PPM on five samples with the steepening weight eta applied before the
    monotonicity fix-ups (eta = 0: plain PPM)."""
    s = np.ascontiguousarray(s5, dtype=np.float64)
    qp = C.c_double()
    qm = C.c_double()
    lib().orc_ppm_line_eta(_dp(s), float(eta), C.byref(qp), C.byref(qm))
    return qp.value, qm.value


def contact_eta(P: OracleParams, a5, rho2, p2) -> float:
    """Steepening weight of a line: a5 the steepened field's samples, rho2/p2
    density and pressure of the two neighbours (towards -d, towards +d)."""
    a = np.ascontiguousarray(a5, dtype=np.float64)
    r = np.ascontiguousarray(rho2, dtype=np.float64)
    p = np.ascontiguousarray(p2, dtype=np.float64)
    return lib().orc_contact_eta(C.byref(P.c()), _dp(a), _dp(r), _dp(p))


def spin_velocity(P: OracleParams, rho: float, eps: float, z, h: float, r) -> np.ndarray:
    """The spin feedback's velocity increment at offset r from the centre of a
    cell of density rho, internal energy density eps, spin density z and
    width h."""
    zz = np.ascontiguousarray(z, dtype=np.float64)
    rr = np.ascontiguousarray(r, dtype=np.float64)
    dv = np.zeros(3)
    lib().orc_spin_velocity(C.byref(P.c()), float(rho), float(eps), _dp(zz), float(h), _dp(rr), _dp(dv))
    return dv


def point_flux(P: OracleParams, qL, qR, axis: int, xq) -> tuple[np.ndarray, float]:
    qL = np.ascontiguousarray(qL, dtype=np.float64)
    qR = np.ascontiguousarray(qR, dtype=np.float64)
    xq = np.ascontiguousarray(xq, dtype=np.float64)
    F = np.zeros(P.nf)
    aq = C.c_double()
    lib().orc_point_flux(C.byref(P.c()), _dp(qL), _dp(qR), axis, _dp(xq), _dp(F), C.byref(aq))
    return F, aq.value


def face_values(P: OracleParams, U: np.ndarray, cells, dirs):
    """R_i[d] for requested (cell, direction) pairs of one padded sub-grid.
    Returns (values [n][nf], limiter-changed flags [n])."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    cells = np.ascontiguousarray(cells, dtype=np.int32).reshape(-1, 3)
    dirs = np.ascontiguousarray(dirs, dtype=np.int32).reshape(-1, 3)
    n = cells.shape[0]
    out = np.zeros((n, P.nf))
    fl = np.zeros(n, dtype=np.int32)
    ip = C.POINTER(C.c_int)
    lib().orc_face_values(C.byref(P.c()), _dp(U), n, cells.ctypes.data_as(ip), dirs.ctypes.data_as(ip), _dp(out),
                          fl.ctypes.data_as(ip))
    return out, fl


OP_NAMES = ("add", "mul", "div", "sqrt", "pow", "cmp", "minmax", "sgn")


def count_ops(P: OracleParams, U: np.ndarray, origin, h: float) -> dict:
    """Exact operation counts of one sub-grid stage and of one RK update."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    origin = np.ascontiguousarray(origin, dtype=np.float64)
    out = (C.c_long * 18)()
    lib().orc_count_ops(C.byref(P.c()), _dp(U), _dp(origin), float(h), out)
    return {"step": dict(zip(OP_NAMES, out[:8])), "update": dict(zip(OP_NAMES, out[8:16])),
            "ppm_ops": out[16], "ppm_calls": out[17]}
