"""Ghost fill and RK3 driver of the oracle on uniform boxes of sub-grids.

Test infrastructure only.  A box is ``nbx x nby x nbz`` sub-grids of N^3 cells
with cell width h; sub-grid s = (kz*nby + ky)*nbx + kx.  Ghost fill between
same-level neighbours is a copy of the neighbour's cells; the domain boundary
is periodic (ghosts wrap around) or outflow (zero-gradient: a ghost copies the
nearest interior cell).  This is the plain definition of the ghost exchange
between leaf sub-grids (octree of Sec. III-B; the exchange of Sec. IV-A.2).
"""
from __future__ import annotations

import numpy as np

from . import core


def pad_box(Ug: np.ndarray, G: int, bc: str) -> np.ndarray:
    """[nf][nz][ny][nx] -> [nf][nz+2G][ny+2G][nx+2G] with boundary ghosts."""
    mode = {"periodic": "wrap", "outflow": "edge"}[bc]
    return np.pad(Ug, ((0, 0), (G, G), (G, G), (G, G)), mode=mode)


def split(Up: np.ndarray, N: int, G: int) -> np.ndarray:
    """Padded box -> [n_sub][nf][S][S][S] ghost-filled sub-grids."""
    nf = Up.shape[0]
    nz, ny, nx = (n - 2 * G for n in Up.shape[1:])
    nbz, nby, nbx = nz // N, ny // N, nx // N
    S = N + 2 * G
    out = np.empty((nbz * nby * nbx, nf, S, S, S))
    s = 0
    for kz in range(nbz):
        for ky in range(nby):
            for kx in range(nbx):
                out[s] = Up[:, kz * N:kz * N + S, ky * N:ky * N + S, kx * N:kx * N + S]
                s += 1
    return out


def join(sub: np.ndarray, nbx: int, nby: int, nbz: int) -> np.ndarray:
    """[n_sub][nf][N][N][N] -> [nf][nz][ny][nx]."""
    n, nf, N = sub.shape[0], sub.shape[1], sub.shape[2]
    out = np.empty((nf, nbz * N, nby * N, nbx * N))
    s = 0
    for kz in range(nbz):
        for ky in range(nby):
            for kx in range(nbx):
                out[:, kz * N:(kz + 1) * N, ky * N:(ky + 1) * N, kx * N:(kx + 1) * N] = sub[s]
                s += 1
    return out


def unjoin(Ug: np.ndarray, N: int) -> np.ndarray:
    """[nf][nz][ny][nx] -> [n_sub][nf][N][N][N] (the inverse of join)."""
    nf, nz, ny, nx = Ug.shape
    nbz, nby, nbx = nz // N, ny // N, nx // N
    v = Ug.reshape(nf, nbz, N, nby, N, nbx, N).transpose(1, 3, 5, 0, 2, 4, 6)
    return np.ascontiguousarray(v.reshape(nbz * nby * nbx, nf, N, N, N))


def interior(sub_padded: np.ndarray, G: int) -> np.ndarray:
    return sub_padded[:, :, G:-G, G:-G, G:-G]


def origins(nbx: int, nby: int, nbz: int, N: int, h: float, lo) -> np.ndarray:
    o = np.empty((nbx * nby * nbz, 3))
    s = 0
    for kz in range(nbz):
        for ky in range(nby):
            for kx in range(nbx):
                o[s] = (lo[0] + kx * N * h, lo[1] + ky * N * h, lo[2] + kz * N * h)
                s += 1
    return o


class BoxRun:
    """RK3 time integration of a uniform box on the oracle.

    Ug: interior state [nf][nz][ny][nx]; lo: lower corner; h: cell width."""

    def __init__(self, P: core.OracleParams, Ug: np.ndarray, h: float, lo, bc: str, g: np.ndarray | None = None,
                 nthreads: int = 0):
        self.P, self.h, self.lo, self.bc, self.nthreads = P, float(h), tuple(lo), bc, nthreads
        self.U = np.array(Ug, dtype=np.float64)
        N = P.N
        self.nbz, self.nby, self.nbx = (n // N for n in Ug.shape[1:])
        self.orig = origins(self.nbx, self.nby, self.nbz, N, self.h, self.lo)
        self.g = g
        self.t = 0.0

    def _sub(self, Ug):
        return split(pad_box(Ug, self.P.G, self.bc), self.P.N, self.P.G)

    def rhs(self, Ug):
        dU, am, _ = core.step(self.P, self._sub(Ug), self.orig, self.h, self.g, nthreads=self.nthreads)
        return dU, am

    def step(self, cfl: float = 0.4, dt: float | None = None, t_end: float | None = None) -> float:
        """One RK3 step; dt = cfl * min(h / amax) from the first stage unless given."""
        P = self.P
        U0s = self._sub(self.U)
        Us = U0s
        for k in range(3):
            if k > 0:
                Us = self._sub(join(interior(Us, P.G), self.nbx, self.nby, self.nbz))
            dU, am = core.step(P, Us, self.orig, self.h, self.g, nthreads=self.nthreads)[:2]
            if k == 0 and dt is None:
                dt = cfl * float(np.min(self.h / am))
                if t_end is not None:
                    dt = min(dt, t_end - self.t)
            Us = core.update(P, Us, U0s, dU, dt, k)
        self.U = join(interior(Us, P.G), self.nbx, self.nby, self.nbz)
        self.t += dt
        return dt

    def run(self, t_end: float, cfl: float = 0.4, max_steps: int = 100000) -> int:
        n = 0
        while self.t < t_end * (1 - 1e-12) and n < max_steps:
            self.step(cfl, t_end=t_end)
            n += 1
        return n
