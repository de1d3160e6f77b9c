"""Oracle of the adaptive-mesh plumbing between stages (test infrastructure).

Octree leaves (level l, i, j, k) on [-1, 1]^3, N^3 cells each (N = 8 by
default, 16 for the larger sub-grids of Sec. III-B); 2:1 balanced
across faces, edges and vertices (octree of Sec. III-B).  Readings (the paper
defers the mesh operations to the method paper):

ghost fill, in two passes.  A ghost cell of a leaf at level l sits at a
global cell index g (level-l cells); outside the domain g is clamped to the
nearest cell (outflow, zero gradient).  Pass 1: if a leaf of level l holds g,
copy that cell; if the position is refined, restrict: the mean of the 8
level-(l+1) cells 2g + d, taken in (dz, dy, dx) lexicographic order a0..a7
and summed pairwise, ((a0+a1)+(a2+a3)) + ((a4+a5)+(a6+a7)), times 1/8 (the
pairwise order keeps a uniform state exact).  Pass 2 (after pass 1 everywhere): if a coarser leaf holds g, prolong
from its cell G = floor(g / 2) with minmod-limited slopes
    s_a = minmod(U[G + e_a] - U[G], U[G] - U[G - e_a]),
    U(g) = U[G] + s_x o_x + s_y o_y + s_z o_z,  o_a = -1/4 or +1/4
(conservative: the mean over the 8 children is U[G]).

flux correction: where a leaf face borders finer leaves, the coarse cell's
flux through it is replaced by the mean of the 4 fine sub-face fluxes, and
its spin torque by the mean of the fine torques moved to the coarse cell
centre (T(x_C) = T(x_f) + (x_f - x_C) x F_s), in sub-face order c-major.

Written with plain loops and a dictionary of leaves, independently of the
CUDA tables.
"""
from __future__ import annotations

import numpy as np

from . import core

G = 3


class Octree:
    def __init__(self, level, ijk, N: int = 8):
        self.N = int(N)
        self.level = [int(v) for v in level]
        self.ijk = [tuple(int(v) for v in t) for t in np.asarray(ijk)]
        self.leaf = {(l,) + c: s for s, (l, c) in enumerate(zip(self.level, self.ijk))}

    def find(self, l, g):
        """Leaf of level l holding global cell g: ('leaf', s, local) or
        ('refined',) or ('coarse',)."""
        N = self.N
        key = (l, g[0] // N, g[1] // N, g[2] // N)
        if key in self.leaf:
            return ("leaf", self.leaf[key], (g[0] % N, g[1] % N, g[2] % N))
        # refined if any descendant leaf exists below this position
        for lc in range(l - 1, -1, -1):
            sh = l - lc
            if (lc, key[1] >> sh, key[2] >> sh, key[3] >> sh) in self.leaf:
                return ("coarse",)
        return ("refined",)


def _clamp(g, n):
    return tuple(min(max(v, 0), n - 1) for v in g)


def fill_ghosts(tree: Octree, U: np.ndarray) -> np.ndarray:
    """Both passes; U [n][F][S][S][S] (interiors valid) -> new array."""
    N = tree.N
    U = U.copy()
    n = U.shape[0]
    todo = []
    for s in range(n):
        l = tree.level[s]
        base = [c * N for c in tree.ijk[s]]
        ncell = N * 2 ** l
        for z in range(-G, N + G):
            for y in range(-G, N + G):
                for x in range(-G, N + G):
                    if 0 <= x < N and 0 <= y < N and 0 <= z < N:
                        continue
                    g = _clamp((base[0] + x, base[1] + y, base[2] + z), ncell)
                    r = tree.find(l, g)
                    dst = (s, slice(None), z + G, y + G, x + G)
                    if r[0] == "leaf":
                        o, (a, b, c) = r[1], r[2]
                        U[dst] = U[o, :, c + G, b + G, a + G]
                    elif r[0] == "refined":
                        kids = []
                        for dz in (0, 1):
                            for dy in (0, 1):
                                for dx in (0, 1):
                                    gf = (2 * g[0] + dx, 2 * g[1] + dy, 2 * g[2] + dz)
                                    rf = tree.find(l + 1, gf)
                                    assert rf[0] == "leaf", "mesh not 2:1 balanced"
                                    o, (a, b, c) = rf[1], rf[2]
                                    kids.append(U[o, :, c + G, b + G, a + G])
                        acc = ((kids[0] + kids[1]) + (kids[2] + kids[3])) + ((kids[4] + kids[5]) + (kids[6] + kids[7]))
                        U[dst] = acc * 0.125
                    else:
                        todo.append((s, l, g, dst))
    V = U.copy()  # pass 2 reads pass-1 values only
    for s, l, g, dst in todo:
        gc = (g[0] // 2, g[1] // 2, g[2] // 2)
        r = tree.find(l - 1, gc)
        assert r[0] == "leaf", "mesh not 2:1 balanced"
        o, (a, b, c) = r[1], r[2]
        C = (o, slice(None), c + G, b + G, a + G)
        val = V[C].copy()
        off = [0.25 if (g[d] % 2) else -0.25 for d in range(3)]
        for d in range(3):
            e = [0, 0, 0]
            e[d] = 1
            up = V[o, :, c + G + e[2], b + G + e[1], a + G + e[0]]
            dn = V[o, :, c + G - e[2], b + G - e[1], a + G - e[0]]
            dp = up - V[C]
            dm = V[C] - dn
            mm = np.where(dp * dm <= 0.0, 0.0, np.where(np.abs(dp) < np.abs(dm), dp, dm))
            val = val + mm * off[d]
        U[dst] = val
    return U


def flux_correct(tree: Octree, dU: np.ndarray, faces: np.ndarray, h) -> np.ndarray:
    """Coarse-fine correction of dU/dt [n][F][N][N][N] from the boundary-face
    sums [n][6][F+3][N][N] of every leaf."""
    N = tree.N
    dU = dU.copy()
    nf = dU.shape[1]
    for s in range(dU.shape[0]):
        l = tree.level[s]
        ijk = tree.ijk[s]
        for a in range(3):
            b = 1 if a == 0 else 0
            c = 1 if a == 2 else 2
            for side in (0, 1):
                nb = list(ijk)
                nb[a] += 1 if side else -1
                if not (0 <= nb[a] < 2 ** l):
                    continue
                if tree.find(l, tuple(v * N for v in nb))[0] != "refined":
                    continue
                sgn = 1.0 if side else -1.0
                hc = h[s]
                for pc in range(N):
                    for pb in range(N):
                        fsum = np.zeros(nf)
                        tsum = np.zeros(3)
                        for dc in (0, 1):
                            for db in (0, 1):
                                gf = [0, 0, 0]
                                gf[a] = (ijk[a] + 1) * 2 * N if side else ijk[a] * 2 * N - 1
                                gf[b] = 2 * (ijk[b] * N + pb) + db
                                gf[c] = 2 * (ijk[c] * N + pc) + dc
                                r = tree.find(l + 1, tuple(gf))
                                assert r[0] == "leaf"
                                o, loc = r[1], r[2]
                                ff = faces[o, 2 * a + (0 if side else 1), :, loc[c], loc[b]]
                                Fs = ff[1:4]
                                rvec = np.zeros(3)
                                rvec[a] = 0.75 * hc * sgn
                                rvec[b] = (0.25 if db else -0.25) * hc
                                rvec[c] = (0.25 if dc else -0.25) * hc
                                tor = np.array([rvec[1] * Fs[2] - rvec[2] * Fs[1], rvec[2] * Fs[0] - rvec[0] * Fs[2],
                                                rvec[0] * Fs[1] - rvec[1] * Fs[0]])
                                fsum = fsum + ff[:nf]
                                tsum = tsum + (ff[nf:] + tor)
                        own = faces[s, 2 * a + side, :, pc, pb]
                        cell = [0, 0, 0]
                        cell[a] = N - 1 if side else 0
                        cell[b] = pb
                        cell[c] = pc
                        idx = (s, slice(None), cell[2], cell[1], cell[0])
                        corr = np.zeros(nf)
                        corr[:] = -(sgn / hc) * (fsum * 0.25 - own[:nf])
                        corr[6:9] += -(sgn / hc) * (tsum * 0.25 - own[nf:])
                        dU[idx] = dU[idx] + corr
    return dU


def rk3_step(P: core.OracleParams, tree: Octree, U: np.ndarray, origin, h, cfl: float = 0.4):
    """One SSP-RK3 step of the whole mesh (ghost fill, step with face sums,
    correction, update, three times; dt from the first stage)."""
    assert P.N == tree.N
    U0 = U.copy()
    Us = U
    dt = None
    for k in range(3):
        Us = fill_ghosts(tree, Us)
        if k == 0:
            U0 = Us.copy()
        dU, am, _, faces = core.step(P, Us, origin, h, faces=True)
        dU = flux_correct(tree, dU, faces, h)
        if k == 0:
            dt = cfl * float(np.min(h / am))
        Us = core.update(P, Us, U0, dU, dt, k)
    return Us, dt
