"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

Nothing here performs a step of the hydro method: these functions only lay
out initial states (ideal-gas cell averages) and mesh geometry.  Field order:
rho, s_x, s_y, s_z, E (gas energy), tau (entropy tracer), z_x, z_y, z_z,
species densities.  tau is set consistent with the internal energy,
tau = eps^(1/gamma), as the dual-energy formalism (Bryan et al. 1995) defines
it.  Arrays are float64, C-ordered, x fastest.
"""
from __future__ import annotations

import math

import numpy as np

NF = 10


def conserved_from_primitive(rho, v, p, gamma, z=None, species=None):
    """Cell averages from density, velocity [3,...], pressure.  Returns [NF,...]."""
    rho = np.asarray(rho, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    eps = np.asarray(p, dtype=np.float64) / (gamma - 1.0)
    U = np.zeros((NF,) + rho.shape)
    U[0] = rho
    U[1:4] = rho * v
    U[4] = eps + 0.5 * rho * (v[0] ** 2 + v[1] ** 2 + v[2] ** 2)
    U[5] = eps ** (1.0 / gamma)
    if z is not None:
        U[6:9] = z
    U[9] = rho if species is None else species
    return U


def cell_centres(shape, lo, h):
    """Centres (x, y, z) of a [nz][ny][nx] box with lower corner lo."""
    nz, ny, nx = shape
    x = lo[0] + (np.arange(nx) + 0.5) * h
    y = lo[1] + (np.arange(ny) + 0.5) * h
    z = lo[2] + (np.arange(nz) + 0.5) * h
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def sedov_box(n: int, gamma: float = 5.0 / 3.0, E_blast: float = 1.0, rho0: float = 1.0, p0: float = 1e-5,
              L: float = 2.0):
    """Sedov-Taylor point blast on [-L/2, L/2]^3 with n^3 cells (n even):
    rho = rho0, p = p0, v = 0, and the blast energy E_blast added uniformly as
    internal energy to the central 2^3 cells.  Returns (U [NF][n][n][n], h, lo)."""
    assert n % 2 == 0
    h = L / n
    lo = (-L / 2, -L / 2, -L / 2)
    rho = np.full((n, n, n), rho0)
    p = np.full((n, n, n), p0)
    c = slice(n // 2 - 1, n // 2 + 1)
    p[c, c, c] += (gamma - 1.0) * E_blast / (8.0 * h ** 3)
    U = conserved_from_primitive(rho, np.zeros((3, n, n, n)), p, gamma)
    return U, h, lo


def sedov_subgrid(gamma: float = 5.0 / 3.0, N: int = 8, G: int = 3):
    """Single 8^3 sub-grid Sedov blast on [-1,1]^3 (h = 2/N) with periodic
    ghosts: returns (U [NF][S][S][S], h, origin)."""
    U, h, lo = sedov_box(N, gamma)
    Up = np.pad(U, ((0, 0), (G, G), (G, G), (G, G)), mode="wrap")
    return Up, h, lo


def sod_box(n_normal: int, normal: str, gamma: float = 1.4, states=((1.0, 0.0, 1.0), (0.125, 0.0, 0.1)),
            n_trans: int = 8):
    """Periodic planar Sod tube on [0,1) along the unit normal 'x', 'xy' or 'xyz'.

    The normal coordinate xi = (n . x) folded onto [0,1); the left state fills
    xi in [0.25, 0.75) and the right state the rest, so the box holds two
    Riemann problems (at xi = 0.75 and, mirrored, at 0.25).  Box shapes:
    'x' -> n x n_trans x n_trans cells of width 1/n; 'xy' -> n x n x n_trans
    on [0,1)^2 with xi = (x + y) mod 1; 'xyz' -> n^3 with xi = (x+y+z) mod 1.
    Returns (U [NF][nz][ny][nx], h, lo, xi_of_cell, nvec)."""
    h = 1.0 / n_normal
    if normal == "x":
        shape = (n_trans, n_trans, n_normal)
        nvec = np.array([1.0, 0.0, 0.0])
    elif normal == "xy":
        shape = (n_trans, n_normal, n_normal)
        nvec = np.array([1.0, 1.0, 0.0]) / math.sqrt(2.0)
    elif normal == "xyz":
        shape = (n_normal, n_normal, n_normal)
        nvec = np.ones(3) / math.sqrt(3.0)
    else:
        raise ValueError(normal)
    X, Y, Z = cell_centres(shape, (0.0, 0.0, 0.0), h)
    k = {"x": X, "xy": X + Y, "xyz": X + Y + Z}[normal]
    xi = np.mod(k, 1.0)  # coordinate along the (unnormalised) normal, period 1
    left = (xi >= 0.25) & (xi < 0.75)
    (rl, ul, pl), (rr, ur, pr) = states
    rho = np.where(left, rl, rr)
    un = np.where(left, ul, ur)
    p = np.where(left, pl, pr)
    v = np.stack([un * nvec[0], un * nvec[1], un * nvec[2]])
    U = conserved_from_primitive(rho, v, p, gamma)
    return U, h, (0.0, 0.0, 0.0), xi, nvec


def random_subgrids(n_sub: int, seed: int, gamma: float = 5.0 / 3.0, N: int = 8, G: int = 3, smooth: bool = False,
                    spin: bool = True):
    """Random ghost-padded sub-grids [n_sub][NF][S][S][S] with positive density
    and pressure: rho in [0.5, 2], |v| <= 1, p in [0.1, 1] (or smooth sinusoidal
    fields when smooth=True), random spin z and species fraction."""
    rng = np.random.default_rng(seed)
    S = N + 2 * G
    shp = (n_sub, S, S, S)
    if smooth:
        ax = np.arange(S)
        Z, Y, X = np.meshgrid(ax, ax, ax, indexing="ij")
        ph = rng.uniform(0, 2 * np.pi, (n_sub, 6, 1, 1, 1))
        k = 2 * np.pi / 23.0
        rho = 1.0 + 0.3 * np.sin(k * X + ph[:, 0]) * np.cos(k * Y + ph[:, 1])
        p = 0.6 + 0.2 * np.sin(k * Z + ph[:, 2])
        v = np.stack([0.3 * np.sin(k * Y + ph[:, 3]), 0.2 * np.cos(k * Z + ph[:, 4]), 0.25 * np.sin(k * X + ph[:, 5])],
                     axis=1)
    else:
        rho = rng.uniform(0.5, 2.0, shp)
        p = rng.uniform(0.1, 1.0, shp)
        v = rng.uniform(-1.0, 1.0, (n_sub, 3, S, S, S)) / math.sqrt(3.0)
    z = rng.uniform(-0.05, 0.05, (n_sub, 3, S, S, S)) if spin else None
    frac = rng.uniform(0.0, 1.0, shp)
    out = np.empty((n_sub, NF, S, S, S))
    for s in range(n_sub):
        out[s] = conserved_from_primitive(rho[s], v[s], p[s], gamma,
                                          z=None if z is None else z[s], species=rho[s] * frac[s])
    return out


def contact_subgrids(n_sub: int, seed: int, gamma: float = 5.0 / 3.0, exact: bool = False, N: int = 8, G: int = 3):
    """Ghost-padded sub-grids [n_sub][NF][S][S][S] full of density contacts
    (the data PPM contact steepening acts on).  exact=False: two density
    levels (1 and 0.3) with 5 % noise, pressure 1 +- 2 %, species fraction
    0.4-0.6, and every fourth sub-grid with a pressure jump (1 to 10) across
    a plane, so that the contact test also meets shocks.  exact=True: density
    levels 1, 1/2 and 1/4, pressure exactly 1, species exactly half the
    density (values exact in FP32).  Velocities |v_i| <= 0.3, small spin."""
    rng = np.random.default_rng(seed)
    S = N + 2 * G
    sh = (S, S, S)
    out = np.empty((n_sub, NF) + sh)
    for i in range(n_sub):
        if exact:
            rho = rng.choice([1.0, 0.5, 0.25], size=sh)
            p = np.ones(sh)
            frac = np.full(sh, 0.5)
        else:
            rho = np.where(rng.random(sh) < 0.5, 1.0, 0.3) * rng.uniform(0.95, 1.05, sh)
            p = rng.uniform(0.98, 1.02, sh)
            if i % 4 == 3:
                p = np.where(np.arange(S)[None, None, :] < S // 2, 10.0, 1.0) * p
            frac = rng.uniform(0.4, 0.6, sh)
        v = rng.uniform(-0.3, 0.3, (3,) + sh)
        z = rng.uniform(-0.01, 0.01, (3,) + sh)
        out[i] = conserved_from_primitive(rho, v, p, gamma, z=z, species=frac * rho)
    return out


def uniform_mesh(nb: int, N: int = 8, L: float = 2.0):
    """Uniform octree level: nb^3 sub-grids of N^3 on [-L/2, L/2]^3.
    Returns (origins [n_sub][3], h); sub-grid s = (kz*nb + ky)*nb + kx."""
    h = L / (nb * N)
    o = np.empty((nb ** 3, 3))
    s = 0
    for kz in range(nb):
        for ky in range(nb):
            for kx in range(nb):
                o[s] = (-L / 2 + kx * N * h, -L / 2 + ky * N * h, -L / 2 + kz * N * h)
                s += 1
    return o, h


def box_to_subgrids(Ug: np.ndarray, N: int = 8):
    """Interior box [NF][nz][ny][nx] -> [n_sub][NF][N][N][N] (x-fastest sub-grid order)."""
    nf, nz, ny, nx = Ug.shape
    nbz, nby, nbx = nz // N, ny // N, nx // N
    out = np.empty((nbz * nby * nbx, nf, N, N, N))
    s = 0
    for kz in range(nbz):
        for ky in range(nby):
            for kx in range(nbx):
                out[s] = Ug[:, kz * N:(kz + 1) * N, ky * N:(ky + 1) * N, kx * N:(kx + 1) * N]
                s += 1
    return out


def lane_emden_table(n: float, dxi: float = 1e-4):
    """Lane-Emden solution of index n (theta'' + 2 theta'/xi + theta^n = 0,
    theta(0) = 1, theta'(0) = 0), integrated with classical RK4 from a series
    start until theta = 0.  Returns (xi, theta, m) on the grid up to the first
    zero xi1, with the mass function m(xi) = -xi^2 theta'(xi) (the integral of
    x^2 theta^n from 0 to xi)."""
    def rhs(x, y):
        th, dth = y
        return np.array([dth, -max(th, 0.0) ** n - 2.0 * dth / x])

    x = dxi
    y = np.array([1.0 - x * x / 6.0 + n * x ** 4 / 120.0, -x / 3.0 + n * x ** 3 / 30.0])
    xs, ths, ms = [0.0, x], [1.0, y[0]], [0.0, -x * x * y[1]]
    while y[0] > 0.0:
        k1 = rhs(x, y)
        k2 = rhs(x + dxi / 2, y + dxi / 2 * k1)
        k3 = rhs(x + dxi / 2, y + dxi / 2 * k2)
        k4 = rhs(x + dxi, y + dxi * k3)
        yn = y + dxi / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        if yn[0] <= 0.0:  # linear interpolation of the zero inside the last step
            f = y[0] / (y[0] - yn[0])
            x1 = x + f * dxi
            dth1 = y[1] + f * (yn[1] - y[1])
            xs.append(x1)
            ths.append(0.0)
            ms.append(-x1 * x1 * dth1)
            return np.array(xs), np.array(ths), np.array(ms)
        x, y = x + dxi, yn
        xs.append(x)
        ths.append(y[0])
        ms.append(-x * x * y[1])
    raise RuntimeError("unreachable")


def lane_emden(n: float, dxi: float = 1e-4):
    """Returns (xi1, -xi1^2 theta'(xi1), xi grid, theta) of lane_emden_table."""
    xs, ths, ms = lane_emden_table(n, dxi)
    return xs[-1], ms[-1], xs, ths


def polytrope_model(n: float = 1.5, R: float = 0.5, rho_c: float = 1.0, G: float = 1.0, dxi: float = 1e-4):
    """A polytrope p = K rho^(1+1/n) of radius R and central density rho_c in
    hydrostatic equilibrium: rho = rho_c theta(r/alpha)^n with alpha = R/xi1,
    K from alpha^2 = (n+1) K rho_c^(1/n-1) / (4 pi G), enclosed mass
    M(r) = 4 pi alpha^3 rho_c m(r/alpha), total M, and the Keplerian rate at
    the surface Omega_K = sqrt(G M / R^3)."""
    xs, ths, ms = lane_emden_table(n, dxi)
    alpha = R / xs[-1]
    K = 4.0 * math.pi * G * alpha * alpha * rho_c ** (1.0 - 1.0 / n) / (n + 1.0)
    M = 4.0 * math.pi * alpha ** 3 * rho_c * ms[-1]
    return {"n": n, "R": R, "rho_c": rho_c, "G": G, "alpha": alpha, "K": K, "M": M,
            "omega_K": math.sqrt(G * M / R ** 3), "xi": xs, "theta": ths, "m": ms}


def polytrope_point(model, X, Y, Z, spin: float = 0.2, rho_amb: float = 1e-10):
    """Density, inertial velocity [3,...], pressure and the static gravitational
    acceleration [3,...] of the model at points (X, Y, Z).  Inside r < R the
    star rotates rigidly about +z at spin * Omega_K; the ambient medium is at
    rest with density rho_amb on the same polytropic K.  g = -G M(r) x / r^3
    (zero at the centre)."""
    mo = model
    r = np.sqrt(X * X + Y * Y + Z * Z)
    xi = r / mo["alpha"]
    th = np.interp(xi, mo["xi"], mo["theta"], right=0.0)
    rho = np.maximum(mo["rho_c"] * th ** mo["n"], rho_amb)
    p = mo["K"] * rho ** (1.0 + 1.0 / mo["n"])
    w = spin * mo["omega_K"]
    inside = r < mo["R"]
    v = np.stack([np.where(inside, -w * Y, 0.0), np.where(inside, w * X, 0.0), np.zeros_like(X)])
    Mr = 4.0 * math.pi * mo["alpha"] ** 3 * mo["rho_c"] * np.interp(xi, mo["xi"], mo["m"], right=mo["m"][-1])
    with np.errstate(divide="ignore", invalid="ignore"):
        f = np.where(r > 0.0, -mo["G"] * Mr / (r * r * r), 0.0)
    g = np.stack([f * X, f * Y, f * Z])
    return rho, v, p, g


def rotating_polytrope(nb: int, gamma: float = 5.0 / 3.0, spin: float = 0.2, rho_amb: float = 1e-10,
                       n: float = 1.5, R: float = 0.5, N: int = 8, L: float = 2.0):
    """Rotating n = 1.5 polytrope on a uniform octree level of nb^3 sub-grids
    of N^3 cells covering [-L/2, L/2]^3 (nb = 32: 32,768 sub-grids, 256^3
    cells).  Cell averages are the point values at cell centres.  Returns
    (U [n_sub][NF][N][N][N] interiors, g [n_sub][3][N][N][N], origins
    [n_sub][3], h, model); sub-grid order as uniform_mesh."""
    model = polytrope_model(n, R)
    o, h = uniform_mesh(nb, N, L)
    c = (np.arange(N) + 0.5) * h
    ns = o.shape[0]
    X = np.broadcast_to(o[:, 0, None, None, None] + c[None, None, None, :], (ns, N, N, N))
    Y = np.broadcast_to(o[:, 1, None, None, None] + c[None, None, :, None], (ns, N, N, N))
    Z = np.broadcast_to(o[:, 2, None, None, None] + c[None, :, None, None], (ns, N, N, N))
    rho, v, p, g = polytrope_point(model, X, Y, Z, spin, rho_amb)
    U = np.ascontiguousarray(np.moveaxis(conserved_from_primitive(rho, v, p, gamma), 0, 1))
    g = np.ascontiguousarray(np.moveaxis(g, 0, 1))
    return U, g, o, h, model


def density_l1(rho, rho_ic, h, R: float = 0.5) -> float:
    """Density error sum |rho_IC - rho| h^3 / V over the whole domain, with V the
    initial volume 4 pi R^3 / 3 of the star (the rotating-star error measure
    of Sec. VI, read with an absolute value)."""
    return float(np.sum(np.abs(np.asarray(rho_ic) - np.asarray(rho))) * h ** 3 / (4.0 * math.pi * R ** 3 / 3.0))


def sedov_box_at(n: int, E_blast: float, center, gamma: float = 5.0 / 3.0, rho0: float = 1.0, p0: float = 1e-5,
                 L: float = 2.0):
    """Sedov blast of energy E_blast deposited as internal energy in the 2^3
    cells nearest to the point `center` of [-L/2, L/2]^3 (n^3 cells).
    Returns (U [NF][n][n][n], h, lo)."""
    h = L / n
    lo = (-L / 2, -L / 2, -L / 2)
    idx = [int(np.clip(np.floor((center[a] - lo[a]) / h - 0.5), 0, n - 2)) for a in range(3)]
    rho = np.full((n, n, n), rho0)
    p = np.full((n, n, n), p0)
    sl = tuple(slice(idx[a], idx[a] + 2) for a in (2, 1, 0))
    p[sl] += (gamma - 1.0) * E_blast / (8.0 * h ** 3)
    return conserved_from_primitive(rho, np.zeros((3, n, n, n)), p, gamma), h, lo


def sod_box_oriented(n: int, normal, offset: float, gamma: float = 1.4,
                     states=((1.0, 0.0, 1.0), (0.125, 0.0, 0.1)), L: float = 2.0):
    """Planar Sod interface with unit normal `normal` through the point
    offset * normal of [-L/2, L/2]^3: left state where (x . n) < offset.
    Returns (U [NF][n][n][n], h, lo)."""
    h = L / n
    lo = (-L / 2, -L / 2, -L / 2)
    nv = np.asarray(normal, dtype=np.float64)
    nv = nv / np.linalg.norm(nv)
    X, Y, Z = cell_centres((n, n, n), lo, h)
    left = (X * nv[0] + Y * nv[1] + Z * nv[2]) < offset
    (rl, ul, pl), (rr, ur, pr) = states
    rho = np.where(left, rl, rr)
    un = np.where(left, ul, ur)
    p = np.where(left, pl, pr)
    v = np.stack([un * nv[0], un * nv[1], un * nv[2]])
    return conserved_from_primitive(rho, v, p, gamma), h, lo


def indicator_runs(seeds, n: int = 64):
    """Seeded initial states of the indicator's training/evaluation runs: for
    each seed, a Sedov blast with energy ~ U(0.1, 10) at a random centre in
    [-0.5, 0.5]^3 (gamma 5/3) for even seeds, a Sod plane at a random
    orientation and offset in [-0.3, 0.3] (gamma 1.4) for odd seeds.
    Yields (seed, kind, gamma, U, h, lo)."""
    for sd in seeds:
        rng = np.random.default_rng(10_000 + sd)
        if sd % 2 == 0:
            E = rng.uniform(0.1, 10.0)
            c = rng.uniform(-0.5, 0.5, 3)
            U, h, lo = sedov_box_at(n, E, c)
            yield sd, "sedov", 5.0 / 3.0, U, h, lo
        else:
            nv = rng.normal(size=3)
            U, h, lo = sod_box_oriented(n, nv, rng.uniform(-0.3, 0.3))
            yield sd, "sod", 1.4, U, h, lo


# ---------------------------------------------------------------------------
# Adaptive octree meshes on [-1, 1]^3.  A leaf at level l has integer
# coordinates (i, j, k) in [0, 2^l)^3, width 2 / 2^l and cell width
# h = 2 / (N 2^l); its origin is -1 + (i, j, k) * width.

def _shell_density(r, R=0.3, gamma=5.0 / 3.0):
    """Stand-in density of a blast shell of radius R used only to decide
    refinement: 1 outside, (g+1)/(g-1) (r/R)^(3/(g-1)) inside (the power-law
    behaviour of the self-similar profile behind a strong shock)."""
    jump = (gamma + 1.0) / (gamma - 1.0)
    return np.where(r < R, jump * np.maximum(r / R, 1e-12) ** (3.0 / (gamma - 1.0)) + 1e-12, 1.0)


def _needs_refinement(level, ijk, theta, R):
    """Refine where the stand-in shell density varies across the node by more
    than theta: (max - min) / (max + min) over the node's 5^3 sample points
    (corners included), a bounded measure of |grad rho| / rho times the width."""
    w = 2.0 / 2 ** level
    lo = -1.0 + np.asarray(ijk, dtype=np.float64) * w
    t = np.linspace(0.0, 1.0, 5)
    P = lo + w * np.stack(np.meshgrid(t, t, t, indexing="ij"), -1).reshape(-1, 3)
    rho = _shell_density(np.linalg.norm(P, axis=1), R)
    return bool((rho.max() - rho.min()) / (rho.max() + rho.min()) > theta)


def _balance(leaves):
    """Refine until every pair of leaves sharing a face, edge or vertex
    differs by at most one level (2:1 balance)."""
    leaves = set(leaves)

    def covering(l, i, j, k):
        # the leaf containing the level-l node (l, i, j, k), or None if that
        # node is refined further
        for lv in range(l, -1, -1):
            sh = l - lv
            key = (lv, i >> sh, j >> sh, k >> sh)
            if key in leaves:
                return key
        return None

    queue = sorted(leaves, key=lambda t: t[0])
    while queue:
        leaf = queue.pop()
        if leaf not in leaves:
            continue
        l, i, j, k = leaf
        n = 2 ** l
        for di in (-1, 0, 1):
            for dj in (-1, 0, 1):
                for dk in (-1, 0, 1):
                    a, b, c = i + di, j + dj, k + dk
                    if not (0 <= a < n and 0 <= b < n and 0 <= c < n) or (di, dj, dk) == (0, 0, 0):
                        continue
                    cov = covering(l, a, b, c)
                    if cov is not None and cov[0] < l - 1:
                        leaves.remove(cov)
                        lc, ic, jc, kc = cov
                        for d in range(8):
                            child = (lc + 1, 2 * ic + (d & 1), 2 * jc + ((d >> 1) & 1), 2 * kc + (d >> 2))
                            leaves.add(child)
                            queue.append(child)
                        queue.append(leaf)
    return sorted(leaves)


def octree_shell_mesh(theta: float, lmin: int = 3, lmax: int = 6, R: float = 0.3):
    """Leaves (level, i, j, k) of the octree refined around a blast shell of
    radius R, 2:1 balanced."""
    leaves = []
    stack = [(lmin, i, j, k) for i in range(2 ** lmin) for j in range(2 ** lmin) for k in range(2 ** lmin)]
    while stack:
        l, i, j, k = stack.pop()
        if l < lmax and _needs_refinement(l, (i, j, k), theta, R):
            for d in range(8):
                stack.append((l + 1, 2 * i + (d & 1), 2 * j + ((d >> 1) & 1), 2 * k + (d >> 2)))
        else:
            leaves.append((l, i, j, k))
    return _balance(leaves)


def amr_shell_mesh(n_target: int = 4096, seed: int = 1234, lmin: int = 3, lmax: int = 6, R: float = 0.3):
    """The batched-AMR configuration: an octree of about n_target leaves at
    levels lmin..lmax, refined around a blast shell of radius R (threshold
    bisected to hit the target), 2:1 balanced, leaf order shuffled by seed.
    Returns (level [n] int32, ijk [n][3] int32, theta)."""
    lo_t, hi_t = 1e-3, 0.999
    best = None
    for _ in range(30):
        th = 0.5 * (lo_t + hi_t)
        leaves = octree_shell_mesh(th, lmin, lmax, R)
        if best is None or abs(len(leaves) - n_target) < abs(len(best[0]) - n_target):
            best = (leaves, th)
        if abs(len(leaves) - n_target) <= 0.02 * n_target:
            break
        if len(leaves) > n_target:
            lo_t = th
        else:
            hi_t = th
    leaves, th = best
    order = np.random.default_rng(seed).permutation(len(leaves))
    arr = np.array(leaves, dtype=np.int32)[order]
    return arr[:, 0].copy(), arr[:, 1:].copy(), th


def amr_geometry(level, ijk, N: int = 8):
    """Origins [n][3] and cell widths [n] of the leaves."""
    w = 2.0 / (2.0 ** np.asarray(level, dtype=np.float64))
    return -1.0 + np.asarray(ijk, dtype=np.float64) * w[:, None], w / N


def amr_shell_state(level, ijk, gamma: float = 5.0 / 3.0, R: float = 0.3, N: int = 8, G: int = 3):
    """A blast-shell state on AMR leaves (cell-centre values, ghosts zero):
    outside r = R gas at rest (rho 1, p 1e-5); inside the shell the stand-in
    density profile, radial velocity 0.75 r/R and pressure 0.3 + 0.45 (r/R)^2.
    Returns [n][NF][S][S][S]."""
    o, h = amr_geometry(level, ijk, N)
    n = len(level)
    S = N + 2 * G
    out = np.zeros((n, NF, S, S, S))
    idx = np.arange(N) + 0.5
    for s in range(n):
        X = o[s, 0] + idx[None, None, :] * h[s]
        Y = o[s, 1] + idx[None, :, None] * h[s]
        Z = o[s, 2] + idx[:, None, None] * h[s]
        X, Y, Z = np.broadcast_arrays(X, Y, Z)
        r = np.sqrt(X * X + Y * Y + Z * Z)
        inside = r < R
        rho = np.where(inside, np.maximum(_shell_density(r, R, gamma), 1e-3), 1.0)
        vr = np.where(inside, 0.75 * r / R, 0.0)
        rr = np.maximum(r, 1e-12)
        v = np.stack([vr * X / rr, vr * Y / rr, vr * Z / rr])
        p = np.where(inside, 0.3 + 0.45 * (r / R) ** 2, 1e-5)
        out[s, :, G:G + N, G:G + N, G:G + N] = conserved_from_primitive(rho, v, p, gamma)
    return out
