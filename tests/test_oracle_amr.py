"""The adaptive-mesh oracle pinned on the CPU: the mesh generator's 2:1
balance and tiling, uniform states and linear fields across refinement
levels, and conservation of mass, momentum, energy and angular momentum,
which holds only with the coarse-fine flux correction."""
import itertools

import numpy as np
import pytest

from paper_2107_10987_gb300 import workloads as W

GAMMA = 5.0 / 3.0


def small_mesh():
    """Level 1 everywhere, one octant refined to 2, one of its children to 3,
    then 2:1 balanced; leaf order shuffled."""
    leaves = [(1, i, j, k) for i in (0, 1) for j in (0, 1) for k in (0, 1) if (i, j, k) != (1, 1, 1)]
    leaves += [(2, 2 + i, 2 + j, 2 + k) for i in (0, 1) for j in (0, 1) for k in (0, 1) if (i, j, k) != (0, 0, 0)]
    leaves += [(3, 4 + i, 4 + j, 4 + k) for i in (0, 1) for j in (0, 1) for k in (0, 1)]
    leaves = W._balance(leaves)
    arr = np.array(leaves)[np.random.default_rng(3).permutation(len(leaves))]
    return arr[:, 0], arr[:, 1:]


def touching(a, b):
    la, ia = a[0], np.array(a[1:])
    lb, ib = b[0], np.array(b[1:])
    L = max(la, lb)
    lo_a, hi_a = ia * 2 ** (L - la), (ia + 1) * 2 ** (L - la)
    lo_b, hi_b = ib * 2 ** (L - lb), (ib + 1) * 2 ** (L - lb)
    return np.all(lo_a <= hi_b) and np.all(lo_b <= hi_a)


def test_generated_meshes_are_balanced_and_tile_the_domain():
    for lev, ijk in (small_mesh(), W.amr_shell_mesh(600, 5, 2, 4, R=0.5)[:2]):
        leaves = [(int(l),) + tuple(int(v) for v in c) for l, c in zip(lev, ijk)]
        vol = sum((2.0 / 2 ** l) ** 3 for l, *_ in leaves)
        assert vol == pytest.approx(8.0)
        for a, b in itertools.combinations(leaves, 2):
            if abs(a[0] - b[0]) > 1:
                assert not touching(a, b), (a, b)


def test_target_mesh_size():
    lev, ijk, th = W.amr_shell_mesh()
    assert abs(len(lev) - 4096) <= 0.05 * 4096
    assert set(np.unique(lev)) == {3, 4, 5, 6}


def _interior_state(lev, ijk, f):
    """Padded sub-grids whose interior holds f(x, y, z) -> [F] at cell centres."""
    o, h = W.amr_geometry(lev, ijk)
    U = np.zeros((len(lev), 10, 14, 14, 14))
    idx = np.arange(8) + 0.5
    for s in range(len(lev)):
        Z, Y, X = np.meshgrid(o[s, 2] + idx * h[s], o[s, 1] + idx * h[s], o[s, 0] + idx * h[s], indexing="ij")
        U[s, :, 3:-3, 3:-3, 3:-3] = f(X, Y, Z)
    return U, o, h


def test_uniform_state_preserved_across_levels(oracle_mod):
    from oracle import amr, core
    lev, ijk = small_mesh()
    tree = amr.Octree(lev, ijk)
    u = W.conserved_from_primitive(np.array(1.2), np.array([0.3, -0.2, 0.1]), np.array(0.7), GAMMA)
    U, o, h = _interior_state(lev, ijk, lambda X, Y, Z: u[:, None, None, None] * np.ones_like(X))
    Uf = amr.fill_ghosts(tree, U)
    assert np.all(Uf == u[None, :, None, None, None])
    dU, am, _, faces = core.step(core.OracleParams(gamma=GAMMA), Uf, o, h, faces=True)
    dU = amr.flux_correct(tree, dU, faces, h)
    assert np.all(dU[:, [0, 1, 2, 3, 4, 5, 9]] == 0.0)


def test_linear_fields_exact_in_ghosts(oracle_mod):
    """Restriction and minmod prolongation reproduce a linear field exactly."""
    from oracle import amr
    lev, ijk = small_mesh()
    tree = amr.Octree(lev, ijk)
    g = np.array([0.3, -0.7, 1.1])

    def lin(X, Y, Z):
        v = 2.0 + g[0] * X + g[1] * Y + g[2] * Z
        return np.broadcast_to(v, (10,) + v.shape)

    U, o, h = _interior_state(lev, ijk, lin)
    Uf = amr.fill_ghosts(tree, U)
    idx = np.arange(14) - 3 + 0.5
    for s in range(len(lev)):
        Z, Y, X = np.meshgrid(o[s, 2] + idx * h[s], o[s, 1] + idx * h[s], o[s, 0] + idx * h[s], indexing="ij")
        want = 2.0 + g[0] * X + g[1] * Y + g[2] * Z
        inside = (np.abs(X) < 1) & (np.abs(Y) < 1) & (np.abs(Z) < 1)  # outflow ghosts are clamped copies
        assert np.allclose(Uf[s, 0][inside], want[inside], atol=1e-13)


def _blob_state(lev, ijk, seed=4):
    rng = np.random.default_rng(seed)
    A = rng.uniform(0.1, 0.3, 10)

    def f(X, Y, Z):
        r2 = X * X + Y * Y + Z * Z
        bump = np.maximum(1.0 - r2 / 0.3, 0.0) ** 2  # compact: the boundary is exactly at rest
        rho = 1.0 + 0.8 * bump * (1 + 0.3 * np.sin(7 * X))
        v = np.stack([A[0] * bump * np.cos(5 * Y), A[1] * bump * np.sin(4 * Z), A[2] * bump * np.cos(3 * X)])
        p = 0.5 + 0.6 * bump
        z = np.stack([A[3] * bump, -A[4] * bump, A[5] * bump * X])
        return W.conserved_from_primitive(rho, v, p, GAMMA, z=z, species=0.3 * rho)

    return _interior_state(lev, ijk, f)


def _totals(U, dU, o, h):
    vol = h ** 3
    tot = (dU * vol[:, None, None, None, None]).sum(axis=(0, 2, 3, 4))
    scale = (np.abs(dU) * vol[:, None, None, None, None]).sum(axis=(0, 2, 3, 4))
    idx = np.arange(8) + 0.5
    L = np.zeros(3)
    Ls = np.zeros(3)
    for s in range(len(h)):
        Z, Y, X = np.meshgrid(o[s, 2] + idx * h[s], o[s, 1] + idx * h[s], o[s, 0] + idx * h[s], indexing="ij")
        ds = dU[s, 1:4]
        tq = np.stack([Y * ds[2] - Z * ds[1], Z * ds[0] - X * ds[2], X * ds[1] - Y * ds[0]])
        L += ((tq + dU[s, 6:9]) * vol[s]).sum(axis=(1, 2, 3))
        Ls += (np.abs(tq) * vol[s]).sum(axis=(1, 2, 3))
    return tot, scale, L, Ls


def test_conservation_needs_and_gets_flux_correction(oracle_mod):
    from oracle import amr, core
    lev, ijk = small_mesh()
    tree = amr.Octree(lev, ijk)
    U, o, h = _blob_state(lev, ijk)
    Uf = amr.fill_ghosts(tree, U)
    dU, am, _, faces = core.step(core.OracleParams(gamma=GAMMA), Uf, o, h, faces=True)
    tot0, scale, L0, Ls = _totals(Uf, dU, o, h)
    dUc = amr.flux_correct(tree, dU, faces, h)
    tot, scale, L, Ls = _totals(Uf, dUc, o, h)
    for k in (0, 1, 2, 3, 4, 5, 9):
        assert abs(tot[k]) <= 1e-13 * scale[k], (k, tot[k], scale[k])
        assert abs(tot0[k]) > 1e3 * abs(tot[k])  # the uncorrected sums are visibly off
    assert np.all(np.abs(L) <= 1e-12 * Ls.max()), (L, Ls)
