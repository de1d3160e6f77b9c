"""The oracle pinned to what the method and the mathematics fix (CPU only).

Each test is chosen so that a plausible mistake in the oracle (a dropped term,
a wrong sign, a transposed index or direction) fails at least one of them:
  * uniform state                 -> any asymmetric face handling, stray source
  * linear / quadratic fields     -> PPM coefficients, line sample indexing on
                                     all 26 directions, the point each value is for
  * conservation (linear, angular) -> flux sharing, face signs, the spin torque
  * permutation symmetry          -> axis-specific slips (p e_a, transverse order)
  * flux sign / consistency       -> the dissipation sign, the pressure terms
  * 1-D reduction                 -> the face sum of a 1-D flow (weights summing to 1)
  * transverse quadratic          -> the distribution of the face weights (Simpson,
                                     exact to cubic order) on both transverse axes
  * RK3 polynomial                -> the stage coefficients
  * dual energy                   -> selection and resync thresholds
The analytic solutions (Sod, Sedov) are in test_oracle_analytic.py.
"""
import itertools
import math

import numpy as np
import pytest

from paper_2107_10987_gb300 import workloads as W

GAMMA = 5.0 / 3.0
N, G = 8, 3
S = N + 2 * G
DIRS = [d for d in itertools.product((-1, 0, 1), repeat=3) if d != (0, 0, 0)]


@pytest.fixture(scope="module")
def orc(oracle_mod):
    return oracle_mod.core


def P(orc, **kw):
    return orc.OracleParams(**kw)


def uniform_subgrid(rho, v, p, z=(0.0, 0.0, 0.0), frac=0.3):
    shp = (S, S, S)
    U = W.conserved_from_primitive(np.full(shp, rho), np.stack([np.full(shp, c) for c in v]), np.full(shp, p), GAMMA,
                                   z=np.stack([np.full(shp, c) for c in z]), species=np.full(shp, rho * frac))
    return U


def test_uniform_state_is_preserved_bitwise(orc):
    rho, v, p = 1.3, (0.4, -0.7, 0.2), 0.8
    U = uniform_subgrid(rho, v, p, z=(0.01, -0.02, 0.03))
    dU, am, _ = orc.step(P(orc), U[None], np.array([-0.3, 0.1, 0.7]), 0.05)
    lin = [0, 1, 2, 3, 4, 5, 9]
    assert np.all(dU[:, lin] == 0.0), "a uniform state must have dU/dt == 0 exactly"
    # spin: the torque of a uniform momentum flux is sum_a e_a x F_a = u x s = 0,
    # reached only to round-off (terms of size |s||u|/h cancel)
    assert np.max(np.abs(dU[:, 6:9])) <= 1e-14 * (rho * 1.0 + p) / 0.05
    # amax = max_a |v_a| + c with c from the recovered primitives
    q = orc.primitives(P(orc), U[:, 0, 0, 0].copy())
    c = math.sqrt(GAMMA * (GAMMA - 1.0) * q[4] / q[0])
    assert am[0] == pytest.approx(max(abs(x) for x in q[1:4]) + c, rel=1e-15)


def test_uniform_state_rotating_frame_source_only(orc):
    # with omega != 0 a uniform state at rest feels no flux divergence (the
    # frame velocity is linear in x, so fluxes differ); but a state at rest
    # with uniform pressure: mass flux = rho u_n is linear in x_q and its
    # divergence vanishes (div of omega z x x is 0).  Check the mass equation.
    U = uniform_subgrid(1.0, (0.0, 0.0, 0.0), 1.0)
    dU, am, _ = orc.step(P(orc, omega=0.3), U[None], np.array([-0.2, -0.2, -0.2]), 0.05)
    assert np.max(np.abs(dU[0, 0])) < 1e-12


def _quad_setup(seed):
    rng = np.random.default_rng(seed)
    h = 0.1
    origin = np.array([0.2, -0.4, 0.3])
    a = 1.0
    b = np.array([1.0, 2.0, 4.0]) * 0.05  # b.d != 0 for every direction d
    C = rng.uniform(-1, 1, (3, 3)) * 0.002
    C = 0.5 * (C + C.T)
    idx = np.arange(S) - G
    Z, Y, X = np.meshgrid(idx, idx, idx, indexing="ij")
    xc = np.stack([origin[0] + (X + 0.5) * h, origin[1] + (Y + 0.5) * h, origin[2] + (Z + 0.5) * h])

    def f(x):  # x [3,...]
        return a + np.tensordot(b, x, axes=1) + np.einsum("i...,ij,j...->...", x, C, x)

    avg = f(xc) + h * h * np.trace(C) / 12.0  # exact cell averages of the quadratic
    return h, origin, C, f, avg


@pytest.mark.parametrize("field", [0, 5, 6, 9])
def test_quadratic_closed_form_all_26_directions(orc, field):
    """Cell averages of f = a + b.x + x^T C x, no limiter active: PPM returns
    R_i[d] = f(x_c + h d/2) + h^2 (tr C - d^T C d)/12 on every direction."""
    h, origin, C, f, avg = _quad_setup(3 + field)
    U = uniform_subgrid(1.0, (0.0, 0.0, 0.0), 1.0)
    U[field] = avg
    if field == 0:  # density also enters v = s/rho; keep s = 0 so v = 0
        U[9] = 0.3 * avg
    cells, dirs = [], []
    for cell in [(0, 0, 0), (3, 5, 2), (7, 7, 7), (-1, 4, 4), (4, 8, 1)]:
        for d in DIRS:
            cells.append(cell)
            dirs.append(d)
    vals, flags = orc.face_values(P(orc), U, cells, dirs)
    assert not flags.any(), "the limiter must stay inactive on this field"
    for (cell, d, v) in zip(cells, dirs, vals[:, field]):
        xc = origin + (np.array(cell) + 0.5) * h
        dd = np.array(d, dtype=float)
        want = f((xc + 0.5 * h * dd)[:, None])[0] + h * h * (np.trace(C) - dd @ C @ dd) / 12.0
        assert v == pytest.approx(want, abs=2e-14), (cell, d)


def test_linear_field_point_values(orc):
    """Linear fields: every reconstructed value is the point value."""
    h = 0.25
    idx = np.arange(S) - G
    Z, Y, X = np.meshgrid(idx, idx, idx, indexing="ij")
    U = uniform_subgrid(1.0, (0.0, 0.0, 0.0), 1.0)
    g = np.array([0.3, -0.7, 1.1])
    U[5] = 2.0 + g[0] * X + g[1] * Y + g[2] * Z
    cells = [(2, 3, 4)] * 26
    vals, flags = orc.face_values(P(orc), U, cells, DIRS)
    for d, v in zip(DIRS, vals[:, 5]):
        want = 2.0 + g @ (np.array((2, 3, 4)) + 0.5 * np.array(d))
        assert v == pytest.approx(want, abs=1e-14)
    assert not flags.any()


def test_ppm_line_limiter_cases(orc):
    # extremum at the centre: flatten
    qp, qm, f = orc.ppm_line([0.0, 1.0, 2.0, 1.0, 0.0])
    assert (qp, qm, f) == (2.0, 2.0, 1)
    # step: values bounded by neighbours (monotone)
    qp, qm, f = orc.ppm_line([0.0, 0.0, 0.0, 1.0, 1.0])
    assert 0.0 <= qm <= qp <= 1.0
    # smooth cubic samples: unlimited 4th-order interface value
    s = [x ** 3 * 0.001 + 0.1 * x + 1 for x in range(-2, 3)]
    qp, qm, f = orc.ppm_line(s)
    assert f == 0
    assert qp == pytest.approx(7 / 12 * (s[2] + s[3]) - 1 / 12 * (s[1] + s[4]), rel=1e-15)
    assert qm == pytest.approx(7 / 12 * (s[1] + s[2]) - 1 / 12 * (s[0] + s[3]), rel=1e-15)
    # reversal symmetry of the line operator (bitwise)
    rng = np.random.default_rng(5)
    for _ in range(200):
        s = rng.uniform(-1, 1, 5)
        a = orc.ppm_line(s)
        b = orc.ppm_line(s[::-1].copy())
        assert a[0] == b[1] and a[1] == b[0]


def test_conservation_periodic_box(orc, oracle_mod):
    """Periodic box of 2x2x2 sub-grids, omega = 0, no gravity: the flux form
    conserves mass, momentum, energy, tracer and species to round-off."""
    from oracle import mesh
    rng = np.random.default_rng(7)
    n = 16
    rho = rng.uniform(0.5, 2.0, (n, n, n))
    v = rng.uniform(-0.5, 0.5, (3, n, n, n))
    p = rng.uniform(0.1, 1.0, (n, n, n))
    z = rng.uniform(-0.1, 0.1, (3, n, n, n))
    Ug = W.conserved_from_primitive(rho, v, p, GAMMA, z=z, species=0.4 * rho)
    run = mesh.BoxRun(P(orc), Ug, 0.1, (0.0, 0.0, 0.0), "periodic")
    dU, am = run.rhs(Ug)
    tot = dU.sum(axis=(0, 2, 3, 4))
    scale = np.abs(dU).sum(axis=(0, 2, 3, 4))
    for k in (0, 1, 2, 3, 4, 5, 9):
        assert abs(tot[k]) <= 1e-13 * scale[k], (k, tot[k], scale[k])


def test_angular_momentum_conserved_by_fluxes(orc):
    """sum(x_c x s + z) has zero rate when no flux crosses the boundary with a
    lever arm: a perturbation at the centre of a periodic box at rest."""
    from oracle import mesh
    rng = np.random.default_rng(11)
    n, h = 24, 0.1
    rho = np.ones((n, n, n))
    v = np.zeros((3, n, n, n))
    p = np.full((n, n, n), 0.5)
    z = np.zeros((3, n, n, n))
    c = slice(8, 16)
    rho[c, c, c] = rng.uniform(0.5, 2.0, (8, 8, 8))
    v[:, c, c, c] = rng.uniform(-0.5, 0.5, (3, 8, 8, 8))
    p[c, c, c] = rng.uniform(0.2, 1.0, (8, 8, 8))
    z[:, c, c, c] = rng.uniform(-0.1, 0.1, (3, 8, 8, 8))
    Ug = W.conserved_from_primitive(rho, v, p, GAMMA, z=z)
    lo = (-1.2, -1.2, -1.2)
    run = mesh.BoxRun(P(orc), Ug, h, lo, "periodic")
    dU, _ = run.rhs(Ug)
    dUg = mesh.join(dU, run.nbx, run.nby, run.nbz)
    X, Y, Z = W.cell_centres((n, n, n), lo, h)
    ds = dUg[1:4]
    torque = np.stack([Y * ds[2] - Z * ds[1], Z * ds[0] - X * ds[2], X * ds[1] - Y * ds[0]])
    Ldot = (torque + dUg[6:9]).sum(axis=(1, 2, 3))
    scale = np.abs(torque).sum(axis=(1, 2, 3))
    assert np.all(np.abs(Ldot) <= 1e-12 * scale), (Ldot, scale)
    # and without the torque term the spin alone would not conserve it
    assert np.max(np.abs(torque.sum(axis=(1, 2, 3)))) > 1e-6 * scale.max()


def _cyc(U):
    """Relabel axes x->y, y->z, z->x: array and vector components."""
    V = np.transpose(U, (0, 2, 3, 1)).copy()  # V[k][a][b][c] = U[k][c][a][b]
    out = V.copy()
    out[1], out[2], out[3] = V[3], V[1], V[2]
    out[6], out[7], out[8] = V[8], V[6], V[7]
    return out


def test_cyclic_permutation_symmetry(orc):
    U = W.random_subgrids(1, 13)[0]
    dU, am, _ = orc.step(P(orc), U[None], np.zeros(3), 0.07)
    Up = _cyc(U)
    dUp, amp, _ = orc.step(P(orc), Up[None], np.zeros(3), 0.07)
    want = _cyc(dU[0])
    scale = np.abs(dU[0]).max(axis=(1, 2, 3))[:, None, None, None]
    assert np.all(np.abs(dUp[0] - want) <= 1e-13 * scale)
    assert amp[0] == pytest.approx(am[0], rel=1e-15)


def test_flux_consistency_and_dissipation_sign(orc):
    Pp = P(orc)
    q = np.array([1.2, 0.3, -0.4, 0.5, 0.9, 0.7, 0.01, 0.02, 0.03, 0.5])
    for a in range(3):
        F, aq = orc.point_flux(Pp, q, q, a, np.zeros(3))
        un = q[1 + a]
        p = (GAMMA - 1) * q[4]
        assert F[0] == pytest.approx(q[0] * un, rel=1e-15)
        assert F[1 + a] == pytest.approx(q[0] * q[1 + a] * un + p, rel=1e-14)
        assert F[9] == pytest.approx(q[9] * un, rel=1e-15)
        assert aq == pytest.approx(abs(un) + math.sqrt(GAMMA * p / q[0]), rel=1e-15)
    # static contact: mass diffuses from the dense side to the light side
    qL = np.array([2.0, 0, 0, 0, 1.0, 1.0, 0, 0, 0, 2.0])
    qR = np.array([1.0, 0, 0, 0, 1.0, 1.0, 0, 0, 0, 1.0])
    F, aq = orc.point_flux(Pp, qL, qR, 0, np.zeros(3))
    assert F[0] > 0 and F[0] == pytest.approx(0.5 * aq * (2.0 - 1.0))
    # mirror: swap sides and reverse the normal velocity -> scalar fluxes flip
    qL2 = np.array([1.1, 0.3, 0.1, -0.2, 0.8, 0.6, 0, 0, 0, 0.4])
    qR2 = np.array([0.7, -0.2, 0.2, 0.1, 0.5, 0.4, 0, 0, 0, 0.3])
    F1, a1 = orc.point_flux(Pp, qL2, qR2, 1, np.zeros(3))
    mL, mR = qR2.copy(), qL2.copy()
    mL[2] *= -1
    mR[2] *= -1
    F2, a2 = orc.point_flux(Pp, mL, mR, 1, np.zeros(3))
    assert a1 == a2
    for k in (0, 1, 3, 4, 5, 9):
        assert F2[k] == pytest.approx(-F1[k], rel=1e-14, abs=1e-15)
    assert F2[2] == pytest.approx(F1[2], rel=1e-14)


def _ppm1d(q):
    """Independent 1-D PPM (periodic), numpy; returns (qp, qm) per cell."""
    dl = np.roll(q, -1) - q  # delta_j = q_{j+1} - q_j
    a, b = np.roll(dl, 1), dl  # delta_{j-1}, delta_j
    m = np.minimum(np.minimum(2 * np.abs(a), 2 * np.abs(b)), 0.5 * np.abs(a + b))
    D = np.where(a * b <= 0, 0.0, np.where(b > 0, m, -m))
    qp = 0.5 * (q + np.roll(q, -1)) - (np.roll(D, -1) - D) / 6.0
    qm = 0.5 * (np.roll(q, 1) + q) - (D - np.roll(D, 1)) / 6.0
    ext = (qp - q) * (q - qm) <= 0
    dq = qp - qm
    lhs = dq * (q - 0.5 * (qp + qm))
    rhs = dq * dq / 6.0
    qp2 = np.where(ext, q, np.where((~ext) & (lhs < -rhs), 3 * q - 2 * qm, qp))
    qm2 = np.where(ext, q, np.where((~ext) & (lhs > rhs), 3 * q - 2 * qp, qm))
    return qp2, qm2


def test_one_dimensional_reduction(orc):
    """Data varying only along x: the 3-D scheme equals a 1-D PPM + KT scheme."""
    rng = np.random.default_rng(17)
    nx, h = 8, 0.125
    rho = rng.uniform(0.5, 2.0, nx)
    vx = rng.uniform(-0.5, 0.5, nx)
    p = rng.uniform(0.2, 1.0, nx)
    sh = (8, 8, nx)
    Ug = W.conserved_from_primitive(np.broadcast_to(rho, sh), np.stack([np.broadcast_to(vx, sh), np.zeros(sh),
                                                                        np.zeros(sh)]), np.broadcast_to(p, sh), GAMMA)
    Up = np.pad(Ug, ((0, 0), (G, G), (G, G), (G, G)), mode="wrap")
    dU, am, _ = orc.step(P(orc), Up[None], np.zeros(3), h)
    # 1-D reference
    eps = Ug[4, 0, 0] - 0.5 * Ug[1, 0, 0] ** 2 / Ug[0, 0, 0]
    prims = [rho, vx, eps, Ug[5, 0, 0], Ug[9, 0, 0]]
    rec = [_ppm1d(q) for q in prims]
    L = [r[0] for r in rec]  # left state of face i+1/2 = qp of cell i
    R = [np.roll(r[1], -1) for r in rec]  # right state = qm of cell i+1

    def flux(st):
        r, u, e, t, sp = st
        pp = (GAMMA - 1) * e
        E = e + 0.5 * r * u * u
        Uc = np.stack([r, r * u, E, t, sp])
        F = np.stack([r * u, r * u * u + pp, (E + pp) * u, t * u, sp * u])
        return Uc, F, np.abs(u) + np.sqrt(GAMMA * pp / r)

    UL, FL, sL = flux(L)
    UR, FR, sR = flux(R)
    a = np.maximum(sL, sR)
    Fh = 0.5 * (FL + FR) - 0.5 * a * (UR - UL)
    div = -(Fh - np.roll(Fh, 1, axis=1)) / h
    got = dU[0][[0, 1, 4, 5, 9]][:, 3, 4, :]  # any transverse position
    scale = np.abs(div).max(axis=1)[:, None]
    assert np.all(np.abs(got - div) <= 1e-13 * scale)
    assert np.all(np.abs(dU[0][[2, 3, 6, 7, 8]]) <= 1e-13 * scale.max())
    assert am[0] == pytest.approx(a.max(), rel=1e-14)


def test_rk3_stage_coefficients(orc):
    """Driving the update with dU/dt = lam * U reproduces the SSP-RK3
    stability polynomial 1 + z + z^2/2 + z^3/6 (z = lam dt) on every field
    that the tracer resync leaves alone."""
    Pp = P(orc, eta2=2.0)  # eps_E > 2E never holds: no resync
    U = W.random_subgrids(1, 3)[0]
    lam, dt = -0.7, 0.13
    U0 = U.copy()
    Us = U.copy()
    for k in range(3):
        dU = lam * Us[:, G:-G, G:-G, G:-G][None]
        Us = orc.update(Pp, Us[None], U0[None], dU, dt, k)[0]
    z = lam * dt
    want = U0[:, G:-G, G:-G, G:-G] * (1 + z + z * z / 2 + z ** 3 / 6)
    assert np.allclose(Us[:, G:-G, G:-G, G:-G], want, rtol=1e-14, atol=0)
    assert np.array_equal(Us[:, :G], U0[:, :G])  # ghosts untouched


def test_dual_energy_selection_and_resync(orc):
    Pp = P(orc)
    # thermal-dominated cell: eps from E - KE
    u = np.array([1.0, 0.1, 0, 0, 2.0, 0.123, 0, 0, 0, 1.0])
    q = orc.primitives(Pp, u)
    assert q[4] == pytest.approx(2.0 - 0.005, rel=1e-15)
    # kinetic-dominated cell (E - KE < eta1 E): eps from the tracer
    u = np.array([1.0, 2.0, 0, 0, 2.0000001, 0.5, 0, 0, 0, 1.0])
    q = orc.primitives(Pp, u)
    assert q[4] == pytest.approx(0.5 ** GAMMA, rel=1e-15)
    # resync: update with zero rate resets tau where eps_E > eta2 E only
    U = uniform_subgrid(1.0, (0.0, 0.0, 0.0), 1.0)
    U[5] = 0.01  # inconsistent tracer
    U[1, G:G + 4] = 1.9  # fast (KE dominated) in the lower half of the cells
    U[4, G:G + 4] = 0.5 * 1.9 ** 2 + 0.01
    out = orc.update(Pp, U[None], U[None], np.zeros((1, 10, N, N, N)), 0.1, 0)[0]
    eps_slow = 1.0 / (GAMMA - 1.0)
    assert out[5, G + 6, G + 2, G + 2] == pytest.approx(eps_slow ** (1 / GAMMA), rel=1e-15)
    assert out[5, G + 1, G + 2, G + 2] == 0.01


def test_operation_counts_are_stable(orc):
    """The counting scalar runs the same code; it must give the same result."""
    U = W.random_subgrids(1, 2)[0]
    c = orc.count_ops(P(orc), U, np.zeros(3), 0.1)
    assert c["step"]["sqrt"] == 2 * 3 * 9 * N * N * (N + 1)  # one sqrt per side per point
    assert c["step"]["div"] == 3 * S ** 3 + 2 * 3 * 9 * N * N * (N + 1)


@pytest.mark.parametrize("ax", [0, 1, 2])
def test_face_quadrature_transverse_quadratic(orc, ax):
    """The face sum of Sec. III-B ("Newtonian quadrature") on data that vary
    quadratically along one axis ax only, f(x) = a + b x_ax + c x_ax^2, with a
    uniform velocity normal to ax and a uniform pressure, seen on the faces
    whose normal is one of the other two axes (ax is then transverse to
    them).  No limiter acts, both sides of every quadrature point hold the
    same state, and the three point values across a face along ax lie on
    the quadratic g(s) = f(y_c + s) + c h^2 (1 - 4 s^2/h^2)/12 (the
    closed-form reconstruction pinned above).  The face average of the
    fluxes is then the exact mean of g and of its first moment over the
    face, which a 3-point rule reproduces only with the Simpson weights
    (exact to cubic order):
        mean g        = f(y_c) + 5 c h^2 / 36,
        mean s g(s)   = f'(y_c) h^2 / 12.
    Weights (1,2,1)/4 give c h^2/6 and f' h^2/8; the centre alone c h^2/12
    and 0; a weight table transposed between the two transverse axes, or
    not summing to 1, fails the pressure and uniform terms."""
    h = 0.05
    origin = np.array([-0.35, 0.2, -0.1])
    origin[ax] = 0.6  # every stored cell at x_ax > 0.45: f is monotone there
    a0, b0, c0 = 1.0, 0.5, 2.0
    idx = np.arange(S) - G
    yc_all = origin[ax] + (idx + 0.5) * h
    avg1 = a0 + b0 * yc_all + c0 * (yc_all ** 2 + h * h / 12.0)  # exact cell averages
    shp = [1, 1, 1]
    shp[2 - ax] = S  # array order is [z][y][x]
    rho = np.broadcast_to(avg1.reshape(shp), (S, S, S))
    vel = np.array([0.3, -0.45, 0.7])
    vel[ax] = 0.0
    p = 1.0
    U = W.conserved_from_primitive(rho, np.stack([np.full((S, S, S), c) for c in vel]), np.full((S, S, S), p),
                                   GAMMA, species=0.3 * rho)
    dU, am, _, faces = orc.step(P(orc), U[None], origin, h, faces=True)
    eps = p / (GAMMA - 1.0)
    tau = eps ** (1.0 / GAMMA)
    for a in range(3):
        if a == ax:
            continue
        b = 1 if a == 0 else 0
        cax = 1 if a == 2 else 2
        ua = vel[a]
        e_a = np.eye(3)[a]
        e_ax = np.eye(3)[ax]
        for side in (0, 1):
            f = faces[0, 2 * a + side]  # [F+3][pc][pb]
            for pc in range(N):
                for pb in range(N):
                    i_ax = pb if ax == b else pc
                    y = origin[ax] + (i_ax + 0.5) * h
                    mean_g = a0 + b0 * y + c0 * y * y + 5.0 * c0 * h * h / 36.0
                    m1 = (b0 + 2.0 * c0 * y) * h * h / 12.0
                    want = np.zeros(13)
                    want[0] = ua * mean_g
                    want[1:4] = ua * vel * mean_g
                    want[1 + a] += p
                    want[4] = ua * (eps + p + 0.5 * vel @ vel * mean_g)
                    want[5] = ua * tau
                    want[9] = 0.3 * ua * mean_g
                    # torque about the adjacent interior cell: the mean of
                    # (x_q - x_c) x F_s, lever (h/2) e_a (upper face, cell on
                    # its left) or -(h/2) e_a (lower face) plus the offset in
                    # the face; the pressure part has zero mean moment
                    lever = 0.5 * h if side == 1 else -0.5 * h
                    want[10:13] = ua * (lever * mean_g * np.cross(e_a, vel) + m1 * np.cross(e_ax, vel))
                    got = f[:, pc, pb]
                    sc = np.array([abs(want[0])] + [np.abs(want[1:4]).max()] * 3 + [abs(want[4]), abs(want[5])]
                                  + [0.0] * 3 + [abs(want[9])] + [h * np.abs(want[1:4]).max()] * 3)
                    sc[6:9] = 1.0  # no spin: its fluxes vanish
                    assert np.all(np.abs(got - want) <= 1e-13 * sc), (a, side, pc, pb, got - want)
    # the rates of this stationary, uniformly moving state: only the ax-faces
    # (which see f vary along their normal) contribute; the faces pinned
    # above cancel in pairs
    assert np.all(np.isfinite(dU))
