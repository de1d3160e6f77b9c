"""Pins of the oracle's gravity and rotating-frame terms and of the rotating
polytrope's initial state, on the CPU.

* a uniform stream in a uniform gravitational field: Newton's second law,
  ds/dt = rho g and dE/dt = s.g, nothing else changes;
* a uniform stream with spin seen from a rotating frame: the components of
  s and z rotate, ds/dt = -Omega x s and dz/dt = -Omega x z, with no flux
  divergence and no spin generated (a uniform flow carries no torque);
* a compact blob with radial motion in a rotating frame: the total angular
  momentum about the rotation axis, sum (x_c x s + z)_z h^3, has zero rate,
  while the frame source on s alone does not;
* the polytrope model: hydrostatic equilibrium dp/dr = -rho G M(r)/r^2 on
  the Lane-Emden profile, its mass integral, and the residual of the
  discrete step on the non-rotating star, which vanishes under refinement
  with the gravity source and stays at 2 rho|g| with its sign flipped;
* the rotating polytrope's total angular momentum about z changes only with
  the ambient gas exchanged through the outflow boundary: its drift over a
  few steps scales with the ambient density.
"""
import math

import numpy as np
import pytest

from paper_2107_10987_gb300 import workloads as W

GAMMA = 5.0 / 3.0


def _uniform_subgrid(rho, v, p, z):
    u = W.conserved_from_primitive(np.array(rho), np.array(v), np.array(p), GAMMA, z=np.array(z))
    return np.broadcast_to(u[:, None, None, None], (10, 14, 14, 14)).copy()[None]


def test_uniform_stream_in_uniform_gravity(oracle_mod):
    core = oracle_mod.core
    rho, v, p = 1.3, np.array([0.4, -0.25, 0.7]), 0.9
    U = _uniform_subgrid(rho, v, p, [0.0, 0.0, 0.0])
    gv = np.array([0.3, -1.1, 0.45])
    g = np.broadcast_to(gv[None, :, None, None, None], (1, 3, 8, 8, 8)).copy()
    dU, _, _ = core.step(core.OracleParams(gamma=GAMMA), U, np.array([-0.3, 0.1, 0.2]), 0.05, g)
    want = np.zeros(10)
    want[1:4] = rho * gv
    want[4] = rho * v @ gv
    got = dU[0].reshape(10, -1)
    assert np.all(np.abs(got - want[:, None]) <= 1e-14 * (1 + np.abs(want[:, None]))), np.abs(got - want[:, None]).max(1)


def test_uniform_stream_in_rotating_frame(oracle_mod):
    core = oracle_mod.core
    om = 0.37
    rho, v, p, z = 0.8, np.array([0.3, 0.55, -0.2]), 1.1, np.array([0.05, -0.08, 0.11])
    U = _uniform_subgrid(rho, v, p, z)
    origin = np.array([0.35, -0.6, 0.1])  # off the axis: the grid velocity varies over the sub-grid
    dU, _, _ = core.step(core.OracleParams(gamma=GAMMA, omega=om), U, origin, 0.05)
    s = rho * v
    want = np.zeros(10)
    want[1:4] = [om * s[1], -om * s[0], 0.0]
    want[6:9] = [om * z[1], -om * z[0], 0.0]
    got = dU[0].reshape(10, -1)
    assert np.all(np.abs(got - want[:, None]) <= 1e-13), np.abs(got - want[:, None]).max(1)


def _blob_box(nb, seed):
    """Compact blob with rotation and radial motion on [-1, 1]^3; at rest and
    uniform near the boundary."""
    rng = np.random.default_rng(seed)
    n = 8 * nb
    h = 2.0 / n
    X, Y, Z = W.cell_centres((n, n, n), (-1, -1, -1), h)
    r2 = X * X + Y * Y + Z * Z
    bump = np.maximum(1.0 - r2 / 0.5, 0.0) ** 2
    a = rng.uniform(0.2, 0.4, 4)
    rho = 1.0 + 0.7 * bump * (1 + 0.2 * np.sin(5 * X + 2 * Y))
    v = np.stack([bump * (a[0] * X - a[1] * Y), bump * (a[2] * Y + a[1] * X), a[3] * bump * Z])
    p = 0.6 + 0.5 * bump
    z = np.stack([0.02 * bump, -0.03 * bump, 0.05 * bump * Y])
    return W.conserved_from_primitive(rho, v, p, GAMMA, z=z), h, (X, Y, Z)


def test_angular_momentum_rate_zero_in_rotating_frame(oracle_mod):
    from oracle import mesh
    core = oracle_mod.core
    om = 0.3
    Ug, h, (X, Y, Z) = _blob_box(2, 8)
    sub = mesh.split(mesh.pad_box(Ug, 3, "outflow"), 8, 3)
    o = mesh.origins(2, 2, 2, 8, h, (-1, -1, -1))
    dU, _, _ = core.step(core.OracleParams(gamma=GAMMA, omega=om), sub, o, h)
    d = mesh.join(dU, 2, 2, 2)
    rate = ((X * d[2] - Y * d[1]) + d[8]).sum() * h ** 3
    scale = (np.abs(X * d[2]) + np.abs(Y * d[1]) + np.abs(d[8])).sum() * h ** 3
    frame = -om * (X * Ug[1] + Y * Ug[2]).sum() * h ** 3  # torque of -Omega x s alone
    assert abs(frame) > 1e-3 * scale
    assert abs(rate) <= 1e-13 * scale, (rate, scale, frame)


def test_polytrope_model_hydrostatic_and_mass():
    m = W.polytrope_model()
    xi, th, mf = m["xi"], m["theta"], m["m"]
    n, a, K, G, rc = m["n"], m["alpha"], m["K"], m["G"], m["rho_c"]
    # dp/dr = -rho G M(r) / r^2 at interior radii, by central differences of
    # p(r) = K (rho_c theta^n)^(1+1/n) on the tabulated profile
    for frac in (0.1, 0.3, 0.5, 0.7, 0.9):
        i = int(frac * (len(xi) - 1))
        r = a * xi[i]
        p = lambda j: K * (rc * th[j] ** n) ** (1 + 1 / n)
        dpdr = (p(i + 1) - p(i - 1)) / (a * (xi[i + 1] - xi[i - 1]))
        Mr = 4 * math.pi * a ** 3 * rc * mf[i]
        want = -rc * th[i] ** n * G * Mr / r ** 2
        assert dpdr == pytest.approx(want, rel=1e-5)
    # M = integral of 4 pi r^2 rho dr (trapezoid on the table)
    r = a * xi
    integrand = 4 * math.pi * r * r * rc * np.maximum(th, 0) ** n
    M = float(np.sum(0.5 * (integrand[1:] + integrand[:-1]) * np.diff(r)))
    assert M == pytest.approx(m["M"], rel=1e-6)
    assert m["omega_K"] == pytest.approx(math.sqrt(G * m["M"] / m["R"] ** 3))


def test_polytrope_state_layout():
    U, g, o, h, m = W.rotating_polytrope(2)
    assert U.shape == (8, 10, 8, 8, 8) and g.shape == (8, 3, 8, 8, 8)
    assert h == 2.0 / 16
    assert U[:, 0].min() == pytest.approx(1e-10)
    # radial, inward gravity; rigid rotation about +z inside the star
    from oracle import mesh
    Ug = mesh.join(U, 2, 2, 2)
    gb = np.stack([mesh.join(np.ascontiguousarray(g[:, k:k + 1]), 2, 2, 2)[0] for k in range(3)])
    X, Y, Z = W.cell_centres(Ug.shape[1:], (-1, -1, -1), h)
    assert np.all(X * gb[0] + Y * gb[1] + Z * gb[2] < 0)
    inside = X * X + Y * Y + Z * Z < 0.25
    w = 0.2 * m["omega_K"]
    assert np.allclose(Ug[1][inside], -w * Y[inside] * Ug[0][inside])
    assert np.allclose(Ug[2][inside], w * X[inside] * Ug[0][inside])


def _hydrostatic_residual(core, nb, sign):
    from oracle import mesh
    U, g, o, h, m = W.rotating_polytrope(nb, spin=0.0)
    Ug = mesh.join(U, nb, nb, nb)
    sub = mesh.split(mesh.pad_box(Ug, 3, "outflow"), 8, 3)
    dU, _, _ = core.step(core.OracleParams(gamma=GAMMA), sub, o, h, sign * g)
    res = np.sqrt((dU[:, 1:4] ** 2).sum(1))
    rhog = U[:, 0] * np.sqrt((g ** 2).sum(1))
    return res.sum() / rhog.sum()


def test_hydrostatic_polytrope_residual_converges(oracle_mod):
    core = oracle_mod.core
    r16 = _hydrostatic_residual(core, 2, 1.0)
    r32 = _hydrostatic_residual(core, 4, 1.0)
    assert r32 < 0.4 * r16, (r16, r32)
    assert r32 < 0.08
    # the sign of the gravity source matters: flipped, the residual is 2 rho|g|
    assert _hydrostatic_residual(core, 4, -1.0) > 1.5


def _lz_drift(core, rho_amb, steps=3):
    from oracle import mesh
    nb = 4
    U, g, o, h, m = W.rotating_polytrope(nb, rho_amb=rho_amb)
    Ug = mesh.join(U, nb, nb, nb)
    run = mesh.BoxRun(core.OracleParams(gamma=GAMMA, omega=0.2), Ug, h, (-1, -1, -1), "outflow", g=g)
    X, Y, Z = W.cell_centres(Ug.shape[1:], (-1, -1, -1), h)

    def lz(u):
        return float(((X * u[2] - Y * u[1]) + u[8]).sum() * h ** 3)

    l0 = lz(run.U)
    for _ in range(steps):
        run.step(0.4)
    return (lz(run.U) - l0) / l0


def test_polytrope_angular_momentum_drift_is_ambient_exchange(oracle_mod):
    core = oracle_mod.core
    d10 = _lz_drift(core, 1e-10)
    d13 = _lz_drift(core, 1e-13)
    assert abs(d10) < 1e-10
    assert abs(d13) < 2e-3 * abs(d10) + 1e-15, (d10, d13)
