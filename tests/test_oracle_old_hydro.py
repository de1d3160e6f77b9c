"""The old hydro module in the oracle (flux values only at the centres of
cell faces, with the same reconstruction: Sec. III-B), pinned independently
of it (CPU only):
  * data varying along x and y: the scheme is the sum of two 1-D PPM + KT
    schemes on the lines through the cell centres, and the spin rate is the
    torque of the face-centre momentum fluxes (an independent numpy
    restatement);
  * data varying along x only: the old and new modules agree, since every
    point of a face sees the same states;
  * periodic random box: mass, momentum, energy, tracer, species and the
    total angular momentum are conserved by the fluxes.
"""
import numpy as np
import pytest

from paper_2107_10987_gb300 import workloads as W
from test_oracle_pins import GAMMA, G, P, _ppm1d


@pytest.fixture(scope="module")
def orc(oracle_mod):
    return oracle_mod.core


def _reference_2d(prim, h):
    """dU/dt of data uniform along z: for each axis a in (x, y), 1-D PPM of
    every primitive along the lines through the cell centres (periodic), the
    KT flux at the face centre, its difference, and the spin rate
    -1/2 e_a x (F_s(i+1/2) + F_s(i-1/2)) from the face-centre torques; plus
    the torques of the z faces."""
    rho, v, eps, tau, z, sp = prim
    q = [rho, v[0], v[1], v[2], eps, tau, z[0], z[1], z[2], sp]
    nf = 10
    out = np.zeros((nf,) + rho.shape)
    amax = 0.0
    for a, ax in ((0, 1), (1, 0)):  # a: x (array axis 1), y (array axis 0)
        # (qp, qm) of every line; apply_along_axis puts the pair where the axis was
        rec = [np.apply_along_axis(lambda r: np.stack(_ppm1d(r)), ax, f) for f in q]
        qp = [r[0] if ax == 0 else r[:, 0] for r in rec]
        qm = [r[1] if ax == 0 else r[:, 1] for r in rec]
        L = qp                                   # left state of face i+1/2: qp of cell i
        R = [np.roll(m, -1, axis=ax) for m in qm]  # right state: qm of cell i+1

        def cons_flux(st):
            r_, vx, vy, vz, e, t, zx, zy, zz, s = st
            pp = (GAMMA - 1) * e
            E = e + 0.5 * r_ * (vx * vx + vy * vy + vz * vz)
            Uc = np.stack([r_, r_ * vx, r_ * vy, r_ * vz, E, t, zx, zy, zz, s])
            un = (vx, vy)[a]
            F = Uc * un
            F[1 + a] = F[1 + a] + pp
            F[4] = F[4] + pp * un
            return Uc, F, np.abs(un) + np.sqrt(GAMMA * pp / r_)

        UL, FL, sL = cons_flux(L)
        UR, FR, sR = cons_flux(R)
        sp_ = np.maximum(sL, sR)
        amax = max(amax, float(sp_.max()))
        Fh = 0.5 * (FL + FR) - 0.5 * sp_ * (UR - UL)
        out += -(Fh - np.roll(Fh, 1, axis=ax + 1)) / h
        Fs = Fh[1:4] + np.roll(Fh[1:4], 1, axis=ax + 1)  # F_s(i+1/2) + F_s(i-1/2)
        e_a = np.zeros(3)
        e_a[a] = 1.0
        cross = np.stack([e_a[1] * Fs[2] - e_a[2] * Fs[1], e_a[2] * Fs[0] - e_a[0] * Fs[2],
                          e_a[0] * Fs[1] - e_a[1] * Fs[0]])
        out[6:9] += -0.5 * cross
    # z faces: the data is uniform along z, so both sides of a face hold the
    # cell's own values, the KT flux is F(q) and its difference vanishes; its
    # torque does not: -1/2 e_z x 2 F_s = (F_sy, -F_sx, 0) with
    # F_s = (rho vx vz, rho vy vz, rho vz^2 + p)
    pz = (GAMMA - 1) * eps
    out[6] += rho * v[1] * v[2]
    out[7] += -rho * v[0] * v[2]
    amax = max(amax, float((np.abs(v[2]) + np.sqrt(GAMMA * pz / rho)).max()))
    return out, amax


def test_old_module_is_two_one_dimensional_schemes(orc):
    from oracle import mesh
    rng = np.random.default_rng(23)
    n, h = 8, 0.1
    rho = rng.uniform(0.5, 2.0, (n, n))
    v = rng.uniform(-0.4, 0.4, (3, n, n))
    p = rng.uniform(0.2, 1.0, (n, n))
    sh = (n, n, n)
    b = lambda f: np.broadcast_to(f, sh)  # noqa: E731  (uniform along z: array axis 0)
    Ug = W.conserved_from_primitive(b(rho), np.stack([b(c) for c in v]), b(p), GAMMA,
                                    z=np.zeros((3,) + sh), species=b(0.3 * rho))
    run = mesh.BoxRun(P(orc, face_points=1), Ug, h, (0.0, 0.0, 0.0), "periodic")
    dU, am = run.rhs(Ug)
    got = mesh.join(dU, run.nbx, run.nby, run.nbz)[:, 0]  # one z-plane: [field][y][x]
    eps = Ug[4, 0] - 0.5 * (Ug[1, 0] ** 2 + Ug[2, 0] ** 2 + Ug[3, 0] ** 2) / Ug[0, 0]
    ref, amax = _reference_2d((rho, v, eps, Ug[5, 0], np.zeros((3, n, n)), 0.3 * rho), h)
    scale = np.abs(ref).max(axis=(1, 2))
    scale[scale == 0] = 1.0
    err = np.abs(got - ref).max(axis=(1, 2)) / scale
    assert np.all(err <= 1e-13), err
    assert float(np.max(am)) == pytest.approx(amax, rel=1e-14)
    # the spin rate is not trivially zero here: the face-centre torques act
    assert np.abs(ref[8]).max() > 1e-3 * np.abs(ref[1:3]).max()
    # and the new module differs on the same data (its 9 points see other states)
    run9 = mesh.BoxRun(P(orc), Ug, h, (0.0, 0.0, 0.0), "periodic")
    dU9, _ = run9.rhs(Ug)
    assert np.abs(mesh.join(dU9, run9.nbx, run9.nby, run9.nbz)[:, 0] - got).max() > 1e-3 * scale.max()


def test_old_and_new_agree_on_one_dimensional_data(orc):
    rng = np.random.default_rng(29)
    nx, h = 8, 0.125
    rho = rng.uniform(0.5, 2.0, nx)
    vx = rng.uniform(-0.5, 0.5, nx)
    p = rng.uniform(0.2, 1.0, nx)
    sh = (8, 8, nx)
    Ug = W.conserved_from_primitive(np.broadcast_to(rho, sh), np.stack([np.broadcast_to(vx, sh), np.zeros(sh),
                                                                        np.zeros(sh)]), np.broadcast_to(p, sh), GAMMA)
    Up = np.pad(Ug, ((0, 0), (G, G), (G, G), (G, G)), mode="wrap")
    d1, a1, _ = orc.step(P(orc, face_points=1), Up[None], np.zeros(3), h)
    d9, a9, _ = orc.step(P(orc), Up[None], np.zeros(3), h)
    # against the largest rate (the spin and transverse rates are rounding
    # noise on this data); the Simpson weights sum to 1 up to rounding
    assert np.abs(d1 - d9).max() <= 1e-14 * np.abs(d9).max()
    assert a1[0] == a9[0]


def test_old_module_conserves(orc):
    from oracle import mesh
    rng = np.random.default_rng(31)
    n, h = 16, 0.1
    rho = rng.uniform(0.5, 2.0, (n, n, n))
    v = rng.uniform(-0.5, 0.5, (3, n, n, n))
    p = rng.uniform(0.1, 1.0, (n, n, n))
    z = rng.uniform(-0.1, 0.1, (3, n, n, n))
    Ug = W.conserved_from_primitive(rho, v, p, GAMMA, z=z, species=0.4 * rho)
    lo = (-0.8, -0.8, -0.8)
    run = mesh.BoxRun(P(orc, face_points=1), Ug, h, lo, "periodic")
    dU, _ = run.rhs(Ug)
    tot = dU.sum(axis=(0, 2, 3, 4))
    scale = np.abs(dU).sum(axis=(0, 2, 3, 4))
    for k in (0, 1, 2, 3, 4, 5, 9):
        assert abs(tot[k]) <= 1e-13 * scale[k], (k, tot[k], scale[k])
    # angular momentum: a perturbation inside a box at rest, so that no flux
    # with a lever arm crosses the periodic boundary
    rho = np.ones((24, 24, 24))
    v = np.zeros((3, 24, 24, 24))
    p = np.full((24, 24, 24), 0.5)
    z = np.zeros((3, 24, 24, 24))
    c = slice(8, 16)
    rho[c, c, c] = rng.uniform(0.5, 2.0, (8, 8, 8))
    v[:, c, c, c] = rng.uniform(-0.5, 0.5, (3, 8, 8, 8))
    p[c, c, c] = rng.uniform(0.2, 1.0, (8, 8, 8))
    z[:, c, c, c] = rng.uniform(-0.1, 0.1, (3, 8, 8, 8))
    Ug = W.conserved_from_primitive(rho, v, p, GAMMA, z=z)
    lo = (-1.2, -1.2, -1.2)
    run = mesh.BoxRun(P(orc, face_points=1), Ug, h, lo, "periodic")
    dU, _ = run.rhs(Ug)
    dUg = mesh.join(dU, run.nbx, run.nby, run.nbz)
    X, Y, Z = W.cell_centres((24, 24, 24), lo, h)
    ds = dUg[1:4]
    torque = np.stack([Y * ds[2] - Z * ds[1], Z * ds[0] - X * ds[2], X * ds[1] - Y * ds[0]])
    Ldot = (torque + dUg[6:9]).sum(axis=(1, 2, 3))
    tscale = np.abs(torque).sum(axis=(1, 2, 3))
    assert np.all(np.abs(Ldot) <= 1e-12 * tscale), (Ldot, tscale)
