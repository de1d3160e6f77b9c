"""The oracle's spin feedback pinned where it can be (CPU only).

The spin treatment of the hydro module is deferred by the paper to the
Octo-Tiger method paper, so the feedback of a cell's spin into the velocity
reconstructed at its quadrature points is a reading (a rigid rotation of the
cell's material, omega = z / I, I = rho h^2 / 6, added as omega x (x_q - x_c),
subsonic at the cell's corners):
parity unpinned beyond these checks, each chosen so that a plausible mistake
fails one of them:
  * rigid rotation by quadrature -> the moment of inertia (the factor 6, h^2),
                                    the orientation of the cross product
  * zero spin                    -> any stray term when z = 0
  * conservation                 -> the flux form (mass, momentum, energy,
                                    tracer, species, total angular momentum)
  * uniform spin                 -> the sign of the feedback (a uniformly
                                    spinning medium at rest must lose spin to
                                    the dissipation between counter-moving cell
                                    surfaces, and change nothing else)
  * sound-speed bound            -> the corner of a fast rotation moves at the
                                    sound speed, in the rotation's direction
"""
import numpy as np
import pytest

from paper_2107_10987_gb300 import workloads as W

GAMMA = 5.0 / 3.0


@pytest.fixture(scope="module")
def orc(oracle_mod):
    return oracle_mod.core


def test_rigid_rotation_moment_of_inertia_by_quadrature(orc):
    """A uniform cube of side h rotating rigidly at omega0 about its centre
    has spin density z = (1/h^3) integral of rho r x (omega0 x r) dV; with
    that z the feedback's velocity at r is omega0 x r.  The integral is done
    by 3-point Gauss-Legendre quadrature per axis (exact for the quadratic
    integrand), independently of the oracle's formula."""
    rng = np.random.default_rng(3)
    xg, wg = np.polynomial.legendre.leggauss(3)
    for _ in range(20):
        rho, h = rng.uniform(0.1, 10.0), rng.uniform(0.01, 1.0)
        om0 = rng.normal(0.0, 1.0, 3)
        z = np.zeros(3)
        for i, wi in zip(xg, wg):
            for j, wj in zip(xg, wg):
                for k, wk in zip(xg, wg):
                    r = 0.5 * h * np.array([i, j, k])
                    z += wi * wj * wk * rho * np.cross(r, np.cross(om0, r))
        z /= 8.0  # the weights integrate over [-1,1]^3: volume 8 in reference units
        P = orc.OracleParams(spin=1)
        for _ in range(5):
            r = rng.uniform(-0.5, 0.5, 3) * h
            dv = orc.spin_velocity(P, rho, 1e12, z, h, r)  # hot: the rotation is subsonic
            want = np.cross(om0, r)
            assert np.allclose(dv, want, rtol=1e-12, atol=1e-14 * np.abs(om0).max() * h), (dv, want)


def test_fast_rotation_is_bounded_by_the_sound_speed(orc):
    """A rotation whose corners would move faster than the cell's sound
    speed c = sqrt(gamma (gamma-1) eps / rho) is scaled down to reach c
    there: with omega perpendicular to a corner's offset the corner moves at
    exactly c, in the direction of omega x r; a slow rotation is unchanged;
    eps <= 0 (no sound speed) leaves no feedback."""
    P = orc.OracleParams(spin=1)
    rho, eps, h = 1.7, 0.3, 0.05
    c = np.sqrt(GAMMA * (GAMMA - 1.0) * eps / rho)
    r = 0.5 * h * np.array([1.0, 1.0, 1.0])
    axis = np.array([1.0, -1.0, 0.0]) / np.sqrt(2.0)  # perpendicular to r
    I = rho * h * h / 6.0
    for speed in (0.5 * c, 3.0 * c, 1e6 * c):
        om = axis * speed / np.linalg.norm(r)  # corner speed |om||r| = speed
        dv = orc.spin_velocity(P, rho, eps, I * om, h, r)
        want = np.cross(om, r) * min(1.0, c / speed)
        assert np.allclose(dv, want, rtol=1e-13, atol=0), (speed, dv, want)
        assert np.linalg.norm(dv) <= c * (1 + 1e-13)
    assert np.array_equal(orc.spin_velocity(P, rho, 0.0, I * axis, h, r), np.zeros(3))


def test_zero_spin_reduces_to_the_plain_method(orc):
    U = W.random_subgrids(6, 21, GAMMA)
    U[:, 6:9] = 0.0
    rng = np.random.default_rng(22)
    o = rng.uniform(-1, 1, (6, 3))
    h = rng.uniform(0.01, 0.1, 6)
    g = rng.normal(0, 0.1, (6, 3, 8, 8, 8))
    a = orc.step(orc.OracleParams(omega=0.3), U, o, h, g)
    b = orc.step(orc.OracleParams(omega=0.3, spin=1), U, o, h, g)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_spin_changes_the_rates(orc):
    """With a nonzero spin the feedback acts (the option is not inert)."""
    U = W.random_subgrids(2, 23, GAMMA)
    o = np.zeros((2, 3))
    h = np.full(2, 0.05)
    a = orc.step(orc.OracleParams(), U, o, h)[0]
    b = orc.step(orc.OracleParams(spin=1), U, o, h)[0]
    assert np.abs(a - b).max() > 1e-6 * np.abs(a).max()


def test_conservation_with_spin_periodic_box(orc):
    """Periodic box, omega = 0, no gravity, random spin: the flux form keeps
    mass, momentum, energy, tracer and species, and the spin torque keeps the
    total angular momentum sum(x_c x s + z), to round-off."""
    from oracle import mesh
    rng = np.random.default_rng(29)
    n, h = 16, 0.1
    rho = rng.uniform(0.5, 2.0, (n, n, n))
    v = rng.uniform(-0.5, 0.5, (3, n, n, n))
    p = rng.uniform(0.1, 1.0, (n, n, n))
    z = rng.uniform(-0.02, 0.02, (3, n, n, n))
    Ug = W.conserved_from_primitive(rho, v, p, GAMMA, z=z, species=0.4 * rho)
    lo = (-0.8, -0.8, -0.8)
    run = mesh.BoxRun(orc.OracleParams(spin=1), Ug, h, lo, "periodic")
    dU, _ = run.rhs(Ug)
    tot = dU.sum(axis=(0, 2, 3, 4))
    scale = np.abs(dU).sum(axis=(0, 2, 3, 4))
    for k in (0, 1, 2, 3, 4, 5, 9):
        assert abs(tot[k]) <= 1e-13 * scale[k], (k, tot[k], scale[k])
    # total angular momentum: only fluxes with a lever arm across the periodic
    # boundary could change it, so use a perturbation confined to the centre
    n, c = 24, slice(8, 16)
    rho = np.ones((n, n, n))
    v = np.zeros((3, n, n, n))
    p = np.full((n, n, n), 0.5)
    z = np.zeros((3, n, n, n))
    rho[c, c, c] = rng.uniform(0.5, 2.0, (8, 8, 8))
    v[:, c, c, c] = rng.uniform(-0.5, 0.5, (3, 8, 8, 8))
    p[c, c, c] = rng.uniform(0.2, 1.0, (8, 8, 8))
    z[:, c, c, c] = rng.uniform(-0.02, 0.02, (3, 8, 8, 8))
    Ug = W.conserved_from_primitive(rho, v, p, GAMMA, z=z)
    lo = (-1.2, -1.2, -1.2)
    run = mesh.BoxRun(orc.OracleParams(spin=1), Ug, h, lo, "periodic")
    dU, _ = run.rhs(Ug)
    dUg = mesh.join(dU, run.nbx, run.nby, run.nbz)
    X, Y, Z = W.cell_centres((n, n, n), lo, h)
    ds = dUg[1:4]
    torque = np.stack([Y * ds[2] - Z * ds[1], Z * ds[0] - X * ds[2], X * ds[1] - Y * ds[0]])
    Ldot = (torque + dUg[6:9]).sum(axis=(1, 2, 3))
    tscale = np.abs(torque).sum(axis=(1, 2, 3)) + np.abs(dUg[6:9]).sum(axis=(1, 2, 3))
    assert np.all(np.abs(Ldot) <= 1e-12 * tscale), (Ldot, tscale)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_uniform_spin_decays_and_changes_nothing_else(orc, axis):
    """A medium at rest with the same spin in every cell (periodic): every
    cell has the same rates, so conservation leaves density, momentum,
    energy and tracer unchanged in each, and the touching surfaces of
    neighbouring cells move against each other, so the central flux's
    dissipation takes spin away: dz/dt is antiparallel to z."""
    from oracle import mesh
    n, h, z0 = 16, 0.1, 0.01
    rho = np.full((n, n, n), 1.3)
    v = np.zeros((3, n, n, n))
    p = np.full((n, n, n), 0.7)
    z = np.zeros((3, n, n, n))
    z[axis] = z0
    Ug = W.conserved_from_primitive(rho, v, p, GAMMA, z=z)
    run = mesh.BoxRun(orc.OracleParams(spin=1), Ug, h, (0.0, 0.0, 0.0), "periodic")
    dU, _ = run.rhs(Ug)
    dUg = mesh.join(dU, run.nbx, run.nby, run.nbz)
    zdot = dUg[6 + axis]
    assert np.all(zdot < 0.0) and np.ptp(zdot) <= 1e-12 * abs(zdot).max()
    others = [k for k in (6, 7, 8) if k != 6 + axis]
    small = 1e-12 * abs(zdot).max()
    for k in [0, 1, 2, 3, 4, 5] + others:
        assert np.abs(dUg[k]).max() <= small, (k, np.abs(dUg[k]).max())
    # the plain method leaves this state unchanged altogether
    run0 = mesh.BoxRun(orc.OracleParams(), Ug, h, (0.0, 0.0, 0.0), "periodic")
    assert np.abs(run0.rhs(Ug)[0]).max() == 0.0
