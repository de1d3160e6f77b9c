"""PPM contact-discontinuity detection and steepening in the oracle (the
option Sec. III-B names, from Colella & Woodward 1984), pinned (CPU only):
  * two worked lines, computed by hand: a one-cell ramp (eta = 1) and a
    partial blend (eta = 1/2), both before and after the monotonicity fix-ups;
  * each condition of the detection on its own: an inflection is required,
    a jump below 1 % of the values is left alone, a shock (large pressure
    jump) is left alone, and eta is clamped to [0, 1];
  * the contact test, evaluated multiplied through by the two minima, gives
    the decision of the quotient form of the criterion in exact rational
    arithmetic, wherever the two sides differ by more than rounding;
  * mirror symmetry and scale invariance of the line; no change on lines of
    two values (every cell is then an extremum and is flattened);
  * on smooth data (16 cells per wavelength) nothing changes, bit for bit;
  * behaviour: an advected density contact stays sharper, the species
    follow the density, and the Sod density error near the contact falls;
  * conservation and the independence of the sub-grid cut still hold.
"""
import numpy as np
import pytest

from paper_2107_10987_gb300 import workloads as W

GAMMA = 5.0 / 3.0


@pytest.fixture(scope="module")
def orc(oracle_mod):
    return oracle_mod.core


def _eta(orc, a, rho=(1.0, 1.0), p=(1.0, 1.0), gamma=GAMMA):
    return orc.contact_eta(orc.OracleParams(gamma=gamma), a, rho, p)


def test_worked_ramp_is_fully_steepened(orc):
    # a = (0, 0, 1/2, 1, 1): second differences 1/2 and -1/2 (an inflection),
    # eta~ = -(-1/2 - 1/2) / (6 * 1) = 1/6 > 0.1, so eta = 1.  The limited
    # slopes of the neighbours vanish (one side of each is flat), so the
    # steepened values are the neighbours themselves: (qp, qm) = (1, 0); the
    # fix-ups keep them (q0 is their mean).  Plain PPM gives (5/6, 1/6).
    a = [0.0, 0.0, 0.5, 1.0, 1.0]
    assert _eta(orc, a) == 1.0
    assert orc.ppm_line_eta(a, 1.0) == (1.0, 0.0)
    qp, qm = orc.ppm_line_eta(a, 0.0)
    assert qp == pytest.approx(5 / 6, abs=1e-15) and qm == pytest.approx(1 / 6, abs=1e-15)
    assert orc.ppm_line(a)[:2] == (qp, qm)


def test_worked_partial_blend(orc):
    # a = (90, 100, 112, 120, 121): differences 10, 12, 8, 1; limited slopes
    # Delta_-1 = min(20, 24, 11) = 11, Delta_0 = min(24, 16, 10) = 10,
    # Delta_1 = min(16, 2, 4.5) = 2.  Plain interface values:
    # qp = 116 - (2 - 10)/6 = 117 1/3, qm = 106 - (10 - 11)/6 = 106 1/6.
    # Second differences 2 and -7: eta~ = 9 / (6 * 20) = 0.075, so
    # eta = 20 (0.075 - 0.05) = 1/2.  Neighbour extrapolations: 120 - 2/2 = 119
    # and 100 + 11/2 = 105.5; blends: qp = 118 1/6, qm = 105 5/6, whose mean
    # is q0, so no fix-up acts.
    a = [90.0, 100.0, 112.0, 120.0, 121.0]
    eta = _eta(orc, a)
    assert eta == pytest.approx(0.5, abs=4e-15)
    qp, qm = orc.ppm_line_eta(a, eta)
    assert qp == pytest.approx(118 + 1 / 6, abs=1e-12)
    assert qm == pytest.approx(105 + 5 / 6, abs=1e-12)
    qp0, qm0 = orc.ppm_line_eta(a, 0.0)
    assert qp0 == pytest.approx(117 + 1 / 3, abs=1e-12)
    assert qm0 == pytest.approx(106 + 1 / 6, abs=1e-12)


def test_steepened_values_still_pass_the_fix_ups(orc):
    # a blend that overshoots: steep ramp into a cell at the top of its
    # neighbourhood; after the blend the monotonicity fix-ups still apply, so
    # the result lies between the neighbours' values
    rng = np.random.default_rng(3)
    for _ in range(2000):
        a = np.cumsum(rng.uniform(0.0, 1.0, 5)) * rng.choice([-1.0, 1.0])
        a[rng.integers(0, 5)] += rng.normal(0.0, 2.0)
        for eta in (0.0, 0.3, 1.0):
            qp, qm = orc.ppm_line_eta(a, eta)
            lo, hi = min(a[1:4]), max(a[1:4])
            assert lo - 1e-12 <= qp <= hi + 1e-12 and lo - 1e-12 <= qm <= hi + 1e-12, (a, eta, qp, qm)


def test_detection_conditions(orc):
    # no inflection (both second differences positive): nothing
    assert _eta(orc, [0.0, 1.0, 3.0, 6.0, 10.0]) == 0.0
    # a 0.8 % jump of values near 100 is below eps = 1 %; a 2 % jump is not
    assert _eta(orc, [100.0, 100.0, 100.4, 100.8, 100.8]) == 0.0
    assert _eta(orc, [100.0, 100.0, 101.0, 102.0, 102.0]) == 1.0
    # the same jump with a shock's pressure ratio is not a contact:
    # gamma K0 |drho|/min(rho) = (5/3)(0.1)(1) = 1/6 < |dp|/min(p) = 9
    a = [1.0, 1.0, 1.5, 2.0, 2.0]
    assert _eta(orc, a, rho=(1.0, 2.0), p=(1.0, 1.0)) == 1.0
    assert _eta(orc, a, rho=(1.0, 2.0), p=(1.0, 10.0)) == 0.0
    # a small pressure jump (10 %) stays below 1/6: still a contact
    assert _eta(orc, a, rho=(1.0, 2.0), p=(1.0, 1.1)) == 1.0
    # and the boundary of the test moves with gamma: at gamma = 1.2 the bound
    # is 0.12, below a 15 % pressure jump, at 5/3 it is 1/6, above it
    assert _eta(orc, a, rho=(1.0, 2.0), p=(1.0, 1.15), gamma=1.2) == 0.0
    assert _eta(orc, a, rho=(1.0, 2.0), p=(1.0, 1.15)) == 1.0
    # eta~ around the threshold eta2 = 0.05 and the clamp at 0.1:
    # a = (0, e, 1/2, 1-e, 1) gives d2 = +-(1/2 - 2e) and eta~ = (1 - 4e) / (6 (1 - 2e)),
    # 0.036 at e = 0.22 (below eta2), 0.056 at 0.2, 0.095 at 0.15, 0.125 at 0.1
    for e, want in ((0.22, 0.0), (0.2, 20 * (0.2 / 3.6 - 0.05)), (0.15, 20 * (0.4 / 4.2 - 0.05)), (0.1, 1.0)):
        got = _eta(orc, [0.0, e, 0.5, 1 - e, 1.0])
        assert got == pytest.approx(want, abs=1e-14), (e, got, want)


def test_contact_test_is_the_exact_criterion(orc):
    """gamma K0 |drho| / min(rho) >= |dp| / min(p), decided in exact rational
    arithmetic (gamma and K0 as the oracle's doubles), against the oracle's
    decision on lines that steepen fully whenever the test passes.  Cases
    whose two sides agree to 1e-12 are skipped: there rounding decides, in
    either form."""
    from fractions import Fraction as Fr
    rng = np.random.default_rng(17)
    a = [1.0, 1.0, 1.5, 2.0, 2.0]
    n_pass = n_fail = 0
    for i in range(4000):
        gamma = (GAMMA, 1.4, 1.2)[i % 3]
        rho = rng.uniform(0.1, 3.0, 2)
        # pressure jumps spread around the test's boundary
        p0 = rng.uniform(0.01, 5.0)
        rel = float(gamma) * 0.1 * abs(rho[1] - rho[0]) / min(rho) * rng.uniform(0.5, 1.5)
        p1 = p0 * (1.0 + rel) if rng.random() < 0.5 else p0 / (1.0 + rel)
        lhs = Fr(gamma) * Fr(0.1) * abs(Fr(rho[1]) - Fr(rho[0])) / min(Fr(rho[0]), Fr(rho[1]))
        rhs = abs(Fr(p1) - Fr(p0)) / min(Fr(p0), Fr(p1))
        if abs(lhs - rhs) <= Fr(1, 10 ** 12) * max(lhs, rhs):
            continue
        want = lhs >= rhs
        got = _eta(orc, a, tuple(rho), (p0, p1), gamma=gamma) > 0.0
        assert got == want, (gamma, rho, p0, p1, float(lhs), float(rhs))
        n_pass += want
        n_fail += not want
    assert n_pass > 1000 and n_fail > 1000


def test_mirror_and_scale(orc):
    rng = np.random.default_rng(5)
    seen = 0
    for _ in range(3000):
        a = np.sort(rng.uniform(0.5, 2.0, 5)) if rng.random() < 0.5 else rng.uniform(0.5, 2.0, 5)
        a[2] = a[1] + rng.uniform(0.0, 1.0) * (a[3] - a[1])
        rho = rng.uniform(0.5, 2.0, 2)
        p = rng.uniform(0.9, 1.1, 2)
        eta = _eta(orc, a, rho, p)
        seen += eta > 0
        # mirror: reversing the line swaps the two values and keeps eta
        assert _eta(orc, a[::-1].copy(), rho[::-1].copy(), p[::-1].copy()) == eta
        qp, qm = orc.ppm_line_eta(a, eta)
        assert orc.ppm_line_eta(a[::-1].copy(), eta) == (qm, qp)
        # a power-of-two scale of every input is exact
        assert _eta(orc, 8.0 * a, 0.25 * rho, 4.0 * p) == eta
        assert orc.ppm_line_eta(8.0 * a, eta) == (8.0 * qp, 8.0 * qm)
    assert seen > 300


def test_two_level_lines_are_flattened_either_way(orc):
    """On a line of two values every cell equals one of its neighbours, so
    the cell is a local extremum of its interface values with or without the
    blend, and the extremum fix-up takes both to the cell value: steepening
    changes nothing there (it acts on intermediate values, as in a smeared
    contact)."""
    import itertools
    for a in itertools.product((0.4, 1.0), repeat=5):
        a = np.array(a)
        eta = _eta(orc, a)
        assert orc.ppm_line_eta(a, eta) == orc.ppm_line_eta(a, 0.0) == (a[2], a[2]), (a, eta)
    # while a third value in the middle is steepened
    a = np.array([0.4, 0.4, 0.7, 1.0, 1.0])
    assert _eta(orc, a) == 1.0 and orc.ppm_line_eta(a, 1.0) == (1.0, 0.4)


def _x_box(orc, rho_x, ny=8, p=1.0, vx=0.0, frac=0.3):
    nx = rho_x.size
    sh = (ny, ny, nx)
    rho = np.broadcast_to(rho_x, sh)
    v = np.stack([np.full(sh, vx), np.zeros(sh), np.zeros(sh)])
    return W.conserved_from_primitive(rho, v, np.full(sh, p), GAMMA, species=frac * rho)


def test_smooth_data_is_untouched(orc):
    from oracle import mesh
    nx = 32
    x = (np.arange(nx) + 0.5) / nx
    Ug = _x_box(orc, 1.0 + 0.2 * np.sin(2 * np.pi * 2 * x), vx=0.7)  # 16 cells per wavelength
    out = []
    for contact in (0, 1):
        run = mesh.BoxRun(orc.OracleParams(gamma=GAMMA, contact=contact), Ug, 1.0 / nx, (0, 0, 0), "periodic")
        out.append(run.rhs(Ug)[0])
    assert np.array_equal(out[0].view(np.int64), out[1].view(np.int64))


def _advect(orc, contact, nx=32, shift=8):
    from oracle import mesh
    x = np.arange(nx)
    rho_x = np.where((x >= nx // 4) & (x < 3 * nx // 4), 1.0, 0.5)
    Ug = _x_box(orc, rho_x, vx=1.0)
    h = 1.0 / nx
    run = mesh.BoxRun(orc.OracleParams(gamma=GAMMA, contact=contact), Ug, h, (0, 0, 0), "periodic")
    run.run(shift * h)
    exact = np.roll(rho_x, shift)
    rho = run.U[0, 0, 0]
    assert np.abs(run.U[0] - rho).max() <= 1e-12  # still planar
    return rho, exact, run.U


def test_advected_contact_stays_sharper(orc):
    r0, ex, U0 = _advect(orc, 0)
    r1, _, U1 = _advect(orc, 1)
    e0 = np.abs(r0 - ex).mean()
    e1 = np.abs(r1 - ex).mean()
    assert e1 < 0.7 * e0, (e0, e1)

    def spread(r):  # sum of 4 f (1 - f) over the jump fraction f: 0 for a sharp step
        f = (r - 0.5) / 0.5
        return float((4.0 * f * (1.0 - f)).sum())

    assert spread(r1) < 0.7 * spread(r0), (spread(r0), spread(r1))
    # the species are steepened with their own weights, which equal the
    # density's up to rounding: the mass fraction stays 0.3
    assert np.abs(U1[9] / U1[0] - 0.3).max() < 1e-12
    # the total mass is the same (the fluxes are conservative either way)
    assert U1[0].sum() == pytest.approx(U0[0].sum(), rel=1e-13)


@pytest.mark.slow
def test_sod_contact_error_falls(orc):
    """Sod (gamma = 1.4) on 128 cells at t = 0.13, when the contact has moved
    15 cells from the shock (earlier it sits in the start-up transient, where
    the pressure is not yet level and the contact test refuses every line).
    The density error near the contact falls by more than a fifth, and the
    error over the tube does not grow (the shock is left alone)."""
    import math
    from oracle import analytic, mesh
    gam = 1.4
    errs = []
    for contact in (0, 1):
        U, h, lo, xi, _ = W.sod_box(128, "x", gamma=gam)
        run = mesh.BoxRun(orc.OracleParams(gamma=gam, contact=contact), U, h, lo, "periodic")
        run.run(0.13)
        d = np.where(xi >= 0.5, xi - 0.75, -(xi - 0.25))
        rho_ex, _, _ = analytic.riemann_exact(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, gam, (d / run.t).ravel())
        err = np.abs(run.U[0] - rho_ex.reshape(d.shape))
        _, u_star = analytic.riemann_star(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, gam)
        near = np.abs(np.abs(d) - u_star * run.t) < 0.05  # both mirrored contacts
        errs.append((err.mean(), err[near].mean()))
        assert math.isfinite(errs[-1][0])
    (all0, near0), (all1, near1) = errs
    assert near1 < 0.8 * near0, errs
    assert all1 < all0, errs


def test_conservation_and_cut_with_steepening(orc):
    from oracle import mesh
    rng = np.random.default_rng(19)
    n = 32
    sh = (n, n, n)
    # density contacts in a pressure-equilibrium box, with some sound
    rho = np.where(rng.random(sh) < 0.5, 1.0, 0.4) * rng.uniform(0.95, 1.05, sh)
    v = rng.uniform(-0.3, 0.3, (3,) + sh)
    p = rng.uniform(0.98, 1.02, sh)
    Ug = W.conserved_from_primitive(rho, v, p, GAMMA, species=0.5 * rho)
    h = 1.0 / n
    rates = {}
    for N in (8, 16):
        for contact in (0, 1):
            run = mesh.BoxRun(orc.OracleParams(gamma=GAMMA, N=N, contact=contact), Ug, h, (0, 0, 0), "periodic")
            dU, _ = run.rhs(Ug)
            rates[N, contact] = mesh.join(dU, run.nbx, run.nby, run.nbz)
    d = rates[8, 1]
    tot = d.sum(axis=(1, 2, 3))
    scale = np.abs(d).sum(axis=(1, 2, 3))
    for k in (0, 1, 2, 3, 4, 5, 9):
        assert abs(tot[k]) <= 1e-13 * scale[k], (k, tot[k], scale[k])
    assert np.array_equal(rates[8, 1].view(np.int64), rates[16, 1].view(np.int64))
    # steepening acts on this machine, on density and species only
    diff = np.abs(rates[8, 1] - rates[8, 0]).max(axis=(1, 2, 3))
    assert diff[0] > 1e-3 * np.abs(rates[8, 0][0]).max()
    assert diff[9] > 1e-3 * np.abs(rates[8, 0][9]).max()


def test_steepening_with_the_smoothness_mask(orc):
    """With the learned indicator's mask: cells marked smooth take the
    unlimited formula and are not steepened, the others are.  So an empty
    mask gives the steepened step and a full mask the unsteepened masked
    step, bit for bit."""
    n = 6
    U = W.contact_subgrids(n, 5, GAMMA)
    rng = np.random.default_rng(6)
    origin = rng.uniform(-1, 1, (n, 3))
    h = rng.uniform(0.01, 0.1, n)
    P1 = orc.OracleParams(gamma=GAMMA, contact=1)
    P0 = orc.OracleParams(gamma=GAMMA)
    none = np.zeros((n, 14, 14, 14), dtype=np.uint8)
    full = np.ones((n, 14, 14, 14), dtype=np.uint8)
    d1, a1, _ = orc.step(P1, U, origin, h)
    m1, b1 = orc.step_masked(P1, U, origin, h, none)
    assert np.array_equal(d1.view(np.int64), m1.view(np.int64)) and np.array_equal(a1, b1)
    f1, _ = orc.step_masked(P1, U, origin, h, full)
    f0, _ = orc.step_masked(P0, U, origin, h, full)
    assert np.array_equal(f1.view(np.int64), f0.view(np.int64))
    # and steepening does act where the mask is empty
    d0, _, _ = orc.step(P0, U, origin, h)
    assert np.abs(d1 - d0).max() > 1e-3 * np.abs(d0).max()
