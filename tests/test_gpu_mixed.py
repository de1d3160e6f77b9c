"""Mixed-precision step (HYDRO_PREC_MIXED) against the FP64 oracle.

Error budget, derived from the arithmetic: the mixed form rounds its inputs
(primitives) to FP32 and runs reconstruction and fluxes in FP32, keeping the
dual-energy recovery, the flux-difference accumulation, the sources and the
update in FP64.  Rounding the inputs alone changes the exact (FP64) method's
result by sens_k (measured here by running the oracle on FP32-rounded
inputs); that is the floor no FP32 method can beat.  The intermediate FP32
operations add at most a few times as much, so per field k the normalised
error (oracle/compare.py) must satisfy
    err_k <= 8 sens_k + 4e-7          (4e-7 ~ 7 units of FP32 roundoff).
Measured: random data ~2e-7, evolved Sedov ~6e-7, smooth data ~1e-5 (where
rates are an order of magnitude smaller than the fluxes they difference).
Conservation is unaffected: every face flux is computed once and enters the
two cells it separates with opposite signs in FP64.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2107_10987_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
GAMMA = 5.0 / 3.0


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2107_10987_gb300 import _build, hydro
    _build.build()
    return hydro


@pytest.fixture(scope="module")
def orc(oracle_mod):
    return oracle_mod.core


def mixed_ctx(H, omega=0.0):
    ctx = H.Context(GAMMA, omega)
    H.hydro_set_mode(ctx, H.HYDRO_PREC_MIXED)
    return ctx


def gpu_step(H, ctx, U, origin, h, g=None):
    dev = torch.device("cuda")
    n = U.shape[0]
    Ut = torch.tensor(U, device=dev)
    ot = torch.tensor(np.broadcast_to(origin, (n, 3)).copy(), device=dev)
    ht = torch.tensor(np.broadcast_to(h, (n,)).copy(), device=dev)
    gt = torch.tensor(g, device=dev) if g is not None else None
    dU = torch.full((n, 10, 8, 8, 8), np.nan, dtype=torch.float64, device=dev)
    am = torch.full((n,), np.nan, dtype=torch.float64, device=dev)
    H.hydro_step(ctx, H.make_batch(Ut, ot, ht, gt), 0.0, dU, am)
    torch.cuda.synchronize()
    return dU.cpu().numpy(), am.cpu().numpy()


def check_budget(orc, P, U, origin, h, g, dU, am):
    from oracle.compare import mixed_worst
    ref, amo, _, faces = orc.step(P, U, origin, h, g, faces=True)
    pert, _, _ = orc.step(P, U.astype(np.float32).astype(np.float64), origin, h, g)
    assert np.all(np.isfinite(dU))
    worst = mixed_worst(dU, ref, pert, faces, h, U, amo)
    print("mixed step: largest err/budget", worst)
    assert worst <= 1.0
    assert np.allclose(am, amo, rtol=1e-6, atol=0)
    return worst


@pytest.mark.parametrize("omega,gravity,smooth", [(0.0, False, False), (0.37, True, False), (0.2, True, True),
                                                  (0.0, False, True)])
def test_mixed_step_random_batches(H, orc, omega, gravity, smooth):
    n = 200
    U = W.random_subgrids(n, 100 + int(omega * 100), GAMMA, smooth=smooth)
    rng = np.random.default_rng(9)
    origin = rng.uniform(-1, 1, (n, 3))
    h = rng.uniform(0.01, 0.1, n)
    g = rng.uniform(-1, 1, (n, 3, 8, 8, 8)) if gravity else None
    dU, am = gpu_step(H, mixed_ctx(H, omega), U, origin, h, g)
    check_budget(orc, orc.OracleParams(gamma=GAMMA, omega=omega), U, origin, h, g, dU, am)


def test_mixed_step_sedov_subgrid(H, orc):
    U, h, lo = W.sedov_subgrid(GAMMA)
    dU, am = gpu_step(H, mixed_ctx(H), U[None], np.array(lo), h)
    check_budget(orc, orc.OracleParams(gamma=GAMMA), U[None], np.array(lo), h, None, dU, am)


def _run(H, ctx, Ug, h, lo, bc, nb, t_end):
    from test_gpu_parity import run_rk3_gpu
    return run_rk3_gpu(H, ctx, Ug, h, lo, bc, nb, t_end=t_end)


def sedov_l1(rho, h, lo, t):
    """L1 density error against the self-similar Sedov profile (rho0 = 1)."""
    from oracle import analytic
    lam, V, Gp, Z = analytic.sedov_profile(GAMMA)
    R = analytic.sedov_radius(1.0, 1.0, t, GAMMA)
    X, Y, Zc = W.cell_centres(rho.shape, lo, h)
    r = np.sqrt(X * X + Y * Y + Zc * Zc) / R
    ex = np.where(r < 1.0, np.interp(r, lam[::-1], Gp[::-1]), 1.0)
    return np.abs(rho - ex).sum() * h ** 3


def test_mixed_equals_fp64_l1_error_on_sedov(H):
    """Config 2 in both forms: equal L1 density error against the analytic
    profile (the discretisation error, ~1e-2, dwarfs FP32 rounding), and mass
    conserved to FP64 round-off in both."""
    Ug, h, lo = W.sedov_box(64, GAMMA)
    ctx64 = H.Context(GAMMA, 0.0)
    u64, t64, n64 = _run(H, ctx64, Ug, h, lo, "outflow", (8, 8, 8), 0.05)
    umx, tmx, nmx = _run(H, mixed_ctx(H), Ug, h, lo, "outflow", (8, 8, 8), 0.05)
    assert t64 == pytest.approx(0.05) and tmx == pytest.approx(0.05)
    l64, lmx = sedov_l1(u64[0], h, lo, t64), sedov_l1(umx[0], h, lo, tmx)
    assert abs(lmx - l64) <= 1e-3 * l64, (l64, lmx)
    assert umx[0].sum() == pytest.approx(64.0 ** 3, rel=1e-12)
    assert np.max(np.abs(umx[0] - u64[0])) <= 1e-3 * u64[0].max()


def test_mixed_conservation_periodic(H):
    from oracle import mesh
    rng = np.random.default_rng(7)
    n = 16
    Ug = W.conserved_from_primitive(rng.uniform(0.5, 2.0, (n, n, n)), rng.uniform(-0.5, 0.5, (3, n, n, n)),
                                    rng.uniform(0.1, 1.0, (n, n, n)), GAMMA, z=rng.uniform(-0.1, 0.1, (3, n, n, n)))
    sub = mesh.split(mesh.pad_box(Ug, 3, "periodic"), 8, 3)
    dU, _ = gpu_step(H, mixed_ctx(H), sub, mesh.origins(2, 2, 2, 8, 0.1, (0, 0, 0)), 0.1)
    tot = dU.sum(axis=(0, 2, 3, 4))
    scale = np.abs(dU).sum(axis=(0, 2, 3, 4))
    for k in (0, 1, 2, 3, 4, 5, 9):
        assert abs(tot[k]) <= 1e-13 * scale[k], (k, tot[k], scale[k])
