"""The old hydro module (flux values only at the centres of cell faces, the
same reconstruction: Sec. III-B), selected with hydro_mode_t.flux_points = 1,
against the oracle's old module (pinned in test_oracle_old_hydro.py):
  * FP64 step kernel: <= 1e-12 per field and amax, on random sub-grids with
    rotation and gravity;
  * mixed step kernel: within the mixed-precision budget;
  * fused RK3 step: bit for bit equal to the separate launches;
  * invalid flux_points values are rejected.
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


def step(H, ctx, U, origin, h, g=None):
    dev = torch.device("cuda")
    n = U.shape[0]
    Ut = torch.tensor(U, device=dev)
    ot = torch.tensor(origin, device=dev)
    ht = torch.tensor(np.broadcast_to(h, (n,)).copy(), device=dev)
    gt = torch.tensor(g, device=dev) if g is not None else None
    dU = torch.full((n, 10, 8, 8, 8), np.nan, dtype=torch.float64, device=dev)
    am = torch.full((n,), np.nan, dtype=torch.float64, device=dev)
    H.hydro_step(ctx, H.make_batch(Ut, ot, ht, gt), 0.0, dU, am)
    torch.cuda.synchronize()
    return dU.cpu().numpy(), am.cpu().numpy()


@pytest.mark.parametrize("mixed", [False, True])
def test_old_module_step_matches_oracle(H, oracle_mod, mixed):
    from oracle import core
    from oracle.compare import max_rel_error, mixed_worst, rate_floor
    n = 160
    U = W.random_subgrids(n, 41, GAMMA, smooth=mixed)
    rng = np.random.default_rng(43)
    origin = rng.uniform(-1, 1, (n, 3))
    h = rng.uniform(0.01, 0.1, n)
    g = rng.uniform(-1, 1, (n, 3, 8, 8, 8))
    omega = 0.3
    ctx = H.Context(GAMMA, omega)
    H.hydro_set_mode(ctx, H.HYDRO_PREC_MIXED if mixed else H.HYDRO_PREC_FP64, flux_points=1)
    dU, am = step(H, ctx, U, origin, h, g)
    P = core.OracleParams(gamma=GAMMA, omega=omega, face_points=1)
    ref, amo, _, faces = core.step(P, U, origin, h, g, faces=True)
    assert H.hydro_status(ctx) == 0
    assert np.all(np.isfinite(dU))
    if not mixed:
        assert max_rel_error(dU, ref, h, rate_floor(U, amo, h, omega, g)) <= 1e-12
        assert np.allclose(am, amo, rtol=1e-14, atol=0)
    else:
        pert, _, _ = core.step(P, U.astype(np.float32).astype(np.float64), origin, h, g)
        worst = mixed_worst(dU, ref, pert, faces, h, U, amo)
        print("old module mixed: largest err/budget", worst)
        assert worst <= 1.0
    # and the new module gives other rates on the same data
    ref9, _, _ = core.step(core.OracleParams(gamma=GAMMA, omega=omega), U, origin, h, g)
    assert max_rel_error(ref9, ref, h) > 1e-6


def test_old_module_fused_equals_separate(H):
    from paper_2107_10987_gb300.uniform import UniformRun
    Ug, h, lo = W.sedov_box(32, GAMMA)
    U = W.box_to_subgrids(Ug)
    o, h = W.uniform_mesh(4)
    ctx = H.Context(GAMMA, 0.0)
    H.hydro_set_mode(ctx, H.HYDRO_PREC_MIXED, flux_points=1)
    sep = UniformRun(ctx, U, o, h, 4, H.HYDRO_BC_OUTFLOW)
    fus = UniformRun(ctx, U, o, h, 4, H.HYDRO_BC_OUTFLOW, fused=True)
    for _ in range(3):
        sep.step()
        fus.step()
    torch.cuda.synchronize()
    a, b = fus.interior(), sep.interior()
    assert bool((a.view(torch.int64) == b.view(torch.int64)).all())
    assert np.float64(fus.last_dt()).view(np.int64) == np.float64(sep.last_dt()).view(np.int64)
    assert H.hydro_status(ctx) == 0


def test_flux_points_validated(H):
    ctx = H.Context(GAMMA, 0.0)
    for bad in (2, 3, 8, -1, 27):
        with pytest.raises(H.HydroError):
            H.hydro_set_mode(ctx, H.HYDRO_PREC_FP64, flux_points=bad)
    for ok in (0, 1, 9):
        H.hydro_set_mode(ctx, H.HYDRO_PREC_FP64, flux_points=ok)
