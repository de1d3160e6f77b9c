"""The two sub-grid decompositions of the mixed-precision step, and the
launch-shape autotuner, through the C ABI.

The row sweep (HYDRO_DECOMP_ROWS, the default: one thread per row of cells,
27 line evaluations per cell) and the plane sweep (HYDRO_DECOMP_PLANES: each
of the 13 lines of a cell reconstructed once, a z-plane at a time, the flux
differences kept on chip) run the same arithmetic in another order of work,
so their results are equal bit for bit:
  * the step kernel on random sub-grids with and without rotation and
    gravity, smooth and discontinuous data, both flux modules (9 points and
    the face centre), with and without contact steepening, boundary-face
    sums included;
  * the fused RK3 step in both decompositions against the separate launches
    in the other, with and without contact steepening (which the fused step
    now runs), on meshes that exercise every neighbour case and on the
    rotating polytrope with gravity;
  * every candidate launch shape of the autotuner (decomposition x
    persistent CTAs) against the default, and the autotuner's choice is one
    of them.
The row sweep is the decomposition every other mixed-precision test holds to
the oracle, so both are.  The last test prints the step kernel's time in
both decompositions.
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


def bits(t):
    return t.contiguous().view(torch.int64)


def run_step(H, ctx, U, o, h, g=None, faces=False):
    n = U.shape[0]
    dU = torch.full((n, 10, 8, 8, 8), float("nan"), dtype=torch.float64, device="cuda")
    am = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    ff = torch.full((n, 6, 13, 8, 8), float("nan"), dtype=torch.float64, device="cuda") if faces else None
    H.hydro_step(ctx, H.make_batch(U, o, h, g), 0.0, dU, am, ff)
    torch.cuda.synchronize()
    return dU, am, ff


@pytest.mark.parametrize("omega,gravity,smooth,points,contact", [
    (0.0, False, False, 9, 0), (0.37, True, False, 9, 0), (0.2, True, True, 9, 0), (0.3, True, False, 1, 0),
    (0.0, False, False, 9, 1), (0.25, True, False, 9, 1)])
def test_planes_equal_rows_bitwise(H, omega, gravity, smooth, points, contact):
    n = 300  # about two sub-grids per SM: the persistent loops wrap
    U = torch.tensor(W.random_subgrids(n, 7 + int(100 * omega) + points, GAMMA, smooth=smooth), device="cuda")
    rng = np.random.default_rng(11)
    o = torch.tensor(rng.uniform(-1, 1, (n, 3)), device="cuda")
    h = torch.tensor(rng.uniform(0.01, 0.1, n), device="cuda")
    g = torch.tensor(rng.uniform(-1, 1, (n, 3, 8, 8, 8)), device="cuda") if gravity else None
    out = {}
    for dec in (H.HYDRO_DECOMP_ROWS, H.HYDRO_DECOMP_PLANES):
        ctx = H.Context(GAMMA, omega)
        H.hydro_set_mode(ctx, H.HYDRO_PREC_MIXED, flux_points=points, contact=contact)
        H.hydro_set_launch(ctx, dec)
        assert H.hydro_get_launch(ctx)[0] == dec
        out[dec] = run_step(H, ctx, U, o, h, g, faces=True)
        assert H.hydro_status(ctx) == 0
    (a, am_a, f_a), (b, am_b, f_b) = out[H.HYDRO_DECOMP_ROWS], out[H.HYDRO_DECOMP_PLANES]
    assert bool(torch.isfinite(a).all())
    assert bool((bits(a) == bits(b)).all()), int((bits(a) != bits(b)).sum())
    assert bool((bits(am_a) == bits(am_b)).all())
    assert bool((bits(f_a) == bits(f_b)).all())


def _fused_vs_separate(H, ctx_f, ctx_s, U, o, h, nb, bc, steps, g=None):
    from paper_2107_10987_gb300.uniform import UniformRun
    sep = UniformRun(ctx_s, U, o, h, nb, bc, g)
    fus = UniformRun(ctx_f, U, o, h, nb, bc, g, fused=True)
    for k in range(steps):
        sep.step()
        fus.step()
        torch.cuda.synchronize()
        assert np.float64(fus.last_dt()).view(np.int64) == np.float64(sep.last_dt()).view(np.int64), k
        a, b = fus.interior(), sep.interior()
        same = bits(a) == bits(b)
        assert bool(same.all()), (k, int((~same).sum()), float((a - b).abs().max()))
    fus.close()
    sep.close()


def _ctx(H, omega, dec, contact=0):
    c = H.Context(GAMMA, omega)
    H.hydro_set_mode(c, H.HYDRO_PREC_MIXED, contact=contact)
    H.hydro_set_launch(c, dec)
    return c


@pytest.mark.parametrize("nb,bc", [((3, 2, 5), "periodic"), ((3, 2, 5), "outflow"), ((1, 1, 1), "periodic"),
                                   ((2, 1, 1), "outflow")])
@pytest.mark.parametrize("contact", [0, 1])
def test_fused_decompositions_against_separate_launches(H, nb, bc, contact):
    """The fused step in each decomposition against the separate launches in
    the other: the interiors after every step and every dt bit for bit."""
    from test_gpu_fused import blast_mesh
    code = {"periodic": H.HYDRO_BC_PERIODIC, "outflow": H.HYDRO_BC_OUTFLOW}[bc]
    U, o, h = blast_mesh(*nb)
    R, P = H.HYDRO_DECOMP_ROWS, H.HYDRO_DECOMP_PLANES
    for df, ds in ((P, R), (R, P)):
        cf, cs = _ctx(H, 0.0, df, contact), _ctx(H, 0.0, ds, contact)
        _fused_vs_separate(H, cf, cs, U, o, h, nb, code, steps=3)
        assert H.hydro_status(cf) == 0 and H.hydro_status(cs) == 0


def test_fused_decompositions_on_rotating_polytrope(H):
    """Rotation (omega = 0.2), the static gravity field and the thin ambient
    gas: 512 sub-grids, outflow, both decompositions crossed."""
    U, g, o, h, _ = W.rotating_polytrope(8, GAMMA)
    gt = torch.tensor(g, device="cuda")
    R, P = H.HYDRO_DECOMP_ROWS, H.HYDRO_DECOMP_PLANES
    for df, ds in ((P, R), (R, P)):
        cf, cs = _ctx(H, 0.2, df), _ctx(H, 0.2, ds)
        _fused_vs_separate(H, cf, cs, U, o, h, 8, H.HYDRO_BC_OUTFLOW, steps=2, g=gt)
        assert H.hydro_status(cf) == 0 and H.hydro_status(cs) == 0


def test_autotune_candidates_are_bitwise_equal(H):
    """Every launch shape the autotuner considers gives the default's bits;
    the autotuner keeps one of them."""
    n = 400
    U = torch.tensor(W.random_subgrids(n, 91, GAMMA), device="cuda")
    rng = np.random.default_rng(92)
    o = torch.tensor(rng.uniform(-1, 1, (n, 3)), device="cuda")
    h = torch.tensor(rng.uniform(0.01, 0.1, n), device="cuda")
    ctx = H.Context(GAMMA, 0.1)
    H.hydro_set_mode(ctx, H.HYDRO_PREC_MIXED)
    ref, am_ref, _ = run_step(H, ctx, U, o, h)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    cands = [(H.HYDRO_DECOMP_ROWS, c) for c in (sms, 3 * sms // 2, 2 * sms, -(-n // -(-n // (2 * sms))))]
    cands += [(H.HYDRO_DECOMP_PLANES, c) for c in (sms, -(-n // -(-n // sms)))]
    for dec, ctas in cands:
        H.hydro_set_launch(ctx, dec, ctas)
        assert H.hydro_get_launch(ctx) == (dec, ctas)
        dU, am, _ = run_step(H, ctx, U, o, h)
        assert bool((bits(dU) == bits(ref)).all()), (dec, ctas)
        assert bool((bits(am) == bits(am_ref)).all()), (dec, ctas)
    H.hydro_set_launch(ctx, H.HYDRO_DECOMP_AUTO, 0)
    dU = torch.empty((n, 10, 8, 8, 8), dtype=torch.float64, device="cuda")
    am = torch.empty(n, dtype=torch.float64, device="cuda")
    ctas = H.hydro_autotune_step(ctx, H.make_batch(U, o, h), dU, am)
    chosen = H.hydro_get_launch(ctx)
    assert chosen[1] == ctas and chosen in cands, (chosen, cands)
    print("autotuner's choice on", n, "random sub-grids: decomposition", chosen[0], "CTAs", chosen[1])
    dU2, am2, _ = run_step(H, ctx, U, o, h)
    assert bool((bits(dU2) == bits(ref)).all())
    # FP64 has the row sweep only
    c64 = H.Context(GAMMA, 0.0)
    with pytest.raises(H.HydroError) as e:
        H.hydro_set_launch(c64, H.HYDRO_DECOMP_PLANES)
    assert e.value.code == H.HYDRO_EUNSUP
    with pytest.raises(H.HydroError):
        H.hydro_set_launch(ctx, 7)
    assert H.hydro_status(ctx) == 0


def test_step_time_by_decomposition(H):
    """The mixed step kernel alone in both decompositions (CUDA events after
    warm-up, printed for the record): 512 Sedov sub-grids after a few steps
    and the 4,096-sub-grid polytrope."""
    from oracle import mesh
    cases = {}
    Ug, h, lo = W.sedov_box(64, GAMMA)
    cases["sedov512"] = (mesh.split(mesh.pad_box(Ug, 3, "outflow"), 8, 3), mesh.origins(8, 8, 8, 8, h, lo), h, None,
                         0.0)
    Ui, g, o, hp, _ = W.rotating_polytrope(16, GAMMA)
    Up = np.zeros((Ui.shape[0], 10, 14, 14, 14))
    Up[:, :, 3:-3, 3:-3, 3:-3] = Ui  # ghosts filled below
    cases["polytrope4096"] = (Up, o, hp, g, 0.2)
    for name, (Uc, oc, hc, gc, om) in cases.items():
        n = Uc.shape[0]
        U = torch.tensor(Uc, device="cuda")
        ot = torch.tensor(oc, device="cuda")
        ht = torch.full((n,), hc, dtype=torch.float64, device="cuda")
        gt = torch.tensor(gc, device="cuda") if gc is not None else None
        B = H.make_batch(U, ot, ht, gt)
        nb = round(n ** (1 / 3))
        H.hydro_fill_ghosts_uniform(H.Context(GAMMA, om), B, nb, nb, nb, H.HYDRO_BC_OUTFLOW)
        dU = torch.empty((n, 10, 8, 8, 8), dtype=torch.float64, device="cuda")
        am = torch.empty(n, dtype=torch.float64, device="cuda")
        t = {}
        for dec in (H.HYDRO_DECOMP_ROWS, H.HYDRO_DECOMP_PLANES):
            ctx = _ctx(H, om, dec)
            for _ in range(3):
                H.hydro_step(ctx, B, 0.0, dU, am)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(10):
                H.hydro_step(ctx, B, 0.0, dU, am)
            e1.record()
            torch.cuda.synchronize()
            t[dec] = e0.elapsed_time(e1) / 10
            assert H.hydro_status(ctx) == 0
        print(f"mixed step kernel, {name}: rows {t[H.HYDRO_DECOMP_ROWS]:.3f} ms, "
              f"planes {t[H.HYDRO_DECOMP_PLANES]:.3f} ms")
