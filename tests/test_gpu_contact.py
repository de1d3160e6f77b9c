"""PPM contact steepening (hydro_mode_t.contact = 1; the option Sec. III-B
names, after Colella & Woodward 1984) in the step kernels, through the C ABI,
against the oracle's steepening (pinned in test_oracle_contact.py):
  * FP64 step: <= 1e-12 per field on contact-rich random sub-grids with and
    without rotation and gravity.  The kernel computes the steepening
    weights with the oracle's explicitly rounded operations, so its
    decisions (contact test, inflection, jump floor) are the oracle's;
  * mixed step: within the mixed-precision budget, on sub-grids whose
    density takes the exact values 1, 1/2 and 1/4 at a level pressure:
    there every steepening decision is exact in FP32 as in FP64, so the
    comparison measures the FP32 arithmetic and not a decision that a
    rounding flips on a borderline line;
  * three RK3 steps of an advected contact: FP64 within 1e-12 of the oracle;
  * conservation on a periodic mesh, and the rates differ from the
    unsteepened ones;
  * with the learned indicator on: the cells it marks smooth take the
    unlimited formula and are not steepened, the others are; the step
    against the oracle's masked steepened step (FP64 to 1e-12, mixed within
    the budget), with a threshold placed in a gap of the network's outputs
    so that the two sides' decisions cannot differ; and the fused step with
    both options bit for bit against the separate launches;
  * the mode's checks: contact outside {0, 1} is rejected (the fused step's
    steepening itself is held to the separate launches bit for bit in
    test_gpu_planes.py).
The last test prints the step times with and without steepening.
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


def contact_subgrids(n, seed, exact=False):
    return W.contact_subgrids(n, seed, GAMMA, exact=exact)


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


@pytest.mark.parametrize("omega,gravity", [(0.0, False), (0.3, True)])
def test_fp64_contact_step_matches_oracle(H, orc, omega, gravity):
    from oracle.compare import max_rel_error, rate_floor
    n = 96
    U = contact_subgrids(n, 61)
    rng = np.random.default_rng(62)
    origin = rng.uniform(-1, 1, (n, 3))
    h = rng.uniform(0.01, 0.1, n)
    g = rng.uniform(-1, 1, (n, 3, 8, 8, 8)) if gravity else None
    ctx = H.Context(GAMMA, omega)
    H.hydro_set_mode(ctx, H.HYDRO_PREC_FP64, contact=1)
    dU, am = gpu_step(H, ctx, U, origin, h, g)
    assert H.hydro_status(ctx) == 0
    P = orc.OracleParams(gamma=GAMMA, omega=omega, contact=1)
    ref, amo, _ = orc.step(P, U, origin, h, g)
    assert np.all(np.isfinite(dU))
    assert max_rel_error(dU, ref, h, rate_floor(U, amo, h, omega, g)) <= 1e-12
    assert np.allclose(am, amo, rtol=1e-14, atol=0)
    # steepening acts on this data: the unsteepened oracle differs
    ref0, _, _ = orc.step(orc.OracleParams(gamma=GAMMA, omega=omega), U, origin, h, g)
    assert max_rel_error(ref0, ref, h) > 1e-3


def test_mixed_contact_step_within_budget(H, orc):
    from oracle.compare import mixed_budget, mixed_error, mixed_worst
    n = 96
    U = contact_subgrids(n, 71, exact=True)
    rng = np.random.default_rng(72)
    origin = rng.uniform(-1, 1, (n, 3))
    h = rng.uniform(0.01, 0.1, n)
    ctx = H.Context(GAMMA, 0.0)
    H.hydro_set_mode(ctx, H.HYDRO_PREC_MIXED, contact=1)
    dU, am = gpu_step(H, ctx, U, origin, h)
    assert H.hydro_status(ctx) == 0
    P = orc.OracleParams(gamma=GAMMA, contact=1)
    ref, amo, _, faces = orc.step(P, U, origin, h, faces=True)
    pert, _, _ = orc.step(P, U.astype(np.float32).astype(np.float64), origin, h)
    assert np.all(np.isfinite(dU))
    worst = mixed_worst(dU, ref, pert, faces, h, U, amo)
    print("mixed contact step: largest err/budget", worst)
    assert worst <= 1.0
    assert np.allclose(am, amo, rtol=1e-6, atol=0)
    # steepening is far above the budget on this data (density and species)
    budget, _ = mixed_budget(ref, pert, faces, h, U, amo)
    ref0, _, _ = orc.step(orc.OracleParams(gamma=GAMMA), U, origin, h)
    d0 = mixed_error(ref0, ref, h)
    assert d0[:, 0].max() > 100 * budget[:, 0].max() and d0[:, 9].max() > 100 * budget[:, 9].max(), (d0, budget)


def _advected_contact(nx=32):
    x = np.arange(nx)
    rho_x = np.where((x >= nx // 4) & (x < 3 * nx // 4), 1.0, 0.5)
    sh = (8, 8, nx)
    rho = np.broadcast_to(rho_x, sh)
    v = np.stack([np.full(sh, 1.0), np.full(sh, 0.1), np.zeros(sh)])
    Ug = W.conserved_from_primitive(rho, v, np.ones(sh), GAMMA, species=0.3 * rho)
    return Ug, 1.0 / nx


def test_contact_rk3_steps_match_oracle(H):
    from oracle import core, mesh
    from oracle.compare import max_rel_error, state_floor
    from paper_2107_10987_gb300.uniform import UniformRun
    Ug, h = _advected_contact()
    nbx = Ug.shape[3] // 8
    sub = np.stack([Ug[:, :, :, 8 * k:8 * k + 8] for k in range(nbx)])
    origin = np.array([[8 * k * h, 0.0, 0.0] for k in range(nbx)])
    ctx = H.Context(GAMMA, 0.0)
    H.hydro_set_mode(ctx, H.HYDRO_PREC_FP64, contact=1)
    run = UniformRun(ctx, sub, origin, h, (nbx, 1, 1), H.HYDRO_BC_PERIODIC)
    ref = mesh.BoxRun(core.OracleParams(gamma=GAMMA, contact=1), Ug, h, (0.0, 0.0, 0.0), "periodic")
    _, am0 = ref.rhs(ref.U)
    U0 = ref._sub(ref.U)
    for _ in range(3):
        run.step()
        dt_ref = ref.step(0.4)
        assert run.last_dt() == pytest.approx(dt_ref, rel=1e-14)
    got = run.interior().cpu().numpy()
    want = np.stack([ref.U[:, :, :, 8 * k:8 * k + 8] for k in range(nbx)])
    assert max_rel_error(got, want, h, state_floor(U0, am0)) <= 1e-12
    assert H.hydro_status(ctx) == 0
    run.close()


@pytest.mark.parametrize("mixed", [False, True])
def test_contact_conserves_on_periodic_mesh(H, mixed):
    from oracle import mesh
    rng = np.random.default_rng(81)
    n = 16
    sh = (n, n, n)
    # three levels: with two, every cell equals one of its line neighbours and
    # the extremum flattening takes both values to the cell's, steepened or not
    rho = rng.choice([1.0, 0.6, 0.3], size=sh)
    v = rng.uniform(-0.3, 0.3, (3,) + sh)
    Ug = W.conserved_from_primitive(rho, v, np.ones(sh), GAMMA, species=0.5 * rho)
    h = 1.0 / n
    U = torch.tensor(mesh.split(mesh.pad_box(Ug, 3, "periodic"), 8, 3), device="cuda")
    o = torch.tensor(mesh.origins(2, 2, 2, 8, h, (0.0, 0.0, 0.0)), device="cuda")
    hh = torch.full((8,), h, dtype=torch.float64, device="cuda")
    out = {}
    for contact in (0, 1):
        ctx = H.Context(GAMMA, 0.0)
        H.hydro_set_mode(ctx, H.HYDRO_PREC_MIXED if mixed else H.HYDRO_PREC_FP64, contact=contact)
        dU = torch.empty((8, 10, 8, 8, 8), dtype=torch.float64, device="cuda")
        am = torch.empty(8, dtype=torch.float64, device="cuda")
        H.hydro_step(ctx, H.make_batch(U, o, hh), 0.0, dU, am)
        torch.cuda.synchronize()
        assert H.hydro_status(ctx) == 0
        out[contact] = dU.cpu().numpy()
    d = out[1]
    tot = d.sum(axis=(0, 2, 3, 4))
    scale = np.abs(d).sum(axis=(0, 2, 3, 4))
    for k in (0, 1, 2, 3, 4, 5, 9):
        assert abs(tot[k]) <= 1e-12 * scale[k], (k, tot[k], scale[k])
    assert np.abs(out[1][:, 0] - out[0][:, 0]).max() > 1e-3 * np.abs(out[0][:, 0]).max()


def test_contact_mode_checks(H):
    ctx = H.Context(GAMMA, 0.0)
    for bad in (2, -1):
        with pytest.raises(H.HydroError):
            H.hydro_set_mode(ctx, H.HYDRO_PREC_FP64, contact=bad)


def planar_contacts(n, seed):
    """Padded sub-grids [n][F][14][14][14], each with one planar density
    contact (1 on one side, 1/4 on the other, 1/2 in the cells the plane
    passes through) at a random normal and offset through the block, level
    pressure 1, a uniform velocity
    (|v_i| <= 0.3), small uniform spin and species half the density: most
    cells sit in uniform neighbourhoods (the indicator's smooth cells), the
    rest at a contact that steepening acts on.  Density and pressure are
    exact in FP32."""
    rng = np.random.default_rng(seed)
    c = np.arange(14) - 6.5
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    out = np.empty((n, 10, 14, 14, 14))
    for i in range(n):
        nrm = rng.normal(size=3)
        nrm /= np.linalg.norm(nrm)
        dist = nrm[0] * X + nrm[1] * Y + nrm[2] * Z - rng.uniform(-3.0, 3.0)
        # 1 behind the plane, 1/4 ahead, 1/2 in the cells it passes through
        # (a contact spread over a cell, which steepening sharpens)
        rho = np.where(dist < -0.5, 1.0, np.where(dist > 0.5, 0.25, 0.5))
        sh = rho.shape
        v = np.stack([np.full(sh, rng.uniform(-0.3, 0.3)) for _ in range(3)])
        z = np.stack([np.full(sh, rng.uniform(-0.01, 0.01)) for _ in range(3)])
        out[i] = W.conserved_from_primitive(rho, v, np.ones(sh), GAMMA, z=z, species=0.5 * rho)
    return out


def _indicator_mask(U, seed):
    """Seeded indicator parameters, a threshold just above the network's
    output for a uniform neighbourhood (all features zero) and in a gap of
    at least 5e-5 to the next output, so that uniform cells are smooth and
    the GPU's and the oracle's decisions cannot differ; and the oracle's
    dilated smooth mask [n][14][14][14] on the reconstructed 10^3 block."""
    from oracle import gate
    n = U.shape[0]
    theta = np.random.default_rng(seed).normal(0, 0.3, gate.NPARAM).astype(np.float32)
    th = gate.bf16_round(theta)
    out = gate.forward_infer(th, gate.features(U, GAMMA, lo=-2, hi=10))
    c0 = float(gate.forward_infer(th, np.zeros((1, 54)))[0])
    above = out[out > c0 + 1e-7]
    gap = float(above.min()) - c0 if above.size else 1.0
    assert gap > 5e-5, gap
    thr = c0 + 0.5 * gap
    pred = (out < thr).reshape(n, 12, 12, 12)
    dil = np.ones((n, 10, 10, 10), bool)
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                dil &= pred[:, dz:dz + 10, dy:dy + 10, dx:dx + 10]
    mask = np.zeros((n, 14, 14, 14), np.uint8)
    mask[:, 2:12, 2:12, 2:12] = dil
    return theta, float(thr), mask


@pytest.mark.parametrize("fp64", [True, False])
def test_contact_with_indicator_matches_masked_oracle(H, orc, fp64):
    """Steepening together with the learned indicator: cells marked smooth
    take the unlimited formula and are not steepened, the others are
    (reading of the indicator with steepening, pinned in
    test_oracle_contact.py).  Planar contacts of density levels 1, 1/2 and
    1/4 at a level pressure: the unlimited formula stays positive there, and
    every steepening decision is exact in FP32 as in FP64."""
    from oracle.compare import max_rel_error, mixed_worst, rate_floor
    n = 12
    U = planar_contacts(n, 81)
    theta, thr, mask = _indicator_mask(U, 82)
    assert 0.02 < mask.sum() / (n * 1000) < 0.98
    rng = np.random.default_rng(83)
    origin = rng.uniform(-1, 1, (n, 3))
    h = rng.uniform(0.01, 0.1, n)
    P = orc.OracleParams(gamma=GAMMA, contact=1)
    ref, amo = orc.step_masked(P, U, origin, h, mask)
    ctx = H.Context(GAMMA, 0.0)
    H.hydro_set_mode(ctx, H.HYDRO_PREC_FP64 if fp64 else H.HYDRO_PREC_MIXED, contact=1)
    H.hydro_set_indicator(ctx, torch.tensor(theta, device="cuda"), thr)
    dU, am = gpu_step(H, ctx, U, origin, h)
    assert H.hydro_status(ctx) == 0
    assert np.all(np.isfinite(dU))
    # steepening acts on this data (the masked unsteepened step differs)
    ref_plain, _ = orc.step_masked(orc.OracleParams(gamma=GAMMA), U, origin, h, mask)
    assert max_rel_error(ref_plain, ref, h) > 1e-3
    if fp64:
        assert max_rel_error(dU, ref, h, rate_floor(U, amo, h)) <= 1e-12
        assert np.allclose(am, amo, rtol=1e-14, atol=0)
        return
    pert, _ = orc.step_masked(P, U.astype(np.float32).astype(np.float64), origin, h, mask)
    worst = mixed_worst(dU, ref, pert, None, h, U, amo)
    print("mixed contact + indicator step: largest err/budget", worst)
    assert worst <= 1.0


def test_fused_contact_with_indicator_equals_separate_launches(H):
    """The fused step with steepening and the indicator against the separate
    launches: the interiors after every step and every dt, bit for bit."""
    from paper_2107_10987_gb300.uniform import UniformRun
    nb = (3, 2, 2)
    n = nb[0] * nb[1] * nb[2]
    U = planar_contacts(n, 91)
    theta, thr, _ = _indicator_mask(U, 92)
    h = 0.05
    o = np.array([(8 * kx * h, 8 * ky * h, 8 * kz * h) for kz in range(nb[2]) for ky in range(nb[1])
                  for kx in range(nb[0])])
    runs = []
    for fused in (False, True):
        ctx = H.Context(GAMMA, 0.0)
        H.hydro_set_mode(ctx, H.HYDRO_PREC_MIXED, contact=1)
        H.hydro_set_indicator(ctx, torch.tensor(theta, device="cuda"), thr)
        runs.append((ctx, UniformRun(ctx, U, o, h, nb, H.HYDRO_BC_PERIODIC, fused=fused)))
    (cs, sep), (cf, fus) = runs
    for k in range(3):
        sep.step()
        fus.step()
        torch.cuda.synchronize()
        assert np.float64(fus.last_dt()).view(np.int64) == np.float64(sep.last_dt()).view(np.int64), k
        a, b = fus.interior(), sep.interior()
        assert bool((a.contiguous().view(torch.int64) == b.contiguous().view(torch.int64)).all()), k
    assert H.hydro_status(cs) == 0 and H.hydro_status(cf) == 0
    fus.close()
    sep.close()


def test_contact_step_cost(H):
    """Step kernel time with and without steepening on 512 sub-grids of the
    Sedov mesh (CUDA events, after warm-up; printed for the record)."""
    Ug, h, lo = W.sedov_box(64, GAMMA)
    from oracle import mesh
    U = torch.tensor(mesh.split(mesh.pad_box(Ug, 3, "outflow"), 8, 3), device="cuda")
    o = torch.tensor(mesh.origins(8, 8, 8, 8, h, lo), device="cuda")
    hh = torch.full((512,), h, dtype=torch.float64, device="cuda")
    dU = torch.empty((512, 10, 8, 8, 8), dtype=torch.float64, device="cuda")
    am = torch.empty(512, dtype=torch.float64, device="cuda")
    B = H.make_batch(U, o, hh)
    times = {}
    for prec, name in ((H.HYDRO_PREC_FP64, "fp64"), (H.HYDRO_PREC_MIXED, "mixed")):
        for contact in (0, 1):
            ctx = H.Context(GAMMA, 0.0)
            H.hydro_set_mode(ctx, prec, contact=contact)
            for _ in range(3):
                H.hydro_step(ctx, B, 0.0, dU, am)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(10):
                H.hydro_step(ctx, B, 0.0, dU, am)
            e1.record()
            torch.cuda.synchronize()
            times[name, contact] = e0.elapsed_time(e1) / 10
            assert H.hydro_status(ctx) == 0
    print("\ncontact steepening, step kernel ms on 512 sub-grids: " +
          ", ".join(f"{k[0]} contact={k[1]}: {v:.3f}" for k, v in times.items()))
    assert all(v > 0 for v in times.values())
