"""Adaptive meshes on the GPU against the oracle: the two-pass ghost fill
(bitwise), the boundary-face export and coarse-fine flux correction, whole
RK3 steps (FP64, <= 1e-12), conservation to round-off, and the batched
4,096-leaf configuration (one launch over all levels equals per-level
launches, graph replay equals direct launches)."""
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


def small():
    from test_oracle_amr import _blob_state, small_mesh
    lev, ijk = small_mesh()
    U, o, h = _blob_state(lev, ijk)
    return lev, ijk, U, o, h


@pytest.mark.parametrize("data", ["perturbed", "uniform-background"])
def test_amr_ghost_fill_bitwise(H, oracle_mod, data):
    """Both passes against the oracle's octree fill, bit for bit: on
    perturbed data, and on the blob at rest outside its compact support,
    where coarse cells with bitwise-equal neighbours are prolonged without
    arithmetic (their slopes are exactly zero) except where the value is -0
    (set in one momentum field: -0 + +0 = +0 decides some children)."""
    from oracle import amr
    from paper_2107_10987_gb300.amr import AMRMesh
    lev, ijk, U, o, h = small()
    if data == "perturbed":
        rng = np.random.default_rng(2)
        U[:, :, 3:-3, 3:-3, 3:-3] *= rng.uniform(0.9, 1.1, U[:, :, 3:-3, 3:-3, 3:-3].shape)  # non-smooth data
    else:
        sx = U[:, 1]
        sx[sx == 0.0] = -0.0
        assert np.signbit(sx).any()
    want = amr.fill_ghosts(amr.Octree(lev, ijk), U)
    ctx = H.Context(GAMMA, 0.0)
    mesh = AMRMesh(lev, ijk)
    Ut = torch.tensor(U, device="cuda")
    B = H.make_batch(Ut, torch.tensor(o, device="cuda"), torch.tensor(h, device="cuda"))
    H.hydro_fill_ghosts_amr(ctx, B, mesh)
    torch.cuda.synchronize()
    assert H.hydro_status(ctx) == 0
    assert np.array_equal(Ut.cpu().numpy(), want)


@pytest.mark.parametrize("bc", ["periodic", "outflow"])
def test_single_level_octree_equals_uniform_ghost_fill(H, bc):
    """All leaves on one level, in shuffled order: the adaptive ghost fill
    must reproduce the uniform-level fill bit for bit, including the
    wrap-around of periodic boundaries (which the oracle's octree fill does
    not model)."""
    from paper_2107_10987_gb300.amr import AMRMesh
    nb = 4
    rng = np.random.default_rng(31)
    Uu = np.zeros((nb ** 3, 10, 14, 14, 14))
    Uu[:, :, 3:-3, 3:-3, 3:-3] = rng.normal(size=(nb ** 3, 10, 8, 8, 8))
    code = {"periodic": H.HYDRO_BC_PERIODIC, "outflow": H.HYDRO_BC_OUTFLOW}[bc]
    ctx = H.Context(GAMMA, 0.0)
    # uniform fill (sub-grid s = (kz*nb + ky)*nb + kx)
    Ut = torch.tensor(Uu, device="cuda")
    z = torch.zeros((nb ** 3, 3), dtype=torch.float64, device="cuda")
    hh = torch.full((nb ** 3,), 0.1, dtype=torch.float64, device="cuda")
    H.hydro_fill_ghosts_uniform(ctx, H.make_batch(Ut, z, hh), nb, nb, nb, code)
    # the same sub-grids as level-2 leaves in shuffled order
    perm = rng.permutation(nb ** 3)
    kk = np.arange(nb ** 3)
    ijk = np.stack([kk % nb, (kk // nb) % nb, kk // (nb * nb)], 1)[perm]
    mesh = AMRMesh(np.full(nb ** 3, 2), ijk, bc=code)
    Ua = torch.tensor(Uu[perm], device="cuda")
    H.hydro_fill_ghosts_amr(ctx, H.make_batch(Ua, z, hh), mesh)
    torch.cuda.synchronize()
    assert H.hydro_status(ctx) == 0
    assert torch.equal(Ua, Ut[torch.tensor(perm, device="cuda")])


def test_amr_faces_and_flux_correction(H, oracle_mod):
    from oracle import amr, core
    from oracle.compare import max_rel_error, rate_floor
    from paper_2107_10987_gb300.amr import AMRMesh
    lev, ijk, U, o, h = small()
    tree = amr.Octree(lev, ijk)
    Uf = amr.fill_ghosts(tree, U)
    dUo, amo, _, fo = core.step(core.OracleParams(gamma=GAMMA), Uf, o, h, faces=True)
    dUc = amr.flux_correct(tree, dUo, fo, h)
    ctx = H.Context(GAMMA, 0.0)
    mesh = AMRMesh(lev, ijk)
    n = len(lev)
    Ut = torch.tensor(Uf, device="cuda")
    B = H.make_batch(Ut, torch.tensor(o, device="cuda"), torch.tensor(h, device="cuda"))
    dU = torch.empty((n, 10, 8, 8, 8), dtype=torch.float64, device="cuda")
    am = torch.empty(n, dtype=torch.float64, device="cuda")
    ff = torch.empty((n, 6, 13, 8, 8), dtype=torch.float64, device="cuda")
    H.hydro_step(ctx, B, 0.0, dU, am, ff)
    torch.cuda.synchronize()
    fs = np.abs(fo).max(axis=(0, 1, 3, 4))
    fs[fs == 0] = 1.0
    assert np.max(np.abs(ff.cpu().numpy() - fo) / fs[None, None, :, None, None]) <= 1e-13
    # correction applied to the oracle's own rates and faces: bitwise
    dUt = torch.tensor(dUo, device="cuda")
    fot = torch.tensor(fo, device="cuda")
    H.hydro_flux_correct_amr(ctx, B, mesh, fot, dUt)
    torch.cuda.synchronize()
    assert np.array_equal(dUt.cpu().numpy(), dUc)
    # and on the GPU's own step results
    H.hydro_flux_correct_amr(ctx, B, mesh, ff, dU)
    torch.cuda.synchronize()
    assert max_rel_error(dU.cpu().numpy(), dUc, h, rate_floor(Uf, amo, h)) <= 1e-12


def test_amr_rk3_steps_match_oracle_and_conserve(H, oracle_mod):
    from oracle import amr, core
    from oracle.compare import max_rel_error, state_floor
    from paper_2107_10987_gb300.amr import AMRRun
    lev, ijk, U, o, h = small()
    tree = amr.Octree(lev, ijk)
    P = core.OracleParams(gamma=GAMMA)
    Uo = U.copy()
    for _ in range(2):
        Uo, dto = amr.rk3_step(P, tree, Uo, o, h)
    ctx = H.Context(GAMMA, 0.0)
    run = AMRRun(ctx, U, lev, ijk)
    sums0 = torch.empty(11, dtype=torch.float64, device="cuda")
    B0 = H.make_batch(run.U, run.origin, run.h)
    H.hydro_conserved_sums(ctx, B0, sums0)
    for _ in range(2):
        run.step()
    torch.cuda.synchronize()
    got = run.U.cpu().numpy()[:, :, 3:-3, 3:-3, 3:-3]
    assert run.dt.item() == pytest.approx(dto, rel=1e-14)
    _, am0, _ = core.step(P, amr.fill_ghosts(tree, U), o, h)
    assert max_rel_error(got, Uo[:, :, 3:-3, 3:-3, 3:-3], h, state_floor(U, am0)) <= 1e-12
    sums1 = torch.empty(11, dtype=torch.float64, device="cuda")
    H.hydro_conserved_sums(ctx, H.make_batch(run.U, run.origin, run.h), sums1)
    torch.cuda.synchronize()
    a, b = sums0.cpu().numpy(), sums1.cpu().numpy()
    # tau is excluded: the dual-energy resync after each stage resets it
    for k in (0, 1, 2, 3, 4, 9):
        assert abs(b[k] - a[k]) <= 1e-13 * max(abs(a[k]), 1.0), (k, a[k], b[k])
    assert H.hydro_status(ctx) == 0


@pytest.mark.parametrize("mixed", [False, True])
def test_batched_4096_leaf_mesh(H, mixed, oracle_mod):
    """The batched configuration: ~4,096 leaves at levels 3-6 in shuffled order.
    One launch over all levels equals per-level launches (level-sorted copy),
    graph replays equal direct launches, mass is conserved."""
    from paper_2107_10987_gb300.amr import AMRMesh, AMRRun
    lev, ijk, th = W.amr_shell_mesh()
    U = W.amr_shell_state(lev, ijk, GAMMA)
    ctx = H.Context(GAMMA, 0.0)
    if mixed:
        H.hydro_set_mode(ctx, H.HYDRO_PREC_MIXED)
    runs = [AMRRun(ctx, U, lev, ijk) for _ in range(2)]
    for k in range(4):
        runs[0].step(use_graph=False)
        runs[1].step(use_graph=True)
    torch.cuda.synchronize()
    assert H.hydro_status(ctx) == 0
    assert torch.equal(runs[0].U, runs[1].U)
    runs[1].close()
    # per-level launches of the step on a level-sorted copy
    order = np.argsort(lev, kind="stable")
    run = runs[0]
    Ug = run.U
    B = H.make_batch(Ug, run.origin, run.h)
    H.hydro_fill_ghosts_amr(ctx, B, run.mesh)
    dU_all = torch.empty_like(run.dU)
    am_all = torch.empty_like(run.am)
    H.hydro_step(ctx, B, 0.0, dU_all, am_all)
    Us = Ug[torch.tensor(order, device="cuda")].contiguous()
    os_ = run.origin[torch.tensor(order, device="cuda")].contiguous()
    hs = run.h[torch.tensor(order, device="cuda")].contiguous()
    dU_lv = torch.empty_like(dU_all)
    am_lv = torch.empty_like(am_all)
    start = 0
    for l in np.unique(lev):
        cnt = int((lev == l).sum())
        Bl = H.make_batch(Us[start:start + cnt], os_[start:start + cnt], hs[start:start + cnt])
        H.hydro_step(ctx, Bl, 0.0, dU_lv[start:start + cnt], am_lv[start:start + cnt])
        start += cnt
    torch.cuda.synchronize()
    inv = torch.tensor(np.argsort(order), device="cuda")
    assert torch.equal(dU_lv[inv], dU_all) and torch.equal(am_lv[inv], am_all)
    # the whole-mesh launch against the oracle on 48 seeded leaves of every level
    from oracle import core
    from oracle.compare import max_rel_error, mixed_worst, rate_floor
    rng = np.random.default_rng(77)
    idx = np.unique(np.concatenate([rng.choice(np.flatnonzero(lev == l), 12, replace=False) for l in np.unique(lev)]))
    ti = torch.tensor(idx, device="cuda")
    Us = Ug[ti].cpu().numpy()
    o_s, h_s = run.origin[ti].cpu().numpy(), run.h[ti].cpu().numpy()
    P = core.OracleParams(gamma=GAMMA)
    ref, amo, _, faces = core.step(P, Us, o_s, h_s, faces=True)
    got = dU_all[ti].cpu().numpy()
    if not mixed:
        assert max_rel_error(got, ref, h_s, rate_floor(Us, amo, h_s)) <= 1e-12
        assert np.allclose(am_all[ti].cpu().numpy(), amo, rtol=1e-14, atol=0)
    else:
        pert, _, _ = core.step(P, Us.astype(np.float32).astype(np.float64), o_s, h_s)
        worst = mixed_worst(got, ref, pert, faces, h_s, Us, amo)
        print("AMR shell mixed: largest err/budget", worst)
        assert worst <= 1.0


def _manual_rk3(H, ctx, mesh, U, origin, h, steps, cfl=0.4, g=None):
    """RK3 steps through the public calls with the full two-pass ghost fill:
    ghost fill, step with boundary faces, coarse-fine flux correction, dt
    after the first stage, update.  Returns the final state and dt."""
    n = U.shape[0]
    X, Y = U.clone(), torch.zeros_like(U)
    dU = torch.empty((n, 10, 8, 8, 8), dtype=torch.float64, device="cuda")
    am = torch.empty(n, dtype=torch.float64, device="cuda")
    dt = torch.empty(1, dtype=torch.float64, device="cuda")
    faces = torch.empty((n, 6, 13, 8, 8), dtype=torch.float64, device="cuda")
    for _ in range(steps):
        for k in range(3):
            B = H.make_batch(X if k == 0 else Y, origin, h, g)
            H.hydro_fill_ghosts_amr(ctx, B, mesh)
            H.hydro_step(ctx, B, 0.0, dU, am, faces)
            H.hydro_flux_correct_amr(ctx, B, mesh, faces, dU)
            if k == 0:
                H.hydro_dt(ctx, am, h, n, cfl, dt)
            H.hydro_update(ctx, B, X, dU, 0.0, dt, k, Y if k == 0 else None)
        X, Y = Y, X
    return X, dt


@pytest.mark.parametrize("case", ["small-outflow", "small-periodic", "small-rotating", "small-gravity", "shell",
                                  "shell-indicator"])
def test_mixed_rk3_reads_neighbours_directly(H, case, oracle_mod):
    """In mixed precision the adaptive RK3 step skips the fill's copies and
    restrictions: its step kernel reads same-level neighbours' interiors and
    finer neighbours' restriction images, and only ghost cells inside coarser
    leaves are prolonged into the leaf's own array.  The state after two RK3
    steps and dt equal, bit for bit, the same sequence through the public
    calls with the full ghost fill, and so do the device status bits; the new
    state buffer's ghost cells held by same-level leaves are left unwritten
    (the direct path ran).  small-rotating: in a frame rotating at 0.2, so
    that the frame's and the spin sources act; small-gravity: with a seeded
    gravitational acceleration field."""
    from paper_2107_10987_gb300.amr import AMRRun
    if case.startswith("small"):
        lev, ijk, U, o, h = small()
        bc = H.HYDRO_BC_PERIODIC if case.endswith("periodic") else H.HYDRO_BC_OUTFLOW
    else:
        lev, ijk, _ = W.amr_shell_mesh()
        U = W.amr_shell_state(lev, ijk, GAMMA)
        bc = H.HYDRO_BC_OUTFLOW
    ctx = H.Context(GAMMA, 0.2 if case.endswith("rotating") else 0.0)
    H.hydro_set_mode(ctx, H.HYDRO_PREC_MIXED)
    if case.endswith("indicator"):
        from oracle import gate
        theta = np.random.default_rng(31).normal(0, 0.3, gate.NPARAM).astype(np.float32)
        c0 = float(gate.forward_infer(gate.bf16_round(theta), np.zeros((1, 54)))[0])
        H.hydro_set_indicator(ctx, torch.tensor(theta, device="cuda"), c0 + 1e-6)  # uniform blocks smooth
    g = None
    if case.endswith("gravity"):
        g = torch.tensor(np.random.default_rng(37).uniform(-1, 1, (len(lev), 3, 8, 8, 8)), device="cuda")
    run = AMRRun(ctx, U, lev, ijk, bc, g=g)
    run.step()
    torch.cuda.synchronize()
    # the first step's state buffer started at zero: same-level ghosts stay so
    Ug = run.U
    lo = Ug[:, 0, 0:3, 3:-3, 3:-3]  # the -z ghost layers over the leaf's face
    assert (lo == 0).any()
    run.step()
    torch.cuda.synchronize()
    st_direct = H.hydro_status(ctx)
    want, dt = _manual_rk3(H, ctx, run.mesh, torch.as_tensor(U, device="cuda"), run.origin, run.h, 2, g=g)
    torch.cuda.synchronize()
    # seeded indicator parameters may mark cells at the shell smooth, where
    # the unlimited formula can leave a non-physical state: both paths flag it
    assert H.hydro_status(ctx) == st_direct
    if not case.endswith("indicator"):
        assert st_direct == 0
    a = run.U[:, :, 3:-3, 3:-3, 3:-3].contiguous().view(torch.int64)
    b = want[:, :, 3:-3, 3:-3, 3:-3].contiguous().view(torch.int64)
    assert torch.equal(a, b)
    assert torch.equal(run.dt.view(torch.int64), dt.view(torch.int64))
    # graph replay of the direct path gives the same state
    grun = AMRRun(ctx, U, lev, ijk, bc, g=g)
    grun.step(use_graph=True)
    grun.step(use_graph=True)
    torch.cuda.synchronize()
    assert torch.equal(grun.U[:, :, 3:-3, 3:-3, 3:-3].contiguous().view(torch.int64), a)
    grun.close()
    run.close()


def test_leaf_order_changes_nothing(H, oracle_mod):
    """The order in which the kernels take the leaves (hydro_amr_t.order)
    changes no bit: the full ghost fill, flux correction and RK3 steps in
    both precisions along the Morton curve equal those in index order; an
    order entry outside the leaves is skipped and flagged (HYDRO_ST_MESH)."""
    from paper_2107_10987_gb300.amr import AMRMesh, AMRRun
    lev, ijk, _ = W.amr_shell_mesh()
    U = W.amr_shell_state(lev, ijk, GAMMA)
    for prec in (H.HYDRO_PREC_MIXED, H.HYDRO_PREC_FP64):
        ctx = H.Context(GAMMA, 0.0)
        H.hydro_set_mode(ctx, prec)
        runs = [AMRRun(ctx, U, lev, ijk, order=o) for o in ("morton", None)]
        assert runs[0].mesh.order is not None and runs[1].mesh.order is None
        for r in runs:
            for _ in range(2 if prec == H.HYDRO_PREC_MIXED else 1):
                r.step()
        torch.cuda.synchronize()
        assert H.hydro_status(ctx) == 0
        a, b = (r.U[:, :, 3:-3, 3:-3, 3:-3].contiguous().view(torch.int64) for r in runs)
        assert torch.equal(a, b)
        # the public two-pass fill in either order
        fills = []
        for r in runs:
            Ut = torch.as_tensor(U, device="cuda").clone()
            H.hydro_fill_ghosts_amr(ctx, H.make_batch(Ut, r.origin, r.h), r.mesh)
            fills.append(Ut)
        torch.cuda.synchronize()
        assert torch.equal(fills[0].view(torch.int64), fills[1].view(torch.int64))
        for r in runs:
            r.close()
    # an entry outside 0 .. n_sub-1: that unit is skipped, the status says so
    mesh = AMRMesh(lev, ijk)
    mesh.order[7] = len(lev)
    Ut = torch.as_tensor(U, device="cuda").clone()
    run = AMRRun(ctx, U, lev, ijk)
    H.hydro_fill_ghosts_amr(ctx, H.make_batch(Ut, run.origin, run.h), mesh)
    torch.cuda.synchronize()
    assert H.hydro_status(ctx) & 4
    run.close()


def test_graph_keeps_its_buffers_when_the_context_grows(H, oracle_mod):
    """A captured graph replays with the work buffers it was captured with:
    after a larger mesh has grown the context's step scratch, restriction
    images and finer-neighbour tables, the small mesh's graph still gives
    the bits of direct launches (the grown-out buffers are kept until the
    context is destroyed)."""
    from paper_2107_10987_gb300.amr import AMRRun
    lev, ijk, U, o, h = small()
    ctx = H.Context(GAMMA, 0.0)
    H.hydro_set_mode(ctx, H.HYDRO_PREC_MIXED)
    grun = AMRRun(ctx, U, lev, ijk)
    grun.step(use_graph=True)  # captured with buffers for the small mesh
    lev2, ijk2, _ = W.amr_shell_mesh()
    big = AMRRun(ctx, W.amr_shell_state(lev2, ijk2, GAMMA), lev2, ijk2)
    big.step()  # grows the context's buffers
    grun.step(use_graph=True)
    ref = AMRRun(ctx, U, lev, ijk)
    ref.step()
    ref.step()
    torch.cuda.synchronize()
    assert H.hydro_status(ctx) == 0
    a = grun.U[:, :, 3:-3, 3:-3, 3:-3].contiguous().view(torch.int64)
    b = ref.U[:, :, 3:-3, 3:-3, 3:-3].contiguous().view(torch.int64)
    assert torch.equal(a, b)
    for r in (grun, big, ref):
        r.close()


@pytest.mark.parametrize("bc", ["periodic", "outflow"])
def test_single_level_direct_rk3_equals_uniform_rk3(H, bc, oracle_mod):
    """On one level nothing is prolonged or corrected, so the mixed
    direct-read RK3 step of a single-level octree (leaves shuffled, taken
    along the Morton curve) must give the uniform mesh's RK3 step (ghost
    fill, row sweep, update) bit for bit, periodic wrap-around and outflow
    clamping included."""
    from paper_2107_10987_gb300.amr import AMRRun
    from paper_2107_10987_gb300.uniform import UniformRun
    nb = 4
    n = nb ** 3
    code = {"periodic": H.HYDRO_BC_PERIODIC, "outflow": H.HYDRO_BC_OUTFLOW}[bc]
    U = W.random_subgrids(n, 53, GAMMA)
    U[:, :, :3] = 0.0
    U[:, :, -3:] = 0.0
    U[:, :, :, :3] = 0.0
    U[:, :, :, -3:] = 0.0
    U[:, :, :, :, :3] = 0.0
    U[:, :, :, :, -3:] = 0.0
    kk = np.arange(n)
    ijk = np.stack([kk % nb, (kk // nb) % nb, kk // (nb * nb)], 1)  # s = (kz nb + ky) nb + kx
    lev = np.full(n, 2)
    o, h = W.amr_geometry(lev, ijk)
    ctx = H.Context(GAMMA, 0.0)
    H.hydro_set_mode(ctx, H.HYDRO_PREC_MIXED)
    uni = UniformRun(ctx, U, o, h, nb, code)
    perm = np.random.default_rng(59).permutation(n)
    amr = AMRRun(ctx, U[perm], lev[perm], ijk[perm], code)
    for _ in range(2):
        uni.step()
        amr.step()
    torch.cuda.synchronize()
    assert H.hydro_status(ctx) == 0
    a = amr.U[:, :, 3:-3, 3:-3, 3:-3].contiguous().view(torch.int64)
    b = uni.U[torch.tensor(perm, device="cuda")][:, :, 3:-3, 3:-3, 3:-3].contiguous().view(torch.int64)
    assert torch.equal(a, b)
    assert torch.equal(amr.dt.view(torch.int64), uni.dt.view(torch.int64))
    uni.close()
    amr.close()
