"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerance: the plain FP64 path must match the oracle to <= 1e-12 relative
error per sub-grid and field, the error of each field normalised by that
field's largest |value| in the sub-grid (a pure relative error is undefined
where dU/dt ~ 0; oracle/compare.py adds the floor for rates that are a
rounding-level residual of large flux terms).  The PPM/limiter arithmetic of the kernel is rounded exactly as
the oracle's, so limiter decisions agree; the remaining differences come
from FMA contraction and summation order in the fluxes (~1e-16 relative).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2107_10987_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-12
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


def rel_err(got, want, h=1.0, floor=None):
    from oracle.compare import max_rel_error
    return max_rel_error(got, want, h, floor)


def rate_floor(U, amax, h, omega=0.0, g=None):
    from oracle.compare import rate_floor as rf
    return rf(U, amax, h, omega, g)


def box_states(Ug, bc, rel_to=None):
    """Interior states of a joined box as [n_sub][F][8][8][8], and with
    rel_to = (P, h, lo) also the state floor of its first stage."""
    from oracle import mesh
    from oracle.compare import state_floor
    sub = mesh.unjoin(Ug, 8)
    if rel_to is None:
        return sub
    P, h, lo = rel_to
    nbz, nby, nbx = (n // 8 for n in Ug.shape[1:])
    pad = mesh.split(mesh.pad_box(Ug, 3, bc), 8, 3)
    _, am, _ = orc_step(P, pad, mesh.origins(nbx, nby, nbz, 8, h, lo), h)
    return sub, state_floor(pad, am)


def orc_step(P, U, o, h):
    from oracle import core
    return core.step(P, U, o, h)


def gpu_step(H, ctx, U, origin, h, g=None):
    dev = torch.device("cuda")
    Ut = torch.tensor(U, device=dev)
    ot = torch.tensor(np.broadcast_to(origin, (U.shape[0], 3)).copy(), device=dev)
    ht = torch.tensor(np.broadcast_to(h, (U.shape[0],)).copy(), device=dev)
    gt = torch.tensor(g, device=dev) if g is not None else None
    dU = torch.full((U.shape[0], 10, 8, 8, 8), np.nan, dtype=torch.float64, device=dev)
    am = torch.full((U.shape[0],), np.nan, dtype=torch.float64, device=dev)
    H.hydro_step(ctx, H.make_batch(Ut, ot, ht, gt), 0.0, dU, am)
    torch.cuda.synchronize()
    return dU.cpu().numpy(), am.cpu().numpy()


def test_step_sedov_subgrid(H, orc):
    """Config 1: one 8^3 Sedov sub-grid, periodic ghosts."""
    U, h, lo = W.sedov_subgrid(GAMMA)
    ctx = H.Context(GAMMA, 0.0)
    dU, am = gpu_step(H, ctx, U[None], np.array(lo), h)
    dUo, amo, _ = orc.step(orc.OracleParams(gamma=GAMMA), U[None], np.array(lo), h)
    assert rel_err(dU, dUo, h, rate_floor(U[None], amo, h)) <= TOL
    assert am[0] == pytest.approx(amo[0], rel=1e-14)
    assert H.hydro_status(ctx) == 0


@pytest.mark.parametrize("omega,gravity,smooth", [(0.0, False, False), (0.37, True, False), (0.2, True, True)])
def test_step_random_batch(H, orc, omega, gravity, smooth):
    """Random sub-grids, more than one per SM so the persistent loop wraps."""
    n = 200
    U = W.random_subgrids(n, 100 + int(omega * 100), GAMMA, smooth=smooth)
    rng = np.random.default_rng(9)
    origin = rng.uniform(-1, 1, (n, 3))
    h = rng.uniform(0.01, 0.1, n)
    g = rng.uniform(-1, 1, (n, 3, 8, 8, 8)) if gravity else None
    ctx = H.Context(GAMMA, omega)
    dU, am = gpu_step(H, ctx, U, origin, h, g)
    dUo, amo, _ = orc.step(orc.OracleParams(gamma=GAMMA, omega=omega), U, origin, h, g)
    assert np.all(np.isfinite(dU))
    assert rel_err(dU, dUo, h, rate_floor(U, amo, h, omega, g)) <= TOL
    assert np.allclose(am, amo, rtol=1e-14, atol=0)


def test_ghost_fill_bitwise(H):
    from oracle import mesh
    rng = np.random.default_rng(3)
    nbx, nby, nbz = 3, 2, 2
    Ug = rng.uniform(0.5, 1.5, (10, nbz * 8, nby * 8, nbx * 8))
    for bc, code in (("periodic", H.HYDRO_BC_PERIODIC), ("outflow", H.HYDRO_BC_OUTFLOW)):
        want = mesh.split(mesh.pad_box(Ug, 3, bc), 8, 3)
        start = want.copy()
        # scramble every ghost cell
        inner = np.zeros((14, 14, 14), bool)
        inner[3:-3, 3:-3, 3:-3] = True
        start[:, :, ~inner] = -7.0
        U = torch.tensor(start, device="cuda")
        n = U.shape[0]
        B = H.make_batch(U, torch.zeros((n, 3), dtype=torch.float64, device="cuda"),
                         torch.ones(n, dtype=torch.float64, device="cuda"))
        ctx = H.Context(GAMMA, 0.0)
        H.hydro_fill_ghosts_uniform(ctx, B, nbx, nby, nbz, code)
        torch.cuda.synchronize()
        assert np.array_equal(U.cpu().numpy(), want), bc


def test_update_and_dt_bitwise_or_ulp(H, orc):
    n = 40
    U = W.random_subgrids(n, 21, GAMMA)
    U0 = W.random_subgrids(n, 22, GAMMA)
    rng = np.random.default_rng(4)
    dUdt = rng.uniform(-1, 1, (n, 10, 8, 8, 8))
    ctx = H.Context(GAMMA, 0.0)
    dev = "cuda"
    for stage in range(3):
        Ut = torch.tensor(U, device=dev)
        B = H.make_batch(Ut, torch.zeros((n, 3), dtype=torch.float64, device=dev),
                         torch.ones(n, dtype=torch.float64, device=dev))
        H.hydro_update(ctx, B, torch.tensor(U0, device=dev), torch.tensor(dUdt, device=dev), dt=0.013, stage=stage)
        torch.cuda.synchronize()
        got = Ut.cpu().numpy()
        want = orc.update(orc.OracleParams(gamma=GAMMA), U, U0, dUdt, 0.013, stage)
        keep = [0, 1, 2, 3, 4, 6, 7, 8, 9]
        assert np.array_equal(got[:, keep], want[:, keep]), stage  # same rounded operations
        tau_err = np.abs(got[:, 5] - want[:, 5]).max() / np.abs(want[:, 5]).max()
        assert tau_err <= 1e-15  # tau from pow(): library ulps
    am = rng.uniform(0.5, 3.0, n)
    hh = rng.uniform(0.01, 0.05, n)
    out = torch.empty(1, dtype=torch.float64, device=dev)
    H.hydro_dt(ctx, torch.tensor(am, device=dev), torch.tensor(hh, device=dev), n, 0.4, out)
    torch.cuda.synchronize()
    assert out.item() == 0.4 * np.min(hh / am)


def test_conserved_sums(H):
    n = 27
    U = W.random_subgrids(n, 5, GAMMA)
    o, h = W.uniform_mesh(3)
    dev = "cuda"
    Ut = torch.tensor(U, device=dev)
    B = H.make_batch(Ut, torch.tensor(o, device=dev), torch.full((n,), h, dtype=torch.float64, device=dev))
    sums = torch.empty(11, dtype=torch.float64, device=dev)
    ctx = H.Context(GAMMA, 0.0)
    H.hydro_conserved_sums(ctx, B, sums)
    torch.cuda.synchronize()
    inner = U[:, :, 3:-3, 3:-3, 3:-3]
    want = inner.sum(axis=(0, 2, 3, 4)) * h ** 3
    assert np.allclose(sums.cpu().numpy()[:10], want, rtol=1e-13)
    idx = (np.arange(8) + 0.5) * h
    X = o[:, 0, None, None, None] + idx[None, None, None, :]
    Y = o[:, 1, None, None, None] + idx[None, None, :, None]
    Lz = ((X * inner[:, 2] - Y * inner[:, 1]) + inner[:, 8]).sum() * h ** 3
    assert sums.cpu().numpy()[10] == pytest.approx(Lz, rel=1e-12, abs=1e-14)


def run_rk3_gpu(H, ctx, Ug, h, lo, bc, nb, steps=1, t_end=None, cfl=0.4):
    """Whole RK3 time steps on the GPU through the C ABI."""
    from oracle import mesh
    dev = "cuda"
    nbx, nby, nbz = nb
    U = torch.tensor(mesh.split(mesh.pad_box(Ug, 3, bc), 8, 3), device=dev)
    n = U.shape[0]
    o = torch.tensor(mesh.origins(nbx, nby, nbz, 8, h, lo), device=dev)
    hh = torch.full((n,), h, dtype=torch.float64, device=dev)
    U0 = torch.empty_like(U)
    dU = torch.empty((n, 10, 8, 8, 8), dtype=torch.float64, device=dev)
    am = torch.empty(n, dtype=torch.float64, device=dev)
    dt = torch.empty(1, dtype=torch.float64, device=dev)
    B = H.make_batch(U, o, hh)
    code = {"periodic": H.HYDRO_BC_PERIODIC, "outflow": H.HYDRO_BC_OUTFLOW}[bc]
    t = 0.0
    nstep = 0
    while (t_end is None and nstep < steps) or (t_end is not None and t < t_end * (1 - 1e-12)):
        U0.copy_(U)
        for k in range(3):
            H.hydro_fill_ghosts_uniform(ctx, B, nbx, nby, nbz, code)
            H.hydro_step(ctx, B, 0.0, dU, am)
            if k == 0:
                H.hydro_dt(ctx, am, hh, n, cfl, dt)
                if t_end is not None:
                    dtv = min(dt.item(), t_end - t)
                    dt.fill_(dtv)
            H.hydro_update(ctx, B, U0, dU, dt_dev=dt, stage=k)
        t += dt.item()
        nstep += 1
    torch.cuda.synchronize()
    return mesh.join(U.cpu().numpy()[:, :, 3:-3, 3:-3, 3:-3], nbx, nby, nbz), t, nstep


def test_full_rk3_step_config1(H, orc):
    """One full RK3 step of the single-sub-grid Sedov blast (config 1)."""
    from oracle import mesh
    Ug, h, lo = W.sedov_box(8, GAMMA)
    ctx = H.Context(GAMMA, 0.0)
    got, t, _ = run_rk3_gpu(H, ctx, Ug, h, lo, "periodic", (1, 1, 1), steps=1)
    P = orc.OracleParams(gamma=GAMMA)
    _, fl = box_states(Ug, "periodic", (P, h, lo))
    run = mesh.BoxRun(P, Ug, h, lo, "periodic")
    run.step(0.4)
    assert t == run.t
    assert rel_err(box_states(got, "periodic"), box_states(run.U, "periodic"), h, fl) <= TOL


def test_rk3_steps_uniform_mesh_outflow(H, orc):
    """Five RK3 steps of a 2x2x2-sub-grid Sedov blast with outflow boundaries."""
    from oracle import mesh
    Ug, h, lo = W.sedov_box(16, GAMMA)
    ctx = H.Context(GAMMA, 0.0)
    got, t, _ = run_rk3_gpu(H, ctx, Ug, h, lo, "outflow", (2, 2, 2), steps=5)
    P = orc.OracleParams(gamma=GAMMA)
    _, fl = box_states(Ug, "outflow", (P, h, lo))
    run = mesh.BoxRun(P, Ug, h, lo, "outflow")
    for _ in range(5):
        run.step(0.4)
    assert t == pytest.approx(run.t, rel=1e-13)
    # five steps of accumulated rounding
    assert rel_err(box_states(got, "outflow"), box_states(run.U, "outflow"), h, fl) <= 1e-11


def test_sedov_64_shock_radius(H):
    """Config 2: 512 sub-grids (64^3 on [-1,1]^3), outflow, to t = 0.05:
    the shell sits at the similarity radius within 1.5 cells; mass conserved."""
    from oracle import analytic
    Ug, h, lo = W.sedov_box(64, GAMMA)
    ctx = H.Context(GAMMA, 0.0)
    got, t, nstep = run_rk3_gpu(H, ctx, Ug, h, lo, "outflow", (8, 8, 8), t_end=0.05)
    assert H.hydro_status(ctx) == 0
    R = analytic.sedov_radius(1.0, 1.0, t, GAMMA)
    X, Y, Z = W.cell_centres(Ug.shape[1:], lo, h)
    r = np.sqrt(X * X + Y * Y + Z * Z)
    bins = np.arange(0.0, 0.9, h / 2)
    idx = np.digitize(r.ravel(), bins)
    rho = got[0]
    prof = np.array([rho.ravel()[idx == i].mean() if np.any(idx == i) else 0 for i in range(1, len(bins))])
    r_peak = 0.5 * (bins[np.argmax(prof)] + bins[np.argmax(prof) + 1])
    assert abs(r_peak - R) < 1.5 * h, (r_peak, R)
    assert rho.sum() == pytest.approx(64.0 ** 3, rel=1e-12)
    for ax in range(3):
        assert np.max(np.abs(rho - np.flip(rho, axis=ax))) < 1e-10 * rho.max()


def test_bench_size_sampled_parity(H, orc):
    """The benchmark's launch (512 sub-grids of a blast that has run a few
    steps) against the oracle on a sample of sub-grids."""
    Ug, h, lo = W.sedov_box(64, GAMMA)
    ctx = H.Context(GAMMA, 0.0)
    got, t, _ = run_rk3_gpu(H, ctx, Ug, h, lo, "outflow", (8, 8, 8), steps=8)
    from oracle import mesh
    sub = mesh.split(mesh.pad_box(got, 3, "outflow"), 8, 3)
    o = mesh.origins(8, 8, 8, 8, h, lo)
    dU, am = gpu_step(H, ctx, sub, o, h)
    pick = np.array([0, 7, 63, 219, 292, 300, 365, 511])
    dUo, amo, _ = orc.step(orc.OracleParams(gamma=GAMMA), sub[pick], o[pick], h)
    assert rel_err(dU[pick], dUo, h, rate_floor(sub[pick], amo, h)) <= TOL
    assert np.allclose(am[pick], amo, rtol=1e-14, atol=0)


def test_empty_batch_is_noop(H):
    ctx = H.Context(GAMMA, 0.0)
    B = H.Batch(0, None, None, None, None)
    H.hydro_step(ctx, B, 0.0, None, None)
    H.hydro_update(ctx, B, None, None, dt=0.1, stage=0)


def test_misaligned_and_invalid_arguments(H):
    ctx = H.Context(GAMMA, 0.0)
    U = torch.zeros(2 * 10 * 14 ** 3 + 1, dtype=torch.float64, device="cuda")
    o = torch.zeros((2, 3), dtype=torch.float64, device="cuda")
    hh = torch.ones(2, dtype=torch.float64, device="cuda")
    dU = torch.zeros((2, 10, 8, 8, 8), dtype=torch.float64, device="cuda")
    am = torch.zeros(2, dtype=torch.float64, device="cuda")
    B = H.Batch(2, U.data_ptr() + 8, o.data_ptr(), hh.data_ptr(), None)  # 8-byte offset: not 16-aligned
    with pytest.raises(H.HydroError) as e:
        H.hydro_step(ctx, B, 0.0, dU, am)
    assert e.value.code == H.HYDRO_EINVAL
    B = H.Batch(2, U.data_ptr(), o.data_ptr(), hh.data_ptr(), None)
    with pytest.raises(H.HydroError):
        H.hydro_step(ctx, B, -1.0, dU, am)
    with pytest.raises(H.HydroError):
        H.hydro_update(ctx, B, U, dU, dt=0.1, stage=3)
    with pytest.raises(H.HydroError):
        H.hydro_fill_ghosts_uniform(ctx, B, 2, 2, 2, H.HYDRO_BC_PERIODIC)  # 8 != 2 sub-grids


def test_nonphysical_state_sets_status(H):
    U = W.random_subgrids(3, 1, GAMMA)
    U[1, 0, 5, 5, 5] = -1.0  # negative density in one cell
    ctx = H.Context(GAMMA, 0.0)
    gpu_step(H, ctx, U, np.zeros(3), 0.1)
    assert H.hydro_status(ctx) & H.HYDRO_ST_NONPHYS
    assert H.hydro_status(ctx) == 0  # cleared by the read


@pytest.mark.parametrize("mixed", [False, True])
def test_rk3_graph_replay_equals_direct_launches(H, mixed):
    """The captured RK3 step (ping-pong buffers, out-of-place first stage)
    replayed 4 times equals the direct launch sequence and the in-place path
    with an explicit copy of the initial state, bitwise."""
    from oracle import mesh
    Ug, h, lo = W.sedov_box(16, GAMMA)
    dev = "cuda"
    nb = (2, 2, 2)
    init = torch.tensor(mesh.split(mesh.pad_box(Ug, 3, "outflow"), 8, 3), device=dev)
    n = init.shape[0]
    o = torch.tensor(mesh.origins(2, 2, 2, 8, h, lo), device=dev)
    hh = torch.full((n,), h, dtype=torch.float64, device=dev)

    def fresh():
        ctx = H.Context(GAMMA, 0.0)
        if mixed:
            H.hydro_set_mode(ctx, H.HYDRO_PREC_MIXED)
        return ctx

    def buffers():
        return (init.clone(), torch.zeros_like(init), torch.empty((n, 10, 8, 8, 8), dtype=torch.float64, device=dev),
                torch.empty(n, dtype=torch.float64, device=dev), torch.empty(1, dtype=torch.float64, device=dev))

    # graph replays
    ctx = fresh()
    Ua, Ub, dU, am, dt = buffers()
    d = H.make_rk3_desc(Ua, Ub, o, hh, nb, H.HYDRO_BC_OUTFLOW, dU, am, dt)
    g = H.hydro_rk3_graph_create(ctx, d)
    for _ in range(4):
        H.hydro_rk3_graph_launch(g)
    torch.cuda.synchronize()
    assert H.hydro_rk3_graph_state(g) == 0
    H.hydro_rk3_graph_destroy(g)
    graph_state = Ua[:, :, 3:-3, 3:-3, 3:-3].cpu().numpy()
    # direct launches
    ctx = fresh()
    Ua2, Ub2, dU2, am2, dt2 = buffers()
    d2 = H.make_rk3_desc(Ua2, Ub2, o, hh, nb, H.HYDRO_BC_OUTFLOW, dU2, am2, dt2)
    for k in range(4):
        H.hydro_rk3_step(ctx, d2, k % 2)
    torch.cuda.synchronize()
    assert np.array_equal(Ua2[:, :, 3:-3, 3:-3, 3:-3].cpu().numpy(), graph_state)
    # in place with a copy of the initial state
    ctx = fresh()
    got, t, _ = run_rk3_gpu(H, ctx, Ug, h, lo, "outflow", nb, steps=4)
    assert np.array_equal(got, mesh.join(graph_state, 2, 2, 2))


def test_interior_scatter_gather(H):
    """Compact interiors <-> padded state: bitwise copies of the interior
    cells, ghost cells untouched, and argument checks."""
    dev = "cuda"
    rng = np.random.default_rng(17)
    n = 37
    U = torch.tensor(rng.normal(size=(n, 10, 14, 14, 14)), device=dev)
    before = U.clone()
    I = torch.tensor(rng.normal(size=(n, 10, 8, 8, 8)), device=dev)
    o = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    hh = torch.full((n,), 0.1, dtype=torch.float64, device=dev)
    ctx = H.Context(GAMMA, 0.0)
    B = H.make_batch(U, o, hh)
    H.hydro_scatter_interior(ctx, B, I)
    torch.cuda.synchronize()
    assert torch.equal(U[:, :, 3:11, 3:11, 3:11], I)
    ghost = torch.ones_like(U, dtype=torch.bool)
    ghost[:, :, 3:11, 3:11, 3:11] = False
    assert torch.equal(U[ghost], before[ghost])
    out = torch.full_like(I, float("nan"))
    H.hydro_gather_interior(ctx, B, out)
    torch.cuda.synchronize()
    assert torch.equal(out, I)
    flat = torch.empty(I.numel() + 1, dtype=torch.float64, device=dev)
    with pytest.raises(RuntimeError):
        H.hydro_gather_interior(ctx, B, flat[1:])  # 8-byte offset: not 16-byte aligned
    # page-locked host memory: the kernels read and write it over the host link
    hI = torch.tensor(rng.normal(size=(n, 10, 8, 8, 8))).pin_memory()
    H.hydro_scatter_interior(ctx, B, hI)
    hout = torch.full(hI.shape, float("nan"), dtype=torch.float64).pin_memory()
    H.hydro_gather_interior(ctx, B, hout)
    torch.cuda.synchronize()
    assert torch.equal(hout, hI) and torch.equal(U[:, :, 3:11, 3:11, 3:11].cpu(), hI)
    # pageable host memory is refused before any launch
    page = np.zeros(I.numel())
    with pytest.raises(RuntimeError):
        H.hydro_gather_interior(ctx, B, page.ctypes.data)
