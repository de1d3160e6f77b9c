"""The fused RK3 time step of a uniform mesh (one persistent launch per step:
ghost cells read from the neighbours' interiors, stages 1 and 2 updating
inside the launch, a sub-grid's third stage waiting only for its 27
neighbours) against the separate launches (ghost fill, step, update per
stage): interiors and dt equal bit for bit over several steps.  The
separate launches are themselves held to the oracle by the other GPU tests.

Meshes cover every neighbour case: cubic, ragged (3 x 2 x 5), a single
sub-grid (its own neighbour on every side under periodic boundaries), rows
of two and three, under both boundary conditions; the headline Sedov mesh; the
rotating polytrope with gravity; the learned indicator's kernel; graph
replay; the configurations the fused form rejects; and the bounded wait's
expiry."""
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


def blast_mesh(nbx, nby, nbz, seed=0, h=0.05, amp=1.0, blast=True):
    """nbx x nby x nbz sub-grids of 8^3 (origin 0, spacing h): seeded random
    density, pressure and velocity in every cell (relative amplitude amp),
    and a blast in the corner cells, so that flow crosses the periodic
    boundaries and no sub-grid is uniform."""
    nx, ny, nz = 8 * nbx, 8 * nby, 8 * nbz
    rng = np.random.default_rng(seed)
    rho = 1.0 + 0.2 * amp * rng.random((nz, ny, nx))
    p = 1e-3 * (1.0 + amp * rng.random((nz, ny, nx)))
    v = 0.1 * amp * rng.normal(size=(3, nz, ny, nx))
    if blast:
        p[:2, :2, :2] += (GAMMA - 1.0) * 1e-3 / (8 * h ** 3)
    Ug = W.conserved_from_primitive(rho, v, p, GAMMA)
    U = W.box_to_subgrids(np.ascontiguousarray(Ug))
    o = np.empty((nbx * nby * nbz, 3))
    s = 0
    for kz in range(nbz):
        for ky in range(nby):
            for kx in range(nbx):
                o[s] = (8 * kx * h, 8 * ky * h, 8 * kz * h)
                s += 1
    return U, o, h


def bits(t):
    return t.contiguous().view(torch.int64)


def run_pair(H, ctx, U, o, h, nb, bc, steps, g=None, graph=False):
    from paper_2107_10987_gb300.uniform import UniformRun
    sep = UniformRun(ctx, U, o, h, nb, bc, g)
    fus = UniformRun(ctx, U, o, h, nb, bc, g, fused=True)
    for k in range(steps):
        sep.step()
        fus.step(use_graph=graph)
        torch.cuda.synchronize()
        assert np.float64(fus.last_dt()).view(np.int64) == np.float64(sep.last_dt()).view(np.int64), k
        a, b = fus.interior(), sep.interior()
        same = bits(a) == bits(b)
        assert bool(same.all()), (k, int((~same).sum()), float((a - b).abs().max()))
    fus.close()
    sep.close()
    return sep


@pytest.mark.parametrize("nb,bc", [((4, 4, 4), "periodic"), ((3, 2, 5), "periodic"), ((3, 2, 5), "outflow"),
                                   ((1, 1, 1), "periodic"), ((2, 1, 1), "outflow"), ((1, 3, 1), "periodic")])
def test_fused_equals_separate_launches(H, nb, bc):
    code = {"periodic": H.HYDRO_BC_PERIODIC, "outflow": H.HYDRO_BC_OUTFLOW}[bc]
    U, o, h = blast_mesh(*nb)
    ctx = H.Context(GAMMA, 0.0)
    H.hydro_set_mode(ctx, H.HYDRO_PREC_MIXED)
    run_pair(H, ctx, U, o, h, nb, code, steps=3)
    assert H.hydro_status(ctx) == 0


def test_fused_headline_sedov_mesh_and_graph(H):
    """The benchmark's 512-sub-grid Sedov mesh (outflow), direct launches and
    graph replays of the fused step, against the separate launches."""
    Ug, h, lo = W.sedov_box(64, GAMMA)
    U = W.box_to_subgrids(Ug)
    o, h2 = W.uniform_mesh(8)
    assert h2 == pytest.approx(h)
    ctx = H.Context(GAMMA, 0.0)
    H.hydro_set_mode(ctx, H.HYDRO_PREC_MIXED)
    run_pair(H, ctx, U, o, h2, 8, H.HYDRO_BC_OUTFLOW, steps=3)
    run_pair(H, ctx, U, o, h2, 8, H.HYDRO_BC_OUTFLOW, steps=4, graph=True)
    assert H.hydro_status(ctx) == 0


def test_fused_rotating_polytrope_with_gravity(H):
    """Rotating frame (omega = 0.2), static gravity and the thin ambient gas:
    4,096 sub-grids, outflow."""
    U, g, o, h, _ = W.rotating_polytrope(16)
    ctx = H.Context(GAMMA, 0.2)
    H.hydro_set_mode(ctx, H.HYDRO_PREC_MIXED)
    gt = torch.tensor(g, device="cuda")
    run_pair(H, ctx, U, o, h, 16, H.HYDRO_BC_OUTFLOW, steps=2, g=gt)
    assert H.hydro_status(ctx) == 0


def test_fused_with_learned_indicator(H):
    """The indicator's instance of the fused kernel: seeded parameters, on
    mildly perturbed data (no jumps, so the unlimited reconstruction stays
    physical), at the first threshold from a ladder at which the indicator
    changes the separate launches' result; the fused step then makes the
    same decisions and gives the same values."""
    from oracle import gate
    from paper_2107_10987_gb300.uniform import UniformRun
    U, o, h = blast_mesh(4, 4, 4, seed=3, amp=0.05, blast=False)
    rng = np.random.default_rng(5)
    theta = torch.tensor(rng.normal(0, 0.3, gate.NPARAM).astype(np.float32), device="cuda")
    ctx = H.Context(GAMMA, 0.0)
    H.hydro_set_mode(ctx, H.HYDRO_PREC_MIXED)

    def one_step():
        run = UniformRun(ctx, U, o, h, 4, H.HYDRO_BC_PERIODIC)
        run.step()
        return run.interior()

    plain = one_step()
    for thr in (0.5, 0.9, 0.99, 0.999, 0.99999, 0.9999999):
        H.hydro_set_indicator(ctx, theta, thr)
        if not bool((bits(one_step()) == bits(plain)).all()):
            break
    else:
        pytest.fail("no threshold made the indicator act")
    run_pair(H, ctx, U, o, h, 4, H.HYDRO_BC_PERIODIC, steps=2)
    assert H.hydro_status(ctx) == 0


def test_fused_rejects_fp64_and_adaptive_meshes(H):
    from paper_2107_10987_gb300.uniform import UniformRun
    U, o, h = blast_mesh(2, 2, 2)
    ctx = H.Context(GAMMA, 0.0)  # FP64 mode
    run = UniformRun(ctx, U, o, h, 2, H.HYDRO_BC_PERIODIC, fused=True)
    with pytest.raises(H.HydroError):
        run.step()
    d = run.desc
    lib = H._lib()
    # any non-null mesh pointer (rejected before it is read) and face buffer
    d.amr = 1
    d.face_flux = d.dUdt
    H.hydro_set_mode(ctx, H.HYDRO_PREC_MIXED)
    import ctypes as C
    assert lib.hydro_rk3_step(H._cp(ctx), C.byref(d), 0, None) == H.HYDRO_EUNSUP
    torch.cuda.synchronize()
    assert H.hydro_status(ctx) == 0


def test_bounded_wait_reports_timeout(H):
    """The fused step's wait, on a flag that nothing sets: it gives up after
    its limit (10 ms here) and sets HYDRO_ST_TIMEOUT; the context stays
    usable."""
    import time
    ctx = H.Context(GAMMA, 0.0)
    assert H.hydro_status(ctx) == 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    H.hydro_selftest_wait(ctx, 0.01)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    assert H.hydro_status(ctx) == H.HYDRO_ST_TIMEOUT
    assert 0.009 < dt < 1.0, dt
    # the context and the device still work: a fused step afterwards
    H.hydro_set_mode(ctx, H.HYDRO_PREC_MIXED)
    U, o, h = blast_mesh(2, 2, 2)
    run_pair(H, ctx, U, o, h, 2, H.HYDRO_BC_PERIODIC, steps=1)
    assert H.hydro_status(ctx) == 0


def _nbhd_max(x, nb, periodic):
    """Largest value over the 27 neighbours (boundary map applied) of a
    per-sub-grid array x [n][F] on an nbx x nby x nbz mesh."""
    nbx, nby, nbz = nb
    a = x.reshape(nbz, nby, nbx, -1)
    pad = np.pad(a, ((1, 1), (1, 1), (1, 1), (0, 0)), mode="wrap" if periodic else "edge")
    out = np.full_like(a, -np.inf)
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                out = np.maximum(out, pad[dz:dz + nbz, dy:dy + nby, dx:dx + nbx])
    return out.reshape(x.shape)


def _oracle_rk3_with_budget(P, Ug, h, lo, bc, dt, g):
    """The oracle's RK3 step from the box state Ug with the given dt, and per
    stage the absolute mixed-precision rate budget [n][F] of every sub-grid
    (oracle.compare.mixed_budget times the sub-grid's field scales).  Returns
    (interiors [n][F][8][8][8], [budget_0, budget_1, budget_2], stage-0
    inputs and rates)."""
    from oracle import core, mesh
    from oracle.compare import mixed_budget, subgrid_scales
    nbz, nby, nbx = (n // 8 for n in Ug.shape[1:])
    o = mesh.origins(nbx, nby, nbz, 8, h, lo)
    U0s = mesh.split(mesh.pad_box(Ug, 3, bc), 8, 3)
    Us = U0s
    delta = []
    stage0 = None
    for k in range(3):
        if k:
            Us = mesh.split(mesh.pad_box(mesh.join(mesh.interior(Us, 3), nbx, nby, nbz), 3, bc), 8, 3)
        ref, am, _, faces = core.step(P, Us, o, h, g, faces=True)
        pert, _, _ = core.step(P, Us.astype(np.float32).astype(np.float64), o, h, g)
        if k == 0:
            stage0 = (Us, ref, pert, faces, am)
        budget, _ = mixed_budget(ref, pert, faces, h, Us, am)
        delta.append(budget * subgrid_scales(ref, h))
        Us = core.update(P, Us, U0s, ref, dt, k)
    return np.ascontiguousarray(mesh.interior(Us, 3)), delta, stage0


@pytest.mark.parametrize("case", ["sedov512", "polytrope"])
def test_fused_step_against_oracle(H, oracle_mod, case):
    """The headline kernel against the FP64 oracle directly, on all 10
    fields: the benchmark's 512-sub-grid Sedov mesh after 6 steps, and the
    rotating polytrope (omega = 0.2, gravity, ambient density 1e-10) on 512
    sub-grids after 3 steps.  One more fused step, then
      * its first-stage rates (the dUdt it leaves) within the mixed-precision
        budget of every sub-grid (oracle.compare.mixed_budget);
      * the new state within the budget carried through the three stages:
        the oracle's RK3 step is taken with the kernel's dt, so the states
        differ only by the stages' rate errors d_k (each within its budget
        B_k, largest over the 27 neighbours, whose errors reach a sub-grid
        through the next stage's stencil).  With U1 = U0 + dt L(U0),
        U2 = 3/4 U0 + 1/4 (U1 + dt L(U1)), U3 = 1/3 U0 + 2/3 (U2 + dt L(U2))
        and a stage amplifying an input error by at most |1 + dt L'| <= 6
        (KT fluxes at CFL 0.4 over 3 axes x 2 faces, PPM slopes at most
        doubling a difference), the error of U3 is at most
        6 dt B_0 + dt B_1 + 2/3 dt B_2, plus the update's own rounding: a
        few FP64 units of each state (its fused products), and for the
        tracer the mixed form's FP32 power in the resync, a few FP32 units
        (__powf: 2 ulp at this exponent, and the FP32 argument)."""
    from oracle import core, mesh
    from oracle.compare import mixed_worst
    from paper_2107_10987_gb300.uniform import UniformRun
    if case == "sedov512":
        Ug, h, lo = W.sedov_box(64, GAMMA)
        nb, omega, g, warm, periodic = 8, 0.0, None, 6, False
        U = W.box_to_subgrids(Ug)
        o, _ = W.uniform_mesh(8)
    else:
        U, g, o, h, _ = W.rotating_polytrope(8, GAMMA)
        nb, omega, warm, periodic = 8, 0.2, 3, False
        lo = (-1.0, -1.0, -1.0)
    ctx = H.Context(GAMMA, omega)
    H.hydro_set_mode(ctx, H.HYDRO_PREC_MIXED)
    gt = torch.tensor(g, device="cuda") if g is not None else None
    run = UniformRun(ctx, U, o, h, nb, H.HYDRO_BC_OUTFLOW, gt, fused=True)
    for _ in range(warm):
        run.step()
    start = run.interior().cpu().numpy()
    run.step()
    dt = run.last_dt()
    got = run.interior().cpu().numpy()
    dU0 = run.dU.cpu().numpy()
    assert H.hydro_status(ctx) == 0
    run.close()
    P = core.OracleParams(gamma=GAMMA, omega=omega)
    want, delta, (U0s, ref0, pert0, faces0, am0) = _oracle_rk3_with_budget(
        P, mesh.join(start, nb, nb, nb), h, lo, "outflow", dt, g)
    worst0 = mixed_worst(dU0, ref0, pert0, faces0, h, U0s, am0)
    nbs = (nb, nb, nb)
    bound = dt * (6 * _nbhd_max(delta[0], nbs, periodic) + _nbhd_max(delta[1], nbs, periodic)
                  + (2.0 / 3.0) * _nbhd_max(delta[2], nbs, periodic))
    um = np.abs(want).reshape(want.shape[0], 10, -1).max(axis=2)
    bound = bound + 4 * 2.0 ** -53 * um
    bound[:, 5] += 8 * 2.0 ** -24 * um[:, 5]
    err = np.abs(got - want).reshape(got.shape[0], 10, -1).max(axis=2)
    worst = float(np.max(np.where(bound > 0, err / np.where(bound > 0, bound, 1.0), np.where(err > 0, np.inf, 0.0))))
    print(f"fused step vs oracle ({case}): stage-0 rates largest err/budget {worst0:.3g}, "
          f"state largest err/bound {worst:.3g}, dt {dt:.6e}")
    # the kernel's dt from its FP32 signal speeds, against the oracle's
    assert dt == pytest.approx(0.4 * np.min(h / am0), rel=1e-6)
    assert worst0 <= 1.0
    assert worst <= 1.0
