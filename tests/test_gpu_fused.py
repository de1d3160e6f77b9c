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
