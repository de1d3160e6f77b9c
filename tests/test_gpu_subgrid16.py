"""16^3 sub-grids on the GPU (the compile-time sub-grid size of Sec. III-B,
the paper's best-performing configuration in Sec. V), through the C ABI.

The step kernels run the eight 8^3 octants of each 16^3 sub-grid as tiles,
each read in place from its 14^3 window of the 22^3 padded array; the mesh
kernels (ghost fill, update, interior copies, sums, adaptive-mesh ghost fill
and flux correction) are templated on the sub-grid size.  Held to:
  * the step: the 16^3 cut of a box equals its 8^3 cut on the GPU bit for
    bit without rotation and gravity (both precisions, both mixed
    decompositions, boundary-face sums included), as the oracle's 16^3 cut
    equals its 8^3 cut (test_oracle_subgrid16.py); with rotation and gravity
    the FP64 form within 1e-12 of the oracle's 16^3 cut and the mixed form
    within its budget;
  * the uniform ghost fill bitwise against the oracle's padding, and the
    interior copies and sums;
  * three RK3 steps of a 16^3-cut Sedov box: FP64 within 1e-12 of the
    oracle's 16^3 run, and the GPU's 16^3 and 8^3 runs bit for bit;
  * an adaptive mesh of 16^3 leaves: the two-pass ghost fill bitwise against
    the oracle's octree, a whole RK3 step within 1e-12 of it, and the GPU's
    16^3 and 8^3-cut runs bit for bit;
  * the fused RK3 step (each octant tile a work unit): bit for bit equal to
    the separate 16^3 launches (row and plane sweeps, with and without
    contact steepening; a ragged box with a blast, periodic and outflow; the
    rotating polytrope with gravity), and without rotation to the fused step
    on the same box cut into 8^3;
  * the allocation-free entry point rejects 16^3 (EUNSUP).
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
    t = torch.as_tensor(t)
    return t.contiguous().view(torch.int64)


def cut(Ug, N, bc, h, lo):
    """Padded sub-grids of a box cut into N^3 (ghosts filled by the oracle's
    padding), and their origins."""
    from oracle import mesh
    sub = mesh.split(mesh.pad_box(Ug, 3, bc), N, 3)
    nb = Ug.shape[1] // N
    return sub, mesh.origins(nb, nb, nb, N, h, lo)


def gpu_step(H, N, prec, U, o, h, omega=0.0, g=None, decomp=None):
    ctx = H.Context(GAMMA, omega, N=N)
    H.hydro_set_mode(ctx, prec)
    if decomp is not None:
        H.hydro_set_launch(ctx, decomp)
    n = U.shape[0]
    Ut = torch.tensor(U, device="cuda")
    ot = torch.tensor(o, device="cuda")
    ht = torch.full((n,), h, dtype=torch.float64, device="cuda")
    gt = torch.tensor(g, device="cuda") if g is not None else None
    dU = torch.full((n, 10, N, N, N), float("nan"), dtype=torch.float64, device="cuda")
    am = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    ff = torch.full((n, 6, 13, N, N), float("nan"), dtype=torch.float64, device="cuda")
    H.hydro_step(ctx, H.make_batch(Ut, ot, ht, gt), 0.0, dU, am, ff)
    torch.cuda.synchronize()
    assert H.hydro_status(ctx) == 0
    return dU.cpu().numpy(), am.cpu().numpy(), ff.cpu().numpy()


def _faces16_from_8(f8, nb16):
    """The 16^3 sub-grids' boundary-face sums assembled from the 8^3 cut's:
    [n16][6][13][16][16] from [n8][6][13][8][8] (sub-grid order of both cuts
    as mesh.split)."""
    nb8 = 2 * nb16
    out = np.zeros((nb16 ** 3, 6, 13, 16, 16))
    for kz in range(nb16):
        for ky in range(nb16):
            for kx in range(nb16):
                s16 = (kz * nb16 + ky) * nb16 + kx
                for oz in (0, 1):
                    for oy in (0, 1):
                        for ox in (0, 1):
                            s8 = ((2 * kz + oz) * nb8 + 2 * ky + oy) * nb8 + 2 * kx + ox
                            o = (ox, oy, oz)
                            for f in range(6):
                                a = f // 2
                                if o[a] != f % 2:  # an inner face of the 16^3 sub-grid
                                    continue
                                b, c = (1, 2) if a == 0 else ((0, 2) if a == 1 else (0, 1))
                                out[s16, f, :, 8 * o[c]:8 * o[c] + 8, 8 * o[b]:8 * o[b] + 8] = f8[s8, f]
    return out


@pytest.mark.parametrize("prec,decomp", [("fp64", None), ("mixed", "rows"), ("mixed", "planes")])
@pytest.mark.parametrize("bc", ["periodic", "outflow"])
def test_sixteen_equals_eight_on_the_gpu(H, prec, decomp, bc):
    from oracle import mesh
    from test_oracle_subgrid16 import _box
    Ug = _box(32, 3)
    h, lo = 1.0 / 32, (-0.5, -0.5, -0.5)
    p = {"fp64": H.HYDRO_PREC_FP64, "mixed": H.HYDRO_PREC_MIXED}[prec]
    dec = {None: None, "rows": H.HYDRO_DECOMP_ROWS, "planes": H.HYDRO_DECOMP_PLANES}[decomp]
    U8, o8 = cut(Ug, 8, bc, h, lo)
    U16, o16 = cut(Ug, 16, bc, h, lo)
    d8, a8, f8 = gpu_step(H, 8, p, U8, o8, h, decomp=dec)
    d16, a16, f16 = gpu_step(H, 16, p, U16, o16, h, decomp=dec)
    j8, j16 = mesh.join(d8, 4, 4, 4), mesh.join(d16, 2, 2, 2)
    assert np.array_equal(j8.view(np.int64), j16.view(np.int64))
    # amax: the largest over each 16^3 sub-grid's octants
    want = a8.reshape(2, 2, 2, 2, 2, 2).transpose(0, 2, 4, 1, 3, 5).reshape(8, 8).max(axis=1)
    assert np.array_equal(a16, want)
    assert np.array_equal(f16.view(np.int64), _faces16_from_8(f8, 2).view(np.int64))


def test_sixteen_with_rotation_and_gravity_against_oracle(H, oracle_mod):
    from oracle import core, mesh
    from oracle.compare import max_rel_error, mixed_worst, rate_floor
    from test_oracle_subgrid16 import _box
    Ug = _box(32, 5)
    rng = np.random.default_rng(7)
    gbox = rng.uniform(-1.0, 1.0, (3, 32, 32, 32))
    h, lo, omega = 1.0 / 32, (-0.37, -0.61, -0.5), 0.4
    U16, o16 = cut(Ug, 16, "outflow", h, lo)
    g16 = np.ascontiguousarray(mesh.unjoin(gbox, 16))
    P = core.OracleParams(gamma=GAMMA, omega=omega, N=16)
    ref, amo, _, faces = core.step(P, U16, o16, h, g16, faces=True)
    d64, a64, _ = gpu_step(H, 16, H.HYDRO_PREC_FP64, U16, o16, h, omega, g16)
    assert max_rel_error(d64, ref, h, rate_floor(U16, amo, h, omega, g16)) <= 1e-12
    assert np.allclose(a64, amo, rtol=1e-14, atol=0)
    pert, _, _ = core.step(P, U16.astype(np.float32).astype(np.float64), o16, h, g16)
    for dec in (H.HYDRO_DECOMP_ROWS, H.HYDRO_DECOMP_PLANES):
        dmx, amx, _ = gpu_step(H, 16, H.HYDRO_PREC_MIXED, U16, o16, h, omega, g16, decomp=dec)
        worst = mixed_worst(dmx, ref, pert, faces, h, U16, amo)
        print("16^3 mixed step, decomposition", dec, ": largest err/budget", worst)
        assert worst <= 1.0
        assert np.allclose(amx, amo, rtol=1e-6, atol=0)


@pytest.mark.parametrize("bc", ["periodic", "outflow"])
def test_sixteen_ghost_fill_and_interior_copies(H, bc):
    from oracle import mesh
    rng = np.random.default_rng(3)
    Ug = rng.uniform(0.5, 1.5, (10, 32, 16, 48))  # 3 x 1 x 2 sub-grids of 16^3
    want = mesh.split(mesh.pad_box(Ug, 3, bc), 16, 3)
    start = want.copy()
    inner = np.zeros((22, 22, 22), bool)
    inner[3:-3, 3:-3, 3:-3] = True
    start[:, :, ~inner] = -7.0
    U = torch.tensor(start, device="cuda")
    n = U.shape[0]
    o = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    hh = torch.full((n,), 0.1, dtype=torch.float64, device="cuda")
    B = H.make_batch(U, o, hh)
    ctx = H.Context(GAMMA, 0.0, N=16)
    H.hydro_fill_ghosts_uniform(ctx, B, 3, 1, 2, {"periodic": H.HYDRO_BC_PERIODIC, "outflow": H.HYDRO_BC_OUTFLOW}[bc])
    torch.cuda.synchronize()
    assert np.array_equal(U.cpu().numpy(), want)
    # interiors out and back in
    I = torch.empty((n, 10, 16, 16, 16), dtype=torch.float64, device="cuda")
    H.hydro_gather_interior(ctx, B, I)
    torch.cuda.synchronize()
    assert np.array_equal(I.cpu().numpy(), want[:, :, 3:-3, 3:-3, 3:-3])
    U2 = torch.zeros_like(U)
    H.hydro_scatter_interior(ctx, H.make_batch(U2, o, hh), I)
    torch.cuda.synchronize()
    assert np.array_equal(U2.cpu().numpy()[:, :, 3:-3, 3:-3, 3:-3], want[:, :, 3:-3, 3:-3, 3:-3])
    # conserved sums: the interior sums times h^3 (fixed-order reduction)
    sums = torch.empty(11, dtype=torch.float64, device="cuda")
    H.hydro_conserved_sums(ctx, B, sums)
    torch.cuda.synchronize()
    tot = want[:, :, 3:-3, 3:-3, 3:-3].sum(axis=(0, 2, 3, 4)) * 0.1 ** 3
    assert np.allclose(sums.cpu().numpy()[:10], tot, rtol=1e-13, atol=0)


def test_sixteen_rk3_steps(H, oracle_mod):
    """Three RK3 steps of a Sedov box of 2^3 sub-grids of 16^3 (outflow):
    FP64 within 1e-12 of the oracle's 16^3 run; the GPU's 16^3 and 8^3 runs
    give the same bits in both precisions (no rotation)."""
    from oracle import core, mesh
    from oracle.compare import max_rel_error, state_floor
    from paper_2107_10987_gb300.uniform import UniformRun
    Ug, h, lo = W.sedov_box(32, GAMMA)
    out = {}
    for prec in (H.HYDRO_PREC_FP64, H.HYDRO_PREC_MIXED):
        for N in (8, 16):
            ctx = H.Context(GAMMA, 0.0, N=N)
            H.hydro_set_mode(ctx, prec)
            nb = 32 // N
            o = mesh.origins(nb, nb, nb, N, h, lo)
            run = UniformRun(ctx, np.ascontiguousarray(mesh.unjoin(Ug, N)), o, h, nb, H.HYDRO_BC_OUTFLOW)
            for _ in range(3):
                run.step()
            torch.cuda.synchronize()
            assert H.hydro_status(ctx) == 0
            out[prec, N] = mesh.join(run.interior().cpu().numpy(), nb, nb, nb)
            run.close()
        assert np.array_equal(out[prec, 8].view(np.int64), out[prec, 16].view(np.int64)), prec
    P = core.OracleParams(gamma=GAMMA, N=16)
    ref = mesh.BoxRun(P, Ug, h, lo, "outflow")
    _, am0 = ref.rhs(ref.U)
    U0 = ref._sub(ref.U)
    for _ in range(3):
        ref.step(0.4)
    got = mesh.unjoin(out[H.HYDRO_PREC_FP64, 16], 16)
    assert max_rel_error(got, mesh.unjoin(ref.U, 16), h, state_floor(U0, am0)) <= 1e-12


def test_sixteen_adaptive_mesh(H, oracle_mod):
    """An adaptive mesh of 16^3 leaves (seven at level 1, one octant refined
    into eight at level 2): the two-pass ghost fill bitwise against the
    oracle's octree, one RK3 step within 1e-12 of the oracle's, and the same
    bits as its 8^3 cut run on the GPU."""
    from oracle import amr, core
    from oracle.compare import max_rel_error, state_floor
    from paper_2107_10987_gb300.amr import AMRMesh, AMRRun
    from test_oracle_subgrid16 import _leaf_state, _octree_cut
    lev16 = [1] * 7 + [2] * 8
    ijk16 = [c for c in np.ndindex(2, 2, 2) if c != (0, 0, 0)] + list(np.ndindex(2, 2, 2))
    ijk16 = [(c[2], c[1], c[0]) for c in ijk16]
    t16 = amr.Octree(lev16, ijk16, N=16)
    U16, o16, h16 = _leaf_state(lev16, ijk16, 16)
    # ghost fill
    ctx = H.Context(GAMMA, 0.0, N=16)
    Ut = torch.tensor(U16, device="cuda")
    B = H.make_batch(Ut, torch.tensor(o16, device="cuda"), torch.tensor(h16, device="cuda"))
    m16 = AMRMesh(lev16, ijk16)
    H.hydro_fill_ghosts_amr(ctx, B, m16)
    torch.cuda.synchronize()
    assert H.hydro_status(ctx) == 0
    assert np.array_equal(Ut.cpu().numpy(), amr.fill_ghosts(t16, U16))
    # one RK3 step against the oracle
    P = core.OracleParams(gamma=GAMMA, N=16)
    Uf = amr.fill_ghosts(t16, U16)
    Uo, dto = amr.rk3_step(P, t16, Uf, o16, h16)
    _, am0, _ = core.step(P, Uf, o16, h16)
    run = AMRRun(ctx, U16, lev16, ijk16)
    run.step()
    torch.cuda.synchronize()
    assert H.hydro_status(ctx) == 0
    assert run.dt.item() == pytest.approx(dto, rel=1e-14)
    got = run.U.cpu().numpy()[:, :, 3:-3, 3:-3, 3:-3]
    assert max_rel_error(got, Uo[:, :, 3:-3, 3:-3, 3:-3], h16, state_floor(U16, am0)) <= 1e-12
    # the 8^3 cut on the GPU: the same bits
    lev8, ijk8, src = _octree_cut(lev16, ijk16)
    U8, _, _ = _leaf_state(lev8, ijk8, 8)
    c8 = H.Context(GAMMA, 0.0, N=8)
    run8 = AMRRun(c8, U8, lev8, ijk8)
    run8.step()
    torch.cuda.synchronize()
    assert run8.dt.item() == run.dt.item()
    U8n = run8.U.cpu().numpy()
    U16n = run.U.cpu().numpy()
    for s, (p, (ox, oy, oz)) in enumerate(src):
        a = U8n[s][:, 3:-3, 3:-3, 3:-3]
        b = U16n[p][:, 3 + oz:11 + oz, 3 + oy:11 + oy, 3 + ox:11 + ox]
        assert np.array_equal(a.view(np.int64), b.view(np.int64)), s
    run.close()
    run8.close()


def _blast_box(nx, ny, nz, seed=0, h=0.05):
    """A box of seeded random density, pressure and velocity with a blast in
    one corner (flow crosses periodic boundaries; no sub-grid is uniform)."""
    rng = np.random.default_rng(seed)
    rho = 1.0 + 0.2 * rng.random((nz, ny, nx))
    p = 1e-3 * (1.0 + rng.random((nz, ny, nx)))
    v = 0.1 * rng.normal(size=(3, nz, ny, nx))
    p[:2, :2, :2] += (GAMMA - 1.0) * 1e-3 / (8 * h ** 3)
    return W.conserved_from_primitive(rho, v, p, GAMMA), h


def _run(H, N, Ui, o, h, nb, bc, fused, decomp, contact=0, omega=0.0, g=None, steps=3):
    from paper_2107_10987_gb300.uniform import UniformRun
    ctx = H.Context(GAMMA, omega, N=N)
    H.hydro_set_mode(ctx, H.HYDRO_PREC_MIXED, contact=contact)
    H.hydro_set_launch(ctx, decomp)
    run = UniformRun(ctx, Ui, o, h, nb, bc, g, fused=fused)
    dts = []
    for _ in range(steps):
        run.step()
        dts.append(run.last_dt())
    torch.cuda.synchronize()
    assert H.hydro_status(ctx) == 0
    out = run.interior()
    run.close()
    return out, np.array(dts)


@pytest.mark.parametrize("decomp,contact", [("rows", 0), ("planes", 0), ("rows", 1), ("planes", 1)])
@pytest.mark.parametrize("bc", ["periodic", "outflow"])
def test_sixteen_fused_step(H, decomp, contact, bc):
    """The fused step on a ragged box of 2 x 1 x 3 sub-grids of 16^3 with a
    blast: the interiors and dt after each of three steps equal the separate
    16^3 launches' bit for bit, and the fused step on the box cut into 8^3
    (4 x 2 x 6 sub-grids) bit for bit."""
    from oracle import mesh
    dec = {"rows": H.HYDRO_DECOMP_ROWS, "planes": H.HYDRO_DECOMP_PLANES}[decomp]
    code = {"periodic": H.HYDRO_BC_PERIODIC, "outflow": H.HYDRO_BC_OUTFLOW}[bc]
    Ug, h = _blast_box(32, 16, 48)
    lo = (0.0, 0.0, 0.0)
    res = {}
    for N, nb in ((16, (2, 1, 3)), (8, (4, 2, 6))):
        Ui = mesh.unjoin(Ug, N)
        o = mesh.origins(*nb, N, h, lo)
        for fused in ((True, False) if N == 16 else (True,)):
            got, dts = _run(H, N, Ui, o, h, nb, code, fused, dec, contact)
            res[N, fused] = (mesh.join(got.cpu().numpy(), *nb), dts)
    (a, da), (b, db), (c, dc) = res[16, True], res[16, False], res[8, True]
    assert np.array_equal(da.view(np.int64), db.view(np.int64)) and np.array_equal(da.view(np.int64),
                                                                                    dc.view(np.int64))
    assert np.array_equal(a.view(np.int64), b.view(np.int64)), int((a != b).sum())
    assert np.array_equal(a.view(np.int64), c.view(np.int64)), int((a != c).sum())


@pytest.mark.parametrize("decomp", ["rows", "planes"])
def test_sixteen_fused_polytrope(H, decomp):
    """The fused step on the rotating polytrope (omega = 0.2, gravity) cut
    into 4^3 sub-grids of 16^3: bit for bit equal to the separate launches."""
    dec = {"rows": H.HYDRO_DECOMP_ROWS, "planes": H.HYDRO_DECOMP_PLANES}[decomp]
    Ui, g, o, h, _ = W.rotating_polytrope(4, GAMMA, N=16)
    a, da = _run(H, 16, Ui, o, h, 4, H.HYDRO_BC_OUTFLOW, True, dec, omega=0.2, g=g, steps=2)
    b, db = _run(H, 16, Ui, o, h, 4, H.HYDRO_BC_OUTFLOW, False, dec, omega=0.2, g=g, steps=2)
    assert np.array_equal(da.view(np.int64), db.view(np.int64))
    assert bool((bits(a) == bits(b)).all()), int((bits(a) != bits(b)).sum())


def test_sixteen_rejections(H):
    ctx = H.Context(GAMMA, 0.0, N=16)
    H.hydro_set_mode(ctx, H.HYDRO_PREC_FP64)
    with pytest.raises(H.HydroError) as e:
        H.hydro_step_static(ctx, H.Batch(2, 16, 16, 16, None), 0.0, 16, 16)
    assert e.value.code == H.HYDRO_EUNSUP
    with pytest.raises(H.HydroError) as e:
        H.Context(GAMMA, 0.0, N=12)
    assert e.value.code == H.HYDRO_EINVAL
