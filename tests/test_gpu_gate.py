"""The learned smoothness indicator on the GPU, against the CPU oracle.

* training data: GPU features (FP32) against the oracle's FP64 definition,
  GPU labels (FP32 reconstruction) against the oracle's limiter flags;
* gradients: the GPU loss and gradient against a hand-written FP64
  backpropagation on the same BF16-rounded parameters (tolerance: FP32
  accumulation over the batch, 1e-4 of the largest gradient entry);
* gated step: with seeded parameters, the fused indicator (tensor cores,
  BF16 operands, FP32 accumulation) and the gated step against the oracle's
  masked step (its own decisions with the same BF16 rounding);
* gain: a short training on seeded runs, evaluated on held-out seeds, and the
  gated mixed step against the ungated one at equal L1 error.
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


def _batch(H, U, dev="cuda"):
    n = U.shape[0]
    Ut = torch.tensor(U, device=dev)
    return Ut, H.make_batch(Ut, torch.zeros((n, 3), dtype=torch.float64, device=dev),
                            torch.full((n,), 0.05, dtype=torch.float64, device=dev))


def _evolved_sedov(H, steps=6):
    from test_gpu_parity import run_rk3_gpu
    from oracle import mesh
    Ug, h, lo = W.sedov_box(32, GAMMA)
    got, _, _ = run_rk3_gpu(H, H.Context(GAMMA, 0.0), Ug, h, lo, "outflow", (4, 4, 4), steps=steps)
    return mesh.split(mesh.pad_box(got, 3, "outflow"), 8, 3)


def test_gate_data_matches_oracle(H, oracle_mod):
    from oracle import gate
    U = np.concatenate([W.random_subgrids(6, 4, GAMMA, smooth=True), _evolved_sedov(H)[20:28]])
    Ut, B = _batch(H, U)
    n = U.shape[0]
    X = torch.empty((n * 512, 54), dtype=torch.float32, device="cuda")
    y = torch.empty(n * 512, dtype=torch.uint8, device="cuda")
    ctx = H.Context(GAMMA, 0.0)
    H.hydro_gate_data(ctx, B, X, y)
    torch.cuda.synchronize()
    # the FP32 reconstruction cannot see differences below FP32 resolution:
    # compare with the oracle on the inputs rounded to FP32
    U32 = U.astype(np.float32).astype(np.float64)
    Xo = gate.features(U32, GAMMA)
    yo = gate.labels(U32, GAMMA)
    assert np.max(np.abs(X.cpu().numpy() - Xo)) < 2e-6
    agree = (y.cpu().numpy() == yo).mean()
    assert agree >= 0.998, agree
    assert 0.05 < yo.mean() < 0.95  # both classes present


def test_mlp_gradient_matches_cpu_backprop(H, oracle_mod):
    from oracle import gate
    rng = np.random.default_rng(5)
    n = 1000
    theta = rng.normal(0, 0.25, gate.NPARAM).astype(np.float32)
    X = rng.uniform(-1, 1, (n, 54)).astype(np.float32)
    y = (rng.uniform(size=n) < 0.3).astype(np.float32)
    dev = "cuda"
    p, Xt, yt = (torch.tensor(a, device=dev) for a in (theta, X, y))
    grad = torch.empty_like(p)
    loss = torch.empty(1, dtype=torch.float32, device=dev)
    H.hydro_mlp_loss_grad(p, Xt, yt, grad, loss, w1=4.0, w0=0.5)
    out = torch.empty(n, dtype=torch.float32, device=dev)
    H.hydro_mlp_forward(p, Xt, out)
    torch.cuda.synchronize()
    th = gate.bf16_round(theta)
    Lo, go = gate.loss_and_grad(th, X.astype(np.float64), y.astype(np.float64), 4.0, 0.5)
    # the standalone forward is the deployed form: BF16 inputs and first hidden layer
    oo = gate.forward_infer(th, X.astype(np.float64))
    assert loss.item() == pytest.approx(Lo, rel=1e-5)
    assert np.max(np.abs(grad.cpu().numpy() - go)) <= 1e-4 * np.max(np.abs(go))
    assert np.max(np.abs(out.cpu().numpy() - oo)) < 1e-5
    # and the step of the optimiser moves every parameter against its gradient
    m, v = torch.zeros_like(p), torch.zeros_like(p)
    p0 = p.clone()
    H.hydro_mlp_adam(p, m, v, grad, 1, 1e-3)
    torch.cuda.synchronize()
    moved = (p - p0).cpu().numpy()
    gg = grad.cpu().numpy()
    nz = np.abs(gg) > 1e-6
    assert np.all(np.sign(moved[nz]) == -np.sign(gg[nz]))


@pytest.mark.parametrize("fp64", [False, True])
def test_gated_step_matches_masked_oracle(H, oracle_mod, fp64):
    """Seeded parameters; a threshold placed in a gap of the oracle's outputs
    so that the kernel's and the oracle's decisions cannot differ; the gated
    step then matches the oracle's masked step: the FP64 form to 1e-12, the
    mixed form within the mixed-precision budget."""
    from oracle import core, gate
    from oracle.compare import max_rel_error, mixed_worst, rate_floor
    # smooth data only: seeded random parameters also gate cells at jumps,
    # where the unlimited formula may leave density or energy negative
    U = W.random_subgrids(10, 8, GAMMA, smooth=True)
    n = U.shape[0]
    rng = np.random.default_rng(21)
    theta = rng.normal(0, 0.3, gate.NPARAM).astype(np.float32)
    th = gate.bf16_round(theta)
    # predictions on the 12^3 block [-2, N+1]^3, then the dilated decision on
    # the 10^3 reconstructed cells: smooth iff the whole 3x3x3 block is
    Xo = gate.features(U, GAMMA, lo=-2, hi=10)
    out = gate.forward_infer(th, Xo)  # the step kernel evaluates it on the tensor cores
    srt = np.sort(out)
    gaps = np.diff(srt)
    lo_i, hi_i = len(srt) // 10, 9 * len(srt) // 10
    mid = lo_i + np.argmax(gaps[lo_i:hi_i])  # the widest gap with >= 10% of cells on each side
    thr = 0.5 * (srt[mid] + srt[mid + 1])
    assert gaps[mid] > 5e-5, gaps[mid]
    pred = (out < thr).reshape(n, 12, 12, 12)
    dil = np.ones((n, 10, 10, 10), bool)
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                dil &= pred[:, dz:dz + 10, dy:dy + 10, dx:dx + 10]
    mask = np.zeros((n, 14, 14, 14), np.uint8)
    mask[:, 2:12, 2:12, 2:12] = dil
    P = core.OracleParams(gamma=GAMMA)
    origin = np.zeros((n, 3))
    ref, amo = core.step_masked(P, U, origin, 0.05, mask)
    pert, _ = core.step_masked(P, U.astype(np.float32).astype(np.float64), origin, 0.05, mask)
    ctx = H.Context(GAMMA, 0.0)
    H.hydro_set_mode(ctx, H.HYDRO_PREC_FP64 if fp64 else H.HYDRO_PREC_MIXED)
    H.hydro_set_indicator(ctx, torch.tensor(theta, device="cuda"), float(thr))
    Ut, B = _batch(H, U)
    dU = torch.full((n, 10, 8, 8, 8), np.nan, dtype=torch.float64, device="cuda")
    am = torch.empty(n, dtype=torch.float64, device="cuda")
    H.hydro_step(ctx, B, 0.0, dU, am)
    torch.cuda.synchronize()
    got = dU.cpu().numpy()
    assert 0.02 < mask.sum() / (n * 1000) < 0.98
    if fp64:
        assert max_rel_error(got, ref, 0.05, rate_floor(U, amo, 0.05)) <= 1e-12
        assert np.allclose(am.cpu().numpy(), amo, rtol=1e-14, atol=0)
        return
    # the masked oracle exports no face sums: the budget's flux terms come
    # from the states and signal speeds alone
    worst = mixed_worst(got, ref, pert, None, 0.05, U, amo)
    print("gated mixed step: largest err/budget", worst)
    assert worst <= 1.0
    # the indicator off again: the plain mixed step
    H.hydro_set_indicator(ctx, None)
    H.hydro_step(ctx, B, 0.0, dU, am)
    torch.cuda.synchronize()
    plain, amp, _, faces = core.step(P, U, origin, 0.05, faces=True)
    plain_p, _, _ = core.step(P, U.astype(np.float32).astype(np.float64), origin, 0.05)
    worst = mixed_worst(dU.cpu().numpy(), plain, plain_p, faces, 0.05, U, amp)
    print("plain mixed step after the indicator: largest err/budget", worst)
    assert worst <= 1.0


def test_training_gain_on_held_out_runs(H):
    """Train on seeded runs (Sedov at random energy and centre, Sod planes at
    random orientation), evaluate on held-out seeds: limiter-active cells are
    recalled, a large share of cells skips the limiter, and the gated run of
    the Sedov benchmark problem keeps the plain method's L1 density error."""
    from paper_2107_10987_gb300 import gate as GT
    X, y, ch = GT.collect(range(0, 8), n=32, snapshots=(6, 16, 30))
    params, hist = GT.train(X, y, iters=600, batch=16384, lr=3e-3)
    assert hist[-1][1] < 0.5 * hist[0][1], hist
    thr = GT.choose_threshold(params, X, y, ch, recall=0.9995)
    Xh, yh, chh = GT.collect(range(1000, 1004), n=32, snapshots=(6, 16, 30))
    ev = GT.evaluate(params, thr, Xh, yh, chh)
    print("indicator on held-out runs:", ev)
    assert ev["recall"] >= 0.98, ev
    assert ev["frac_smooth"] >= 0.25, ev
    # Sedov to t = 0.05 on 64^3: gated vs plain mixed, equal L1 error
    from test_gpu_mixed import sedov_l1
    from test_gpu_parity import run_rk3_gpu
    Ug, h, lo = W.sedov_box(64, GAMMA)
    res = {}
    for gated in (False, True):
        ctx = H.Context(GAMMA, 0.0)
        H.hydro_set_mode(ctx, H.HYDRO_PREC_MIXED)
        if gated:
            H.hydro_set_indicator(ctx, params, thr)
        u, t, _ = run_rk3_gpu(H, ctx, Ug, h, lo, "outflow", (8, 8, 8), t_end=0.05)
        res[gated] = sedov_l1(u[0], h, lo, t)
    assert abs(res[True] - res[False]) <= 0.02 * res[False], res
