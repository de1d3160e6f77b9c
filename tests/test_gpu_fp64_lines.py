"""The FP64 step (every PPM line once per cell) under every launch shape.

Each persistent CTA owns a line-end buffer and prefetches its next tile
while it sweeps the faces of the current one, so the number of CTAs
decides which buffer a tile's lines go through and how long each CTA's
chain of prefetches is.  None of that may change a bit: one CTA looping
over every tile, odd counts, more CTAs than SMs (a second wave) and the
autotuner's choice all give the default launch's dU/dt and amax, and a
single sub-grid gives the axis-sweep kernel's (hydro_step_static) bits.
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


def _inputs(n, seed):
    U = torch.tensor(W.random_subgrids(n, seed, GAMMA), device="cuda")
    rng = np.random.default_rng(seed + 1)
    o = torch.tensor(rng.uniform(-1, 1, (n, 3)), device="cuda")
    h = torch.tensor(rng.uniform(0.01, 0.1, n), device="cuda")
    g = torch.tensor(rng.normal(0, 0.1, (n, 3, 8, 8, 8)), device="cuda")
    return U, o, h, g


def _step(H, ctx, U, o, h, g, static=False):
    n = U.shape[0]
    dU = torch.full((n, 10, 8, 8, 8), float("nan"), dtype=torch.float64, device="cuda")
    am = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    B = H.make_batch(U, o, h, g)
    if static:
        H.hydro_step_static(ctx, B, 0.0, dU, am)
    else:
        H.hydro_step(ctx, B, 0.0, dU, am)
    torch.cuda.synchronize()
    return dU, am


def _bits(t):
    return t.contiguous().view(torch.int64)


def test_launch_shapes_give_the_same_bits(H):
    n = 400
    U, o, h, g = _inputs(n, 61)
    ctx = H.Context(GAMMA, 0.13)
    ref, am_ref = _step(H, ctx, U, o, h, g)
    assert torch.isfinite(ref).all() and H.hydro_status(ctx) == 0
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for ctas in (1, 5, sms - 1, 2 * sms, n):
        H.hydro_set_launch(ctx, H.HYDRO_DECOMP_ROWS, ctas)
        dU, am = _step(H, ctx, U, o, h, g)
        assert bool((_bits(dU) == _bits(ref)).all()), ctas
        assert bool((_bits(am) == _bits(am_ref)).all()), ctas
    H.hydro_set_launch(ctx, H.HYDRO_DECOMP_AUTO, 0)
    dU = torch.empty_like(ref)
    am = torch.empty_like(am_ref)
    ctas = H.hydro_autotune_step(ctx, H.make_batch(U, o, h, g), dU, am)
    assert ctas > 0
    dU2, am2 = _step(H, ctx, U, o, h, g)
    assert bool((_bits(dU2) == _bits(ref)).all()) and bool((_bits(am2) == _bits(am_ref)).all())
    assert H.hydro_status(ctx) == 0


@pytest.mark.parametrize("contact", [0, 1])
def test_single_subgrid_matches_the_axis_sweeps(H, contact):
    U, o, h, g = _inputs(1, 71 + contact)
    ctx = H.Context(GAMMA, 0.2)
    H.hydro_set_mode(ctx, H.HYDRO_PREC_FP64, contact=contact)
    dU, am = _step(H, ctx, U, o, h, g)
    dUs, ams = _step(H, ctx, U, o, h, g, static=True)
    assert bool((_bits(dU) == _bits(dUs)).all()) and bool((_bits(am) == _bits(ams)).all())
    assert H.hydro_status(ctx) == 0
