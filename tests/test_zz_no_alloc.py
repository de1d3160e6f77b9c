"""hydro_step_static: the allocation-free variant of hydro_step.

Callers that cannot call cudaMalloc (a host code whose device memory all
belongs to its own pool allocator, or a time loop that cannot afford an
allocation's device-wide synchronisation) use this entry point; it runs the
FP64 step with its scratch in a fixed array of the library: the axis-sweep
kernel, which reconstructs each line inside its three sweeps, where
hydro_step's kernel evaluates every line once per cell into a per-CTA buffer.
The two organisations compute the same operations on the same operands, so
the comparison below is also a bit-for-bit check of one against the other.  This
file is collected last so that a run stopping at the first failure has run
everything else before it.
"""
import gc

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


def _inputs(n, seed, dev, smooth=False):
    U = torch.tensor(W.random_subgrids(n, seed, GAMMA, smooth=smooth), device=dev)
    rng = np.random.default_rng(seed)
    o = torch.tensor(rng.uniform(-1, 1, (n, 3)), device=dev)
    h = torch.tensor(rng.uniform(0.01, 0.1, n), device=dev)
    return U, o, h


def _bits(t):
    return t.contiguous().view(torch.int64)


@pytest.mark.parametrize("variant", ["default", "old_module", "contact", "indicator", "contact_indicator"])
def test_static_step_matches_hydro_step_on_two_calls_in_a_row(H, variant):
    """Both entry points run the same arithmetic in a fixed order per
    sub-grid (each line's values are ppm64's, the face sums keep their order),
    so the results are equal bit for bit, for every mode the FP64
    kernels have: the 9-point faces, the face-centre flux (old module),
    contact steepening, the learned indicator, and steepening with the
    indicator.  A second call, after a
    warm-up, changes neither torch's nor the driver's count of free device
    memory."""
    dev = torch.device("cuda")
    ctx = H.Context(GAMMA, 0.23)
    if variant == "old_module":
        H.hydro_set_mode(ctx, H.HYDRO_PREC_FP64, flux_points=1)
    elif variant == "contact":
        H.hydro_set_mode(ctx, H.HYDRO_PREC_FP64, contact=1)
    elif variant in ("indicator", "contact_indicator"):
        from oracle import gate
        if variant == "contact_indicator":
            H.hydro_set_mode(ctx, H.HYDRO_PREC_FP64, contact=1)
        rng = np.random.default_rng(21)
        theta = torch.tensor(rng.normal(0, 0.3, gate.NPARAM).astype(np.float32), device=dev)
        H.hydro_set_indicator(ctx, theta, 0.9)
    status = torch.full((1,), 7, dtype=torch.int32, device=dev)
    # a full batch first, then a smaller one with other data: the second call
    # must not see anything the first left in the shared array
    for call, (n, seed) in enumerate(((H.HYDRO_STATIC_MAX_SUB, 31), (37, 32))):
        # smooth data under the indicator: the unlimited formula stays physical
        U, o, h = _inputs(n, seed, dev, smooth=variant in ("indicator", "contact_indicator"))
        B = H.make_batch(U, o, h)
        dU_ref = torch.empty((n, 10, 8, 8, 8), dtype=torch.float64, device=dev)
        am_ref = torch.empty(n, dtype=torch.float64, device=dev)
        H.hydro_step(ctx, B, 0.0, dU_ref, am_ref)
        dU = torch.full_like(dU_ref, float("nan"))
        am = torch.full_like(am_ref, float("nan"))
        H.hydro_step_static(ctx, B, 0.0, dU, am, status=status)
        torch.cuda.synchronize()
        assert bool((_bits(dU) == _bits(dU_ref)).all()), call
        assert bool((_bits(am) == _bits(am_ref)).all()), call
        assert status.item() == 0, call  # cleared by the call, no fault bits
        if call == 1:
            # the entry point allocates nothing: an already warmed-up call
            # leaves the device's free memory and torch's pool as they were
            # (unreferenced tensors of earlier tests collected first, so that
            # no deallocation lands between the two readings)
            gc.collect()
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            res0, alloc0 = torch.cuda.memory_reserved(), torch.cuda.memory_allocated()
            H.hydro_step_static(ctx, B, 0.0, dU, am, status=status)
            torch.cuda.synchronize()
            assert torch.cuda.mem_get_info()[0] == free0
            assert torch.cuda.memory_reserved() == res0
            assert torch.cuda.memory_allocated() == alloc0
            assert bool((_bits(dU) == _bits(dU_ref)).all())
    assert H.hydro_status(ctx) == 0


def test_static_step_unsupported_modes(H):
    ctx = H.Context(GAMMA, 0.0)
    B = H.Batch(4, 16, 16, 16, None)  # rejected on the host before any pointer is used
    H.hydro_set_mode(ctx, H.HYDRO_PREC_MIXED)
    with pytest.raises(H.HydroError) as e:
        H.hydro_step_static(ctx, B, 0.0, 16, 16)
    assert e.value.code == H.HYDRO_EUNSUP
    H.hydro_set_mode(ctx, H.HYDRO_PREC_FP64)
    for bad_dt in (float("nan"), float("inf"), -1.0):
        with pytest.raises(H.HydroError) as e:
            H.hydro_step_static(ctx, B, bad_dt, 16, 16)
        assert e.value.code == H.HYDRO_EINVAL


def test_static_step_rejects_batches_beyond_its_scratch(H):
    dev = torch.device("cuda")
    ctx = H.Context(GAMMA, 0.0)
    n = H.HYDRO_STATIC_MAX_SUB + 1
    B = H.Batch(n, 16, 16, 16, None)  # rejected on the host before any pointer is used
    with pytest.raises(H.HydroError) as e:
        H.hydro_step_static(ctx, B, 0.0, 16, 16)
    assert e.value.code == H.HYDRO_ERANGE
    H.hydro_step_static(ctx, H.Batch(0, None, None, None, None), 0.0, None, None)  # empty: no-op
    del dev
