"""hydro_step_static: the allocation-free variant of hydro_step.

Callers that cannot call cudaMalloc (a host code whose device memory all
belongs to its own pool allocator, or a time loop that cannot afford an
allocation's device-wide synchronisation) use this entry point; it runs the
same FP64 step kernel with its scratch in a fixed array of the library.  This
file is collected last so that a run stopping at the first failure has run
everything else before it.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2107_10987_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-12  # the parity tolerance of the FP64 path
GAMMA = 5.0 / 3.0


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2107_10987_gb300 import _build, hydro
    _build.build()
    return hydro


def _inputs(n, seed, dev):
    U = torch.tensor(W.random_subgrids(n, seed, GAMMA), device=dev)
    rng = np.random.default_rng(seed)
    o = torch.tensor(rng.uniform(-1, 1, (n, 3)), device=dev)
    h = torch.tensor(rng.uniform(0.01, 0.1, n), device=dev)
    return U, o, h


def test_static_step_matches_hydro_step_on_two_calls_in_a_row(H):
    from oracle.compare import max_rel_error
    dev = torch.device("cuda")
    ctx = H.Context(GAMMA, 0.23)
    status = torch.full((1,), 7, dtype=torch.int32, device=dev)
    # a full batch first, then a smaller one with other data: the second call
    # must not see anything the first left in the shared array
    for call, (n, seed) in enumerate(((H.HYDRO_STATIC_MAX_SUB, 31), (37, 32))):
        U, o, h = _inputs(n, seed, dev)
        B = H.make_batch(U, o, h)
        dU_ref = torch.empty((n, 10, 8, 8, 8), dtype=torch.float64, device=dev)
        am_ref = torch.empty(n, dtype=torch.float64, device=dev)
        H.hydro_step(ctx, B, 0.0, dU_ref, am_ref)
        dU = torch.full_like(dU_ref, float("nan"))
        am = torch.full_like(am_ref, float("nan"))
        H.hydro_step_static(ctx, B, 0.0, dU, am, status=status)
        torch.cuda.synchronize()
        got, want = dU.cpu().numpy(), dU_ref.cpu().numpy()
        assert np.all(np.isfinite(got)), call
        assert max_rel_error(got, want, h.max().item()) <= TOL, call
        assert np.allclose(am.cpu().numpy(), am_ref.cpu().numpy(), rtol=1e-15, atol=0), call
        assert status.item() == 0, call  # cleared by the call, no fault bits


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
