"""Training driver of the learned smoothness indicator (host-side loop only).

Every arithmetic step runs in the library's kernels through the C ABI:
the runs that generate the data (hydro_rk3_step, mixed precision),
the features and labels (hydro_gate_data), the loss and gradient
(hydro_mlp_loss_grad) and the optimiser (hydro_mlp_adam).  This module only
orders the calls, draws minibatch indices and picks the decision threshold.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import hydro as H
from . import workloads as W

NPARAM = H.HYDRO_GATE_NPARAM


def collect(seeds, n: int = 64, snapshots=(8, 24, 48), device="cuda"):
    """Evolve each seeded run (uniform mesh, outflow, mixed precision) and
    gather (features, labels) of every interior cell at the given step
    counts.  Returns (X [m][54] float32, y [m] float32, chunks) with chunks
    the list of (offset, nb) of every snapshot (nb^3 sub-grids of 8^3)."""
    nb = n // 8
    Xs, ys, chunks = [], [], []
    off = 0
    for sd, kind, gamma, Ug, h, lo in W.indicator_runs(seeds, n):
        ctx = H.Context(gamma, 0.0)
        H.hydro_set_mode(ctx, H.HYDRO_PREC_MIXED)
        sub = np.zeros((nb ** 3, 10, 14, 14, 14))
        sub[:, :, 3:-3, 3:-3, 3:-3] = W.box_to_subgrids(Ug)
        Ua = torch.tensor(sub, device=device)
        Ub = torch.zeros_like(Ua)
        o = torch.tensor(W.uniform_mesh(nb, 8, 2.0)[0], device=device)
        hv = torch.full((nb ** 3,), h, dtype=torch.float64, device=device)
        dU = torch.empty((nb ** 3, 10, 8, 8, 8), dtype=torch.float64, device=device)
        am = torch.empty(nb ** 3, dtype=torch.float64, device=device)
        dt = torch.empty(1, dtype=torch.float64, device=device)
        desc = H.make_rk3_desc(Ua, Ub, o, hv, (nb, nb, nb), H.HYDRO_BC_OUTFLOW, dU, am, dt)
        bufs = (Ua, Ub)
        step = 0
        for target in snapshots:
            while step < target:
                H.hydro_rk3_step(ctx, desc, step % 2)
                step += 1
            cur = bufs[step % 2]
            B = H.make_batch(cur, o, hv)
            H.hydro_fill_ghosts_uniform(ctx, B, nb, nb, nb, H.HYDRO_BC_OUTFLOW)
            X = torch.empty((nb ** 3 * 512, 54), dtype=torch.float32, device=device)
            y = torch.empty(nb ** 3 * 512, dtype=torch.uint8, device=device)
            H.hydro_gate_data(ctx, B, X, y)
            Xs.append(X)
            ys.append(y.float())
            chunks.append((off, nb))
            off += X.shape[0]
        torch.cuda.synchronize()
        ctx.close()
    return torch.cat(Xs), torch.cat(ys), chunks


def init_params(seed: int = 0, device="cuda") -> torch.Tensor:
    """He-style seeded initialisation (host RNG), packed as the C ABI expects."""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0, math.sqrt(2.0 / 54), 32 * 54), np.zeros(32), rng.normal(0, math.sqrt(2.0 / 32), 32 * 32),
             np.zeros(32), rng.normal(0, math.sqrt(1.0 / 32), 32), np.zeros(1)]
    return torch.tensor(np.concatenate(parts), dtype=torch.float32, device=device)


def train(X, y, iters: int = 2000, batch: int = 65536, lr: float = 3e-3, w1: float = 8.0, w0: float = 1.0,
          seed: int = 0):
    """Adam on minibatches; returns (params, loss history)."""
    dev = X.device
    params = init_params(seed, dev)
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    grad = torch.empty_like(params)
    loss = torch.empty(1, dtype=torch.float32, device=dev)
    work = torch.empty(H.hydro_mlp_work_bytes(batch) // 4 + 1, dtype=torch.float32, device=dev)
    g = torch.Generator(device="cpu").manual_seed(seed)
    # one shuffle of the data set, then contiguous minibatches (epochs)
    perm = torch.randperm(X.shape[0], generator=g).to(dev)
    Xs, ys = X[perm].contiguous(), y[perm].contiguous()
    nb = max(1, Xs.shape[0] // batch)
    hist = []
    for t in range(1, iters + 1):
        b = (t - 1) % nb
        Xb, yb = Xs[b * batch:(b + 1) * batch], ys[b * batch:(b + 1) * batch]
        H.hydro_mlp_loss_grad(params, Xb, yb, grad, loss, w1, w0, work)
        H.hydro_mlp_adam(params, m, v, grad, t, lr * (0.1 ** (t / iters)))
        if t % 100 == 0 or t == 1:
            hist.append((t, loss.item()))
    return params, hist


def predict(params, X, chunk: int = 1 << 22):
    out = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
    for i in range(0, X.shape[0], chunk):
        H.hydro_mlp_forward(params, X[i:i + chunk], out[i:i + chunk])
    return out


def _box(v, nb):
    """[nb^3 * 512] per-cell values in sub-grid order -> [1][1][n][n][n] box."""
    return v.view(nb, nb, nb, 8, 8, 8).permute(0, 3, 1, 4, 2, 5).reshape(1, 1, nb * 8, nb * 8, nb * 8)


def dilated_smooth(pred, thr: float, chunks):
    """The step kernel's decision: smooth where every cell of the 3x3x3 block
    is predicted smooth (outflow edges replicated).  Returns per-cell boxes."""
    out = []
    for off, nb in chunks:
        ns = _box((pred[off:off + nb ** 3 * 512] >= thr).float(), nb)
        ns = torch.nn.functional.pad(ns, (1, 1, 1, 1, 1, 1), mode="replicate")
        out.append(torch.nn.functional.max_pool3d(ns, 3, stride=1) < 0.5)
    return out


def _stats(pred, thr, y, chunks):
    tp = fn = fp = sm = tot = pos = 0
    for (off, nb), smooth in zip(chunks, dilated_smooth(pred, thr, chunks)):
        yy = _box(y[off:off + nb ** 3 * 512], nb) > 0.5
        tp += (~smooth & yy).sum().item()
        fn += (smooth & yy).sum().item()
        fp += (~smooth & ~yy).sum().item()
        sm += smooth.sum().item()
        tot += smooth.numel()
        pos += yy.sum().item()
    return {"recall": tp / max(tp + fn, 1), "precision": tp / max(tp + fp, 1), "frac_smooth": sm / tot,
            "frac_active": pos / tot, "n": tot, "threshold": thr}


def choose_threshold(params, X, y, chunks, recall: float = 0.999) -> float:
    """Largest threshold whose dilated decisions keep the recall of
    limiter-active cells at or above `recall` (bisection; recall does not
    increase with the threshold)."""
    pred = predict(params, X)
    lo, hi = 0.0, 1.0
    for _ in range(40):
        mid = 0.5 * (lo + hi)
        if _stats(pred, mid, y, chunks)["recall"] >= recall:
            lo = mid
        else:
            hi = mid
    return float(min(max(lo, 1e-7), 1 - 1e-7))


def evaluate(params, thr: float, X, y, chunks) -> dict:
    return _stats(predict(params, X), thr, y, chunks)
