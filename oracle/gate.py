"""FP64 oracle of the learned smoothness indicator (test infrastructure only).

The indicator is a small MLP that predicts, per cell, whether the PPM limiter
would change any reconstructed value on any of the 13 lines through the cell;
where it predicts "smooth", the unlimited interface formula may be used.

Definitions written out plainly:
  * features (54): for the 3x3x3 neighbourhood k of cell i, in (z, y, x)
    lexicographic order, first density then pressure,
        x = (q(i+k) - q(i)) / (|q(i+k)| + |q(i)|),
    a bounded, scale-invariant relative difference (the centre entry is 0);
    pressure p = (gamma - 1) eps from the oracle's primitive recovery;
  * label: 1 where the oracle's limiter acted significantly on a line through
    the cell (``core.step(..., want_flags=True)``): for density, velocity,
    internal energy, tracer or species, the limited interface pair differs
    from the unlimited one by more than 1e-4 of the field's scale at the cell
    (|q0|; |v| + c for velocities); the spin fields are always limited;
  * network: h1 = relu(W1 x + b1) (32), h2 = relu(W2 h1 + b2) (32),
    out = sigmoid(w3 . h2 + b3); parameters packed in the order
    W1[32][54], b1[32], W2[32][32], b2[32], w3[32], b3.  Training uses it
    with BF16-rounded parameters and exact activations (forward); the
    deployed form also rounds x and h1 to BF16 (forward_infer: BF16
    operands of the tensor cores, FP32 accumulation);
  * loss: class-weighted binary cross-entropy, mean over the batch,
        L = -mean( w1 y log(out) + w0 (1-y) log(1-out) ).
"""
from __future__ import annotations

import numpy as np

NIN, NH = 54, 32
SIZES = [("W1", (NH, NIN)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("w3", (NH,)), ("b3", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shp in SIZES:
        n = int(np.prod(shp))
        out[name] = theta[o:o + n].reshape(shp)
        o += n
    return out


def features(U: np.ndarray, gamma: float, N: int = 8, G: int = 3, lo: int = 0, hi: int | None = None) -> np.ndarray:
    """U [n_sub][F][S][S][S] (ghosts filled) -> [n_sub * M^3][54] for the cells
    with interior coordinates in [lo, hi)^3 (default: the N^3 interior cells;
    lo = -1, hi = N + 1 adds the ghost shell whose lines are reconstructed)."""
    from . import core
    hi = N if hi is None else hi
    M = hi - lo
    n = U.shape[0]
    P = core.OracleParams(gamma=gamma)
    rho = U[:, 0]
    pres = np.empty_like(rho)
    for s in range(n):
        flat = U[s].reshape(U.shape[1], -1)
        for c in range(flat.shape[1]):
            pres[s].reshape(-1)[c] = (gamma - 1.0) * core.primitives(P, flat[:, c].copy())[4]
    out = np.empty((n, M, M, M, 2 * 27))
    j = 0
    a = G + lo
    for q in (rho, pres):
        qc = q[:, a:a + M, a:a + M, a:a + M]
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    qk = q[:, a + dz:a + dz + M, a + dy:a + dy + M, a + dx:a + dx + M]
                    out[..., j] = (qk - qc) / (np.abs(qk) + np.abs(qc))
                    j += 1
    return out.reshape(n * M ** 3, 54)


def labels(U: np.ndarray, gamma: float, origin=None, h=1.0) -> np.ndarray:
    from . import core
    n = U.shape[0]
    o = np.zeros((n, 3)) if origin is None else origin
    _, _, fl = core.step(core.OracleParams(gamma=gamma), U, o, h, want_flags=True)
    return fl.reshape(-1).astype(np.float64)


def forward(theta: np.ndarray, X: np.ndarray):
    p = unpack(theta)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    z3 = h2 @ p["w3"] + p["b3"][0]
    out = 1.0 / (1.0 + np.exp(-z3))
    return out, (X, z1, h1, z2, h2, z3)


def forward_infer(theta: np.ndarray, X: np.ndarray) -> np.ndarray:
    """The deployed indicator (BF16 operands, FP32 accumulation, as in the
    step kernel's tensor-core evaluation): the features and the first hidden
    layer are rounded to BF16 (ties to even), everything else is exact here.
    theta: parameters already rounded to BF16.  Returns the sigmoid output."""
    p = unpack(theta)
    xb = bf16_round(X)
    h1 = bf16_round(np.maximum(xb @ p["W1"].T + p["b1"], 0.0))
    h2 = np.maximum(h1 @ p["W2"].T + p["b2"], 0.0)
    z3 = h2 @ p["w3"] + p["b3"][0]
    return 1.0 / (1.0 + np.exp(-z3))


def loss_and_grad(theta: np.ndarray, X: np.ndarray, y: np.ndarray, w1: float = 1.0, w0: float = 1.0):
    """Mean class-weighted BCE and its gradient (backpropagation by hand)."""
    out, (X, z1, h1, z2, h2, z3) = forward(theta, X)
    n = X.shape[0]
    eps = 1e-300
    L = -np.mean(w1 * y * np.log(out + eps) + w0 * (1 - y) * np.log(1 - out + eps))
    # dL/dz3 for the weighted BCE through the sigmoid
    g3 = (w1 * y * (out - 1.0) + w0 * (1 - y) * out) / n
    p = unpack(theta)
    gw3 = h2.T @ g3
    gb3 = np.array([g3.sum()])
    gh2 = np.outer(g3, p["w3"])
    gz2 = gh2 * (z2 > 0)
    gW2 = gz2.T @ h1
    gb2 = gz2.sum(axis=0)
    gh1 = gz2 @ p["W2"]
    gz1 = gh1 * (z1 > 0)
    gW1 = gz1.T @ X
    gb1 = gz1.sum(axis=0)
    grad = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gw3, gb3])
    return L, grad


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round FP32 values to the nearest BF16 (ties to even), returned as FP64."""
    f = np.asarray(a, dtype=np.float32).copy()
    u = f.view(np.uint32)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.view(np.float32).astype(np.float64)
