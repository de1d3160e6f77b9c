"""Parity measure between a tested result and the oracle (test infrastructure).

Per-field relative error: the largest |got - want| of a field divided by that
field's largest |want| over the compared set.  A pure relative error per cell
is undefined where a rate is ~0, and a field can be zero up to rounding
altogether: the spin rate dz/dt of a reflection-symmetric flow is a sum of
torques (h/2) d x F_s that cancel only to round-off.  Such a field is
normalised instead by the size of the terms it is made of, the lever arm h
times the largest momentum rate (or momentum), so rounding noise in it is
measured against the quantities that produced it.
"""
import numpy as np

SPIN = (6, 7, 8)
MOMENTUM = (1, 2, 3)


def field_scales(want: np.ndarray, h) -> np.ndarray:
    """want [n][F][...] -> per-field normalisation [F]."""
    axes = tuple(i for i in range(want.ndim) if i != 1)
    sc = np.abs(want).max(axis=axes)
    hmax = float(np.max(h))
    mom = np.abs(want[:, list(MOMENTUM)]).max()
    for k in SPIN:
        sc[k] = max(sc[k], hmax * mom)
    sc[sc == 0] = 1.0
    return sc


def max_rel_error(got: np.ndarray, want: np.ndarray, h) -> float:
    """Largest per-field normalised error (see module docstring)."""
    axes = tuple(i for i in range(want.ndim) if i != 1)
    err = np.abs(got - want).max(axis=axes)
    return float((err / field_scales(want, h)).max())


EPS32 = 2.0 ** -24  # unit roundoff of FP32


def flux_ratio(faces: np.ndarray, scale: np.ndarray, h) -> np.ndarray:
    """R_k: the size of the terms rate k is computed from, over its normalisation.

    faces: the oracle's boundary-face sums [n][6][F+3][N][N] (F face fluxes,
    then the 3 torque components).  A rate is a difference of face fluxes
    over h, so its non-spin terms are max|F_k| / h.  The spin rate is also
    made of point torques (x_q - x_c) x F_s with |x_q - x_c| ~ h/2, divided
    by h: terms of size max|F_s| / 2, which cancel when the pressure is
    nearly uniform across a face."""
    F = scale.shape[0]
    fm = np.abs(faces).max(axis=(0, 1, 3, 4))
    hmax = float(np.max(h))
    R = fm[:F] / hmax
    for m, k in enumerate(SPIN):
        R[k] = max(R[k], fm[F + m] / hmax, 0.5 * fm[list(MOMENTUM)].max())
    return R / scale


def mixed_budget(ref: np.ndarray, pert: np.ndarray, faces: np.ndarray, h) -> tuple[np.ndarray, np.ndarray]:
    """Per-field error budget of the mixed-precision step against the oracle.

    ref: the oracle's rates; pert: the oracle's rates on the inputs rounded
    to FP32 (sens = their normalised difference: what FP32 storage of the
    primitives alone costs).  The FP32 reconstruction and flux arithmetic
    adds rounding of relative size ~EPS32 to every face flux and point
    torque, which the FP64 divergence keeps: at most a few EPS32 times the
    terms of the rate (R_k, flux_ratio).  That term dominates where a rate
    is a small residual of large fluxes (near hydrostatic equilibrium).
    Budget: 8 sens + 8 EPS32 R + 4e-7.  Returns (budget [F], sens [F])."""
    sc = field_scales(ref, h)
    axes = tuple(i for i in range(ref.ndim) if i != 1)
    sens = (np.abs(pert - ref) / sc.reshape((1, -1) + (1,) * (ref.ndim - 2))).max(axis=axes)
    return 8 * sens + 8 * EPS32 * flux_ratio(faces, sc, h) + 4e-7, sens
