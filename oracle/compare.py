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


def flux_ratio(faces: np.ndarray, scale: np.ndarray, h, U: np.ndarray | None = None,
               amax: np.ndarray | None = None) -> np.ndarray:
    """R_k: the size of the terms rate k is computed from, over its normalisation.

    faces: the oracle's boundary-face sums [n][6][F+3][N][N] (F face fluxes,
    then the 3 torque components); h: cell width, scalar or per sub-grid.
    A rate is a difference of face fluxes over h, so its terms are at least
    max|F_k| / h.  Each point flux is F = (F_L + F_R)/2 - a (U_R - U_L)/2:
    where the two reconstructed states nearly agree and the signal speed a
    is large (hot, thin gas), the face flux is small but the dissipation
    terms a|U_k| / 2 are not, so with the padded states U [n][F][S][S][S]
    and the signal speeds amax [n] the terms a |U_k| / h count too.  The
    spin rate is also made of point torques (x_q - x_c) x F_s with
    |x_q - x_c| ~ h/2, divided by h: terms of size max|F_s| / 2 and
    a |s| / 2, which cancel when the pressure or the momentum is nearly
    uniform across a face."""
    n = faces.shape[0]
    F = scale.shape[0]
    hs = np.broadcast_to(np.asarray(h, dtype=np.float64), (n,))
    fm = np.abs(faces).max(axis=(1, 3, 4))  # [n][F+3]
    R = fm[:, :F] / hs[:, None]
    mom = fm[:, list(MOMENTUM)].max(axis=1)
    for m, k in enumerate(SPIN):
        R[:, k] = np.maximum(np.maximum(R[:, k], fm[:, F + m] / hs), 0.5 * mom)
    if U is not None and amax is not None:
        um = np.abs(U).max(axis=(2, 3, 4))[:, :F]  # [n][F]
        R = np.maximum(R, np.asarray(amax)[:, None] * um / hs[:, None])
        smax = um[:, list(MOMENTUM)].max(axis=1)
        for k in SPIN:
            R[:, k] = np.maximum(R[:, k], 0.5 * np.asarray(amax) * smax)
    return R.max(axis=0) / scale


def mixed_budget(ref: np.ndarray, pert: np.ndarray, faces: np.ndarray, h, U: np.ndarray | None = None,
                 amax: np.ndarray | None = None) -> tuple[np.ndarray, np.ndarray]:
    """Per-field error budget of the mixed-precision step against the oracle.

    ref: the oracle's rates; pert: the oracle's rates on the inputs rounded
    to FP32 (sens = their normalised difference: what FP32 storage of the
    primitives alone costs).  The FP32 reconstruction and flux arithmetic
    adds rounding of relative size ~EPS32 to every term of every point flux
    and point torque, which the FP64 divergence keeps: at most a few EPS32
    times the terms of the rate (R_k, flux_ratio; pass the padded states U
    and the oracle's amax to include the dissipation terms).  That term
    dominates where a rate is a small residual of large terms (near
    hydrostatic equilibrium, hot thin gas).
    Budget: 8 sens + 8 EPS32 R + 4e-7.  Returns (budget [F], sens [F])."""
    hmax = float(np.max(h))
    sc = field_scales(ref, hmax)
    axes = tuple(i for i in range(ref.ndim) if i != 1)
    sens = (np.abs(pert - ref) / sc.reshape((1, -1) + (1,) * (ref.ndim - 2))).max(axis=axes)
    return 8 * sens + 8 * EPS32 * flux_ratio(faces, sc, h, U, amax) + 4e-7, sens
