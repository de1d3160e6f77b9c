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
