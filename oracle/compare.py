"""Parity measure between a tested result and the oracle (test infrastructure).

Per sub-grid and per field.  The error of field k in sub-grid s is the
largest |got - want| over that sub-grid's cells, divided by the field's
scale in that sub-grid:

    scale[s, k] = max( max_cells |want[s, k]|,  floor[s, k] ).

The first term makes the measure a relative error against the sub-grid's
own values, so a thin ambient sub-grid (density 1e-10) is held to its own
rates, not to those of a dense one elsewhere in the batch.  A pure relative
error per cell would be undefined where a rate is ~0.

The floor is needed only where a field of a sub-grid is zero up to
rounding while the terms it is computed from are not:
  * the spin rate dz/dt of a reflection-symmetric flow is a sum of torques
    (h/2) d x F_s that cancel only to round-off: its floor is the lever arm
    h times the sub-grid's largest momentum rate (or momentum);
  * a rate in a sub-grid near equilibrium (a uniform stream, hydrostatic or
    thin gas moving with the rotating frame) is a small residual of large
    flux terms.  rate_floor() states the size of those terms; two
    implementations that round the same terms differently disagree by a
    few units of roundoff of the terms, not of the residual.
Without a floor argument only the spin floor applies.
"""
import numpy as np

SPIN = (6, 7, 8)
MOMENTUM = (1, 2, 3)
RHO, EGAS = 0, 4


def _ratio(err: np.ndarray, sc: np.ndarray) -> np.ndarray:
    """err / sc, with 0/0 = 0 and x/0 = inf (a field that is exactly zero in
    a sub-grid must be matched exactly)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(sc > 0, err / np.where(sc > 0, sc, 1.0), np.where(err > 0, np.inf, 0.0))


def _per_sub(x: np.ndarray) -> np.ndarray:
    """[n][F][...] -> max |x| per (sub-grid, field), shape [n][F]."""
    n, F = x.shape[:2]
    return np.abs(x).reshape(n, F, -1).max(axis=2)


def subgrid_scales(want: np.ndarray, h, floor: np.ndarray | None = None) -> np.ndarray:
    """Normalisation [n][F] of each field in each sub-grid (module docstring)."""
    n = want.shape[0]
    sc = _per_sub(want)
    hs = np.broadcast_to(np.asarray(h, dtype=np.float64), (n,))
    if floor is not None:
        sc = np.maximum(sc, floor)
    # the spin's lever-arm floor from the (floored) momentum scale: where the
    # pressure is uniform the momentum rate cancels exactly while the point
    # torques of the same pressure terms cancel only to round-off
    mom = sc[:, list(MOMENTUM)].max(axis=1)
    for k in SPIN:
        sc[:, k] = np.maximum(sc[:, k], hs * mom)
    return sc


def max_rel_error(got: np.ndarray, want: np.ndarray, h, floor: np.ndarray | None = None) -> float:
    """Largest per-sub-grid, per-field normalised error.  A field that is
    exactly zero in a sub-grid (scale 0) must be matched exactly."""
    return float(_ratio(_per_sub(got - want), subgrid_scales(want, h, floor)).max())


# Fraction of the largest flux term below which a rate counts as a
# cancellation residual.  A rate is -(1/h) sum over 3 axes x 2 faces x 9
# points of weighted point fluxes (F_L + F_R)/2 - a (U_R - U_L)/2, plus
# sources: about 160 terms, each no larger than T (rate_floor).  Two FP64
# evaluations that contract different products into FMAs differ by at most
# about one unit of roundoff (1.1e-16) per term, so by at most ~1.8e-14 T,
# and typically by the square root of that count, ~1.4e-15 T.  With the
# FP64 tolerance 1e-12 and KAPPA = 1e-2 a residual rate may differ by 1e-14
# T, about 90 units of roundoff of its largest term; a rate larger than
# KAPPA T is held to 1e-12 of itself.
KAPPA = 1e-2


def rate_floor(U: np.ndarray, amax, h, omega: float = 0.0, g: np.ndarray | None = None, gamma: float = 5.0 / 3.0,
               kappa: float = KAPPA) -> np.ndarray:
    """kappa times the size T[s, k] of the largest term that rate k of
    sub-grid s is computed from, [n][F].

    U: the padded states [n][F][S][S][S] the rates were computed from; amax:
    the sub-grid's largest signal speed |u_n| + c (every |u_n| and c of its
    points is below it); h: cell width, scalar or per sub-grid; omega, g:
    the frame rotation and the gravity input of the step.
      - a conserved field U_k is advected with |u_n| <= amax: flux terms of
        size amax max|U_k|, divided by h in the divergence;
      - momentum also carries the pressure, p = rho c^2 / gamma <= rho
        amax^2, and the sources omega |s| and rho |g|;
      - energy carries (E + p) u_n with p <= (gamma - 1) E: gamma amax E,
        and the source s.g;
      - spin gets the point torques (h/2)|F_s| / h, F_s up to
        amax (|s| + rho amax), and the frame term omega |z|."""
    n, F = U.shape[:2]
    hs = np.broadcast_to(np.asarray(h, dtype=np.float64), (n,))
    a = np.broadcast_to(np.asarray(amax, dtype=np.float64), (n,))
    Um = _per_sub(U)
    rho = Um[:, RHO]
    smax = Um[:, list(MOMENTUM)].max(axis=1)
    T = a[:, None] * Um / hs[:, None]
    mom = a * np.maximum(smax, rho * a) / hs + abs(omega) * smax
    e = gamma * a * Um[:, EGAS] / hs
    spin = np.maximum(a * Um[:, list(SPIN)].max(axis=1) / hs, 0.5 * a * (smax + rho * a)) + \
        abs(omega) * Um[:, list(SPIN)].max(axis=1)
    if g is not None:
        gm = np.abs(np.asarray(g)).reshape(n, -1).max(axis=1)
        mom = mom + rho * gm
        e = e + smax * gm
    for k in MOMENTUM:
        T[:, k] = np.maximum(T[:, k], mom)
    T[:, EGAS] = np.maximum(T[:, EGAS], e)
    for k in SPIN:
        T[:, k] = np.maximum(T[:, k], spin)
    return kappa * T


def state_floor(U0: np.ndarray, amax, kappa: float = KAPPA) -> np.ndarray:
    """Floor [n][F] for states after an RK3 step from padded states U0 with
    signal speeds amax: a momentum component that is ~0 in a sub-grid
    changes by dt times residual rates, dt ~ cfl h / amax, so its rounding
    differences are measured against kappa rho amax (the momentum its
    pressure terms could create in a step).  Other fields are never ~0 next
    to nonzero terms (density, energy, tracer and species are positive), and
    spin keeps its lever-arm floor."""
    n, F = U0.shape[:2]
    a = np.broadcast_to(np.asarray(amax, dtype=np.float64), (n,))
    Um = _per_sub(U0)
    fl = np.zeros((n, F))
    for k in MOMENTUM:
        fl[:, k] = kappa * Um[:, RHO] * a
    return fl


EPS32 = 2.0 ** -24  # unit roundoff of FP32


def flux_ratio(faces: np.ndarray, scale: np.ndarray, h, U: np.ndarray | None = None,
               amax: np.ndarray | None = None, gamma: float = 5.0 / 3.0) -> np.ndarray:
    """R[s, k]: the size of the terms rate k of sub-grid s is computed from,
    over its normalisation scale[s, k] ([n][F]).

    faces: the oracle's boundary-face sums [n][6][F+3][N][N] (F face fluxes,
    then the 3 torque components), or None; h: cell width, scalar or per
    sub-grid.
    A rate is a difference of face fluxes over h, so its terms are at least
    max|F_k| / h.  Each point flux is F = (F_L + F_R)/2 - a (U_R - U_L)/2:
    where the two reconstructed states nearly agree and the signal speed a
    is large (hot, thin gas), the face flux is small but the dissipation
    terms a|U_k| / 2 are not, so with the padded states U [n][F][S][S][S]
    and the signal speeds amax [n] the terms a |U_k| / h count too, and so
    does the pressure that the momentum flux s u_n + p e_a carries, p / h
    with p = (gamma - 1)(E - |s|^2 / (2 rho)) (the face sums, when given,
    include it; a step that exports none is measured by the states).  The
    spin rate is also made of point torques (x_q - x_c) x F_s with
    |x_q - x_c| ~ h/2, divided by h: terms of size max|F_s| / 2 and
    a |s| / 2, which cancel when the pressure or the momentum is nearly
    uniform across a face."""
    n, F = scale.shape
    hs = np.broadcast_to(np.asarray(h, dtype=np.float64), (n,))
    R = np.zeros((n, F))
    if faces is not None:
        fm = np.abs(faces).max(axis=(1, 3, 4))  # [n][F+3]
        R = fm[:, :F] / hs[:, None]
        mom = fm[:, list(MOMENTUM)].max(axis=1)
        for m, k in enumerate(SPIN):
            R[:, k] = np.maximum(np.maximum(R[:, k], fm[:, F + m] / hs), 0.5 * mom)
    if U is not None and amax is not None:
        um = _per_sub(U)[:, :F]  # [n][F]
        R = np.maximum(R, np.asarray(amax)[:, None] * um / hs[:, None])
        smax = um[:, list(MOMENTUM)].max(axis=1)
        for k in SPIN:
            R[:, k] = np.maximum(R[:, k], 0.5 * np.asarray(amax) * smax)
    if U is not None:
        s2 = sum(U[:, k] ** 2 for k in MOMENTUM)
        p = (gamma - 1.0) * (U[:, EGAS] - 0.5 * s2 / U[:, RHO])
        pm = np.abs(p).reshape(n, -1).max(axis=1) / hs
        for k in MOMENTUM:
            R[:, k] = np.maximum(R[:, k], pm)
    return R / scale


# Budget constants of the mixed form (mixed_budget).
C_SENS = 8.0   # FP32 storage: the kernel rounds up to ~4 values per primitive
               # (s, 1/rho, their product, the conversion) where the measured
               # perturbation rounds one
C_ARITH = 8.0  # FP32 reconstruction and flux arithmetic: a few roundings per term
FLOOR32 = 4e-7 # ~7 EPS32: one FP32 rounding of the sub-grid's own largest value,
               # for rates that are neither sensitive nor a residual


def mixed_budget(ref: np.ndarray, pert: np.ndarray, faces: np.ndarray, h, U: np.ndarray | None = None,
                 amax: np.ndarray | None = None, gamma: float = 5.0 / 3.0) -> tuple[np.ndarray, np.ndarray]:
    """Per-sub-grid, per-field error budget [n][F] of the mixed-precision step
    against the oracle, in units of subgrid_scales(ref, h).

    ref: the oracle's rates; pert: the oracle's rates on the inputs rounded
    to FP32 (sens = their normalised difference: what FP32 storage of the
    primitives alone costs).  The FP32 reconstruction and flux arithmetic
    adds rounding of relative size ~EPS32 to every term of every point flux
    and point torque, which the FP64 divergence keeps: at most a few EPS32
    times the terms of the rate (R, flux_ratio; pass the padded states U
    and the oracle's amax to include the dissipation and pressure terms;
    gamma the adiabatic index of the states).  That term
    dominates where a rate is a small residual of large terms (near
    hydrostatic equilibrium, hot thin gas).
    Budget: C_SENS sens + C_ARITH EPS32 R + FLOOR32.  Returns (budget, sens)."""
    sc = subgrid_scales(ref, h)
    sens = _ratio(_per_sub(pert - ref), sc)
    R = flux_ratio(faces, np.where(sc > 0, sc, 1.0), h, U, amax, gamma)
    R = np.where(sc > 0, R, 0.0)
    budget = np.where(sc > 0, C_SENS * sens + C_ARITH * EPS32 * R + FLOOR32, 0.0)
    return budget, sens


def mixed_error(got: np.ndarray, ref: np.ndarray, h) -> np.ndarray:
    """Per-sub-grid, per-field error [n][F] in the units of mixed_budget (a
    field that is exactly zero in a sub-grid gives inf unless matched
    exactly, and 0 then)."""
    return _ratio(_per_sub(got - ref), subgrid_scales(ref, h))


def mixed_worst(got: np.ndarray, ref: np.ndarray, pert: np.ndarray, faces: np.ndarray, h,
                U: np.ndarray | None = None, amax: np.ndarray | None = None, gamma: float = 5.0 / 3.0) -> float:
    """Largest error / budget over sub-grids and fields (<= 1 passes; a field
    exactly zero in the oracle must be exactly zero in the result)."""
    budget, _ = mixed_budget(ref, pert, faces, h, U, amax, gamma)
    err = mixed_error(got, ref, h)
    exact = budget == 0.0
    r = np.where(exact, np.where(err > 0, np.inf, 0.0), err / np.where(exact, 1.0, budget))
    return float(r.max())
