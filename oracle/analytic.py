"""Analytic solutions the oracle is pinned to (test infrastructure only).

* ``riemann_exact``: the exact solution of the 1-D Riemann problem of an ideal
  gas (two-rarefaction / two-shock pressure function solved by Newton
  iteration, then sampled along x/t), written from the Rankine-Hugoniot and
  isentropic-rarefaction relations.
* ``sedov_xi0``: the Sedov-Taylor constant xi0 of R = xi0 (E t^2/rho)^(1/5)
  for a point blast in a uniform gas (spherical), from a numerical
  integration of the self-similar ODEs behind the strong shock and the energy
  integral.
"""
from __future__ import annotations

import math

import numpy as np


# ----------------------------------------------------------------------------
# exact Riemann solver
def _f_side(p, rho, pk, ck, gamma):
    """Velocity jump across the wave on one side and its derivative in p."""
    if p > pk:  # shock
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        sq = math.sqrt(A / (p + B))
        f = (p - pk) * sq
        df = sq * (1.0 - 0.5 * (p - pk) / (B + p))
    else:  # rarefaction
        pr = p / pk
        f = 2.0 * ck / (gamma - 1.0) * (pr ** ((gamma - 1.0) / (2.0 * gamma)) - 1.0)
        df = 1.0 / (rho * ck) * pr ** (-(gamma + 1.0) / (2.0 * gamma))
    return f, df


def riemann_star(rhoL, uL, pL, rhoR, uR, pR, gamma):
    """Star-region pressure and velocity."""
    cL = math.sqrt(gamma * pL / rhoL)
    cR = math.sqrt(gamma * pR / rhoR)
    p = max(1e-12, 0.5 * (pL + pR) - 0.125 * (uR - uL) * (rhoL + rhoR) * (cL + cR))
    for _ in range(200):
        fL, dL = _f_side(p, rhoL, pL, cL, gamma)
        fR, dR = _f_side(p, rhoR, pR, cR, gamma)
        pn = p - (fL + fR + uR - uL) / (dL + dR)
        pn = max(pn, 1e-14)
        if abs(pn - p) <= 1e-15 * (pn + p):
            p = pn
            break
        p = pn
    fL, _ = _f_side(p, rhoL, pL, cL, gamma)
    fR, _ = _f_side(p, rhoR, pR, cR, gamma)
    u = 0.5 * (uL + uR) + 0.5 * (fR - fL)
    return p, u


def riemann_exact(rhoL, uL, pL, rhoR, uR, pR, gamma, xi):
    """Sample (rho, u, p) at similarity coordinates xi = x/t (array)."""
    ps, us = riemann_star(rhoL, uL, pL, rhoR, uR, pR, gamma)
    cL = math.sqrt(gamma * pL / rhoL)
    cR = math.sqrt(gamma * pR / rhoR)
    gm = (gamma - 1.0) / (gamma + 1.0)
    xi = np.asarray(xi, dtype=np.float64)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    for i, s in np.ndenumerate(xi):
        if s <= us:  # left of the contact
            if ps > pL:  # left shock
                rs = rhoL * (ps / pL + gm) / (gm * ps / pL + 1.0)
                S = uL - cL * math.sqrt((gamma + 1.0) / (2 * gamma) * ps / pL + (gamma - 1.0) / (2 * gamma))
                st = (rhoL, uL, pL) if s <= S else (rs, us, ps)
            else:  # left rarefaction
                rs = rhoL * (ps / pL) ** (1.0 / gamma)
                cs = cL * (ps / pL) ** ((gamma - 1.0) / (2 * gamma))
                if s <= uL - cL:
                    st = (rhoL, uL, pL)
                elif s >= us - cs:
                    st = (rs, us, ps)
                else:
                    uu = 2.0 / (gamma + 1.0) * (cL + 0.5 * (gamma - 1.0) * uL + s)
                    cc = 2.0 / (gamma + 1.0) * (cL + 0.5 * (gamma - 1.0) * (uL - s))
                    rr = rhoL * (cc / cL) ** (2.0 / (gamma - 1.0))
                    st = (rr, uu, pL * (cc / cL) ** (2 * gamma / (gamma - 1.0)))
        else:  # right of the contact
            if ps > pR:  # right shock
                rs = rhoR * (ps / pR + gm) / (gm * ps / pR + 1.0)
                S = uR + cR * math.sqrt((gamma + 1.0) / (2 * gamma) * ps / pR + (gamma - 1.0) / (2 * gamma))
                st = (rhoR, uR, pR) if s >= S else (rs, us, ps)
            else:  # right rarefaction
                rs = rhoR * (ps / pR) ** (1.0 / gamma)
                cs = cR * (ps / pR) ** ((gamma - 1.0) / (2 * gamma))
                if s >= uR + cR:
                    st = (rhoR, uR, pR)
                elif s <= us + cs:
                    st = (rs, us, ps)
                else:
                    uu = 2.0 / (gamma + 1.0) * (-cR + 0.5 * (gamma - 1.0) * uR + s)
                    cc = 2.0 / (gamma + 1.0) * (cR - 0.5 * (gamma - 1.0) * (uR - s))
                    rr = rhoR * (cc / cR) ** (2.0 / (gamma - 1.0))
                    st = (rr, uu, pR * (cc / cR) ** (2 * gamma / (gamma - 1.0)))
        rho[i], u[i], p[i] = st
    return rho, u, p


# ----------------------------------------------------------------------------
# Sedov-Taylor similarity constant
def _sedov_rhs(lam_log, y, gamma):
    """d/d(ln lambda) of (V, ln G, ln Z) for v = (2r/5t)V, rho = rho0 G,
    c^2 = (4 r^2 / 25 t^2) Z, from mass, momentum and entropy conservation:
        (V-1) g + V'                      = -3V
        gamma (V-1) V' + Z g + Z zeta     = -gamma (V^2 - 5V/2) - 2Z
        (V-1) ((1-gamma) g + zeta)        = 5 - 2V
    with g = (ln G)', zeta = (ln Z)'."""
    V, lnG, lnZ = y
    Z = math.exp(lnZ)
    A = np.array([[V - 1.0, 1.0, 0.0],
                  [Z, gamma * (V - 1.0), Z],
                  [(V - 1.0) * (1.0 - gamma), 0.0, V - 1.0]])
    b = np.array([-3.0 * V, -gamma * (V * V - 2.5 * V) - 2.0 * Z, 5.0 - 2.0 * V])
    g, dV, zeta = np.linalg.solve(A, b)
    return [dV, g, zeta]


def sedov_profile(gamma: float, lam_min: float = 1e-5, n: int = 4000):
    """Self-similar profile behind the strong shock: lambda = r/R, and
    V(lambda), G = rho/rho0, Z, integrated inwards from the shock."""
    from scipy.integrate import solve_ivp

    V1 = 2.0 / (gamma + 1.0)
    G1 = (gamma + 1.0) / (gamma - 1.0)
    Z1 = 2.0 * gamma * (gamma - 1.0) / (gamma + 1.0) ** 2
    s_eval = np.linspace(0.0, math.log(lam_min), n)
    sol = solve_ivp(_sedov_rhs, (0.0, math.log(lam_min)), [V1, math.log(G1), math.log(Z1)], args=(gamma,),
                    t_eval=s_eval, rtol=1e-11, atol=1e-13, method="DOP853")
    lam = np.exp(sol.t)
    return lam, sol.y[0], np.exp(sol.y[1]), np.exp(sol.y[2])


def sedov_xi0(gamma: float) -> float:
    """xi0 with E = (16 pi / 25) xi0^5 * int_0^1 G lambda^4 (V^2/2 + Z/(gamma(gamma-1))) dlambda = 1."""
    lam, V, G, Z = sedov_profile(gamma)
    f = G * lam ** 4 * (0.5 * V * V + Z / (gamma * (gamma - 1.0)))
    # integrate in ln(lambda): d lambda = lambda d ln lambda (arrays run from lambda=1 inwards)
    s = np.log(lam)
    I = -np.trapezoid(f * lam, s)
    return (25.0 / (16.0 * math.pi * I)) ** 0.2


def sedov_radius(E: float, rho0: float, t: float, gamma: float) -> float:
    return sedov_xi0(gamma) * (E * t * t / rho0) ** 0.2
