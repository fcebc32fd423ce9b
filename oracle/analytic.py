"""Closed forms used to pin the oracle (test infrastructure only).

Each function states the mathematics it evaluates; none of them calls the
oracle's C code, so agreement between the two is evidence, not tautology.

* ``wall_profile_1d`` -- steady diffusion between a first-order reactive wall
  (Eq. reactionRateBoundary) and a Dirichlet plane: the exact linear profile
  that the wet-node reading of Eq. general_RBC reproduces to round-off.
* ``series_2d`` -- the Fourier series of Eq. analytical2Dverification with the
  eigenvalues of Eq. Analytical_PeDa and the norms N_n^2 (Sec. 3.1).
* ``annulus_rate`` -- steady radial diffusion from a Dirichlet circle to a
  reactive disk (wall-orientation invariance pin).
* ``poiseuille``, ``shear_wave_rate``, ``diffusion_wave_rate`` -- textbook
  solutions of the Navier-Stokes / advection-diffusion limits of Eqs.
  fluid_BGK / solute_BGK with nu = cs^2 (tau - 1/2), D = cs^2 (tau - 1/2).
"""
from __future__ import annotations

import math

import numpy as np


def wall_profile_1d(y, k_r: float, D: float, L: float, c_top: float, c_eq: float):
    """C(y) for D C'' = 0 on [0, L], D C'(0) = k_r (C(0) - c_eq), C(L) = c_top.

    The reaction flux J_R = k_r (c_eq - C_wall) of Eq. reactionRateBoundary
    enters the fluid at y = 0, so -D C'(0) = J_R.  Solution:
    C = c_eq + (c_top - c_eq) (1 + kappa y) / (1 + kappa L), kappa = k_r / D.
    """
    y = np.asarray(y, dtype=np.float64)
    if math.isinf(k_r):
        return c_eq + (c_top - c_eq) * y / L
    kap = k_r / D
    return c_eq + (c_top - c_eq) * (1.0 + kap * y) / (1.0 + kap * L)


def beta_roots(peda: float, b: float, n: int):
    """First n positive roots of (beta b) tan(beta b) = PeDa (Eq. Analytical_PeDa).

    The n-th root of t tan t = PeDa lies in ((n-1) pi, (n-1/2) pi); found by
    bisection on t tan t - PeDa, which is increasing there.
    """
    out = np.empty(n)
    for k in range(n):
        lo, hi = k * math.pi + 1e-15, k * math.pi + 0.5 * math.pi - 1e-15
        f = lambda t: t * math.tan(t) - peda
        flo = f(lo)
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            fm = f(mid)
            if (fm > 0) == (flo > 0):
                lo, flo = mid, fm
            else:
                hi = mid
        out[k] = 0.5 * (lo + hi) / b
    return out


def series_2d(x, y, a: float, b: float, peda: float, c0: float, c_eq: float, nterms: int = 100):
    """Eq. analytical2Dverification: C(x, y) on the rectangle [0,a] x [0,b]
    with C = c0 at x = 0, zero gradient at x = a and y = 0, and the reactive
    wall at y = b; sum truncated after ``nterms`` terms as in Sec. 3.1."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    beta = beta_roots(peda, b, nterms)
    s = np.zeros(np.broadcast(x, y).shape)
    for bn in beta:
        n2 = 0.5 * b * (1.0 + math.sin(2.0 * bn * b) / (2.0 * bn * b))
        s = s + math.sin(bn * b) / (n2 * bn) * np.cosh(bn * (x - a)) / math.cosh(bn * a) * np.cos(bn * y)
    return (c0 - c_eq) * s + c_eq


def annulus_rate(R: float, R2: float, k_r: float, D: float, c_out: float, c_eq: float) -> float:
    """Total reaction rate (per unit depth) of a reactive disk of radius R
    inside a Dirichlet circle C(R2) = c_out: C = c_out + B ln(r/R2) with
    D C'(R) = k_r (C(R) - c_eq); rate = 2 pi D B."""
    B = k_r * (c_out - c_eq) / (D / R + k_r * math.log(R2 / R))
    return 2.0 * math.pi * D * B


def poiseuille(y, y0: float, y1: float, u_max: float):
    """Parabolic profile between walls at y0 and y1 with centre value u_max."""
    y = np.asarray(y, dtype=np.float64)
    h = 0.5 * (y1 - y0)
    yc = 0.5 * (y0 + y1)
    return u_max * (1.0 - ((y - yc) / h) ** 2)


def shear_wave_rate(nu: float, k: float) -> float:
    """Decay rate of a transverse shear wave u_x = U sin(k y): nu k^2."""
    return nu * k * k


def diffusion_wave_rate(D: float, k: float) -> float:
    """Decay rate of a concentration wave C = C0 + A sin(k x): D k^2."""
    return D * k * k
