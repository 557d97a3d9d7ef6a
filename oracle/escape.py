"""Closed-form and quadrature results of the single-spin problems of Sec. III
of arXiv:1610.04914: the spin in a field (Fig. 4) and the thermally activated
escape of a uniaxial spin in a transverse field (Sec. III.B, Fig. 6).

TEST INFRASTRUCTURE ONLY, like the rest of the ``oracle`` package: used by the
tests, never by the GPU library.  Units: gamma = mu_0 = 1 (as in the paper's
numerics), energy E = -D s_z^2 - H s_x, h = H/(2D) < 1, sigma = D/T.

Two readings of the low-damping factor F(h) of Eq. (ALD) are provided,
because the paper's two statements of it do not agree away from h -> 0:
  * ``F_ld_reduced``: the one-dimensional integral over u that the paper
    obtains "after some algebra" and evaluates to 1.90 at h = 1/2 (used in
    its Fig. 6 caption);
  * ``F_ld_separatrix``: the paper's defining contour integral, half the
    circulation of (1-x^2) df/dx dphi - (1-x^2)^-1 df/dphi dx along one lobe
    of the separatrix f = 2h, i.e. half the energy (in units of lambda D)
    that the damping removes during one revolution on the separatrix.
Both tend to 8 sqrt(h) for small h.  Parity: every function here is pinned
in tests/test_oracle_escape.py (closed forms, the paper's printed value,
brute-force area and trajectory integrals, the C oracle's own dynamics).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate


def langevin_mz(H: float, T: float) -> float:
    """Equilibrium <s_z> of a classical spin in a field H along z at
    temperature T (the exact curve that Fig. 4 compares with):
    coth(H/T) - T/H."""
    xi = H / T
    if xi < 1e-4:
        return xi / 3.0 - xi ** 3 / 45.0
    return 1.0 / math.tanh(xi) - 1.0 / xi


def barrier(D: float, h: float) -> float:
    """Energy barrier Delta U = D (1-h)^2 between a well bottom and the
    saddle s = (1, 0, 0) (Sec. III.B)."""
    return D * (1.0 - h) ** 2


def well_state(h: float):
    """Bottom of the well phi = 0, sin(theta) = h, s_z > 0 (Sec. III.B)."""
    return (h, 0.0, math.sqrt(1.0 - h * h))


def fmr_frequency(D: float, h: float) -> float:
    """omega_0 = 2 D sqrt(1 - h^2): precession frequency at the well bottom
    (Sec. III.B, below Eq. (GammaEsc))."""
    return 2.0 * D * math.sqrt(1.0 - h * h)


def F_ld_reduced(h: float) -> float:
    """The paper's reduced integral for F(h) over u in [0, 1], with
    x_c = 2 sqrt(h(1-h)) the largest x = cos(theta) on the separatrix."""
    xc = 2.0 * math.sqrt(h * (1.0 - h))

    def integrand(u):
        w = math.sqrt(1.0 - u * u)
        return xc / (1.0 - xc * xc * u * u) * (u * (2.0 * (1.0 - h) - xc * xc * u * u) ** 2 / w + xc * w)

    # u = sin(t) removes the 1/sqrt(1-u^2) end-point singularity
    val, _ = integrate.quad(lambda t: integrand(math.sin(t)) * math.cos(t), 0.0, 0.5 * math.pi, limit=400,
                            epsabs=1e-14, epsrel=1e-13)
    return val


def F_ld_separatrix(h: float) -> float:
    """The defining contour integral of F(h): (1/2) of the circulation along
    one lobe of f(x, phi) = x^2 + 2h sqrt(1-x^2) cos(phi) = 2h.  The lobe is
    symmetric under phi -> -phi, so (1/2) of the loop is the integral over
    its upper half, parametrised by x in (0, x_c) with
    cos(phi(x)) = (2h - x^2) / (2h sqrt(1-x^2)) and dphi/dx = -f_x / f_phi."""
    xc = 2.0 * math.sqrt(h * (1.0 - h))

    def integrand(x):
        u = math.sqrt(1.0 - x * x)
        c = min(1.0, max(-1.0, (2.0 * h - x * x) / (2.0 * h * u)))
        sphi = math.sqrt(max(0.0, 1.0 - c * c))
        fx = 2.0 * x - 2.0 * h * x * c / u
        fphi = -2.0 * h * u * sphi
        dphi_dx = -fx / fphi
        return (1.0 - x * x) * fx * dphi_dx - fphi / (1.0 - x * x)

    # x = x_c sin(t): both ends of the half loop are square-root turning points
    val, _ = integrate.quad(lambda t: integrand(xc * math.sin(t)) * xc * math.cos(t), 1e-12, 0.5 * math.pi - 1e-12,
                            limit=400, epsabs=1e-13, epsrel=1e-12)
    return val


def escape_prefactor(regime: str, lam: float, T: float, D: float, F: float) -> float:
    """Damping factor A of Eq. (GammaEsc): 'ID' -> 1 (transition-state
    theory), 'LD' -> lambda sigma F (Eq. (ALD)), 'ILD' -> A_LD/(1 + A_LD)
    (Eq. (AILD_interpolation))."""
    ald = lam * (D / T) * F
    if regime == "ID":
        return 1.0
    if regime == "LD":
        return ald
    if regime == "ILD":
        return ald / (1.0 + ald)
    raise ValueError(regime)


def escape_rate(T: float, D: float, h: float, lam: float, regime: str, F: float | None = None) -> float:
    """Gamma = (omega_0 / 2 pi) A exp(-sigma (1-h)^2), Eq. (GammaEsc); F
    defaults to the paper's F_ld_reduced(h)."""
    if F is None:
        F = F_ld_reduced(h)
    A = escape_prefactor(regime, lam, T, D, F)
    return fmr_frequency(D, h) / (2.0 * math.pi) * A * math.exp(-barrier(D, h) / T)


def energy(D: float, H: float, s) -> float:
    """E = -D s_z^2 - H s_x of one spin."""
    s = np.asarray(s, dtype=np.float64)
    return -D * s[2] ** 2 - H * s[0]
