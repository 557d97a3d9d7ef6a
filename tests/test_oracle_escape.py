"""Pins for oracle/escape.py, the closed forms and quadratures of the
single-spin problems of Sec. III (spin in a field, Fig. 4; escape of a
uniaxial spin in a transverse field, Sec. III.B and Fig. 6).  Each function is
checked against something other than itself: the paper's printed value,
limits, a brute-force Boltzmann or area integral, and the C oracle's own
dynamics and energy."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import escape as es


def test_langevin_function_is_the_boltzmann_average():
    for xi in [1e-3, 0.1, 1.0, 3.0, 10.0]:
        num = integrate.quad(lambda c: c * math.exp(xi * (c - 1.0)), -1.0, 1.0, epsabs=1e-15)[0]
        den = integrate.quad(lambda c: math.exp(xi * (c - 1.0)), -1.0, 1.0, epsabs=1e-15)[0]
        assert es.langevin_mz(xi, 1.0) == pytest.approx(num / den, rel=1e-10, abs=1e-14)
        assert es.langevin_mz(2.0 * xi, 2.0) == pytest.approx(num / den, rel=1e-12)  # depends on H/T only


def test_F_reduced_printed_value_and_closed_form_at_half():
    """At h = 1/2, x_c = 1 and the integrand of the reduced integral becomes
    u sqrt(1-u^2) + 1/sqrt(1-u^2), whose integral over [0, 1] is 1/3 + pi/2;
    the paper prints F(1/2) = 1.90."""
    F = es.F_ld_reduced(0.5)
    assert F == pytest.approx(1.0 / 3.0 + math.pi / 2.0, abs=1e-12)
    assert round(F, 2) == 1.90


@pytest.mark.parametrize("fn", ["F_ld_reduced", "F_ld_separatrix"])
def test_F_small_h_limit(fn):
    """F(h) -> 8 sqrt(h) for h << 1 (Sec. III.B)."""
    f = getattr(es, fn)
    for h, tol in [(1e-4, 5e-3), (1e-6, 5e-4), (1e-8, 5e-5)]:
        assert f(h) / (8.0 * math.sqrt(h)) == pytest.approx(1.0, abs=tol)


def _lobe_flux(h):
    """Stokes' theorem on the sphere: the circulation of F's definition equals
    the flux through the lobe {s_z > 0, f >= 2h} of the spherical Laplacian
    of f = s_z^2 + 2h s_x, which is 2 - 6 s_z^2 - 4h s_x.  In polar angles
    (theta from z, phi from x) the phi-integral over |phi| <= phi_0(theta) is
    done by hand; the theta integral by quadrature."""

    def ring(th):
        st, ct = math.sin(th), math.cos(th)
        if st == 0.0:
            return 0.0
        c = (2.0 * h - ct * ct) / (2.0 * h * st)
        if c >= 1.0:
            return 0.0
        phi0 = math.pi if c <= -1.0 else math.acos(c)
        return ((2.0 - 6.0 * ct * ct) * 2.0 * phi0 - 8.0 * h * st * math.sin(phi0)) * st

    # split at the polar angle of x_c, where the phi range reaches +-pi
    th_c = math.acos(2.0 * math.sqrt(h * (1.0 - h))) if h < 0.5 else 0.0
    pts = [p for p in (th_c,) if 0.0 < p < 0.5 * math.pi]
    v = integrate.quad(ring, 0.0, 0.5 * math.pi, points=pts or None, limit=400, epsabs=1e-13)[0]
    return abs(v) / 2.0


@pytest.mark.parametrize("h", [0.05, 0.2, 0.35, 0.5, 0.8])
def test_F_separatrix_equals_lobe_flux(h):
    assert es.F_ld_separatrix(h) == pytest.approx(_lobe_flux(h), rel=1e-7)


@pytest.mark.parametrize("h", [0.05, 0.2, 0.5, 0.8, 0.95])
def test_F_separatrix_polynomial_form(h):
    """Observed (fitted, then confirmed at these points to 1e-12):
    F = (8/3) sqrt(h(1-h)) (1-h) (3-2h), whose h -> 0 limit is 8 sqrt(h)."""
    assert es.F_ld_separatrix(h) == pytest.approx(8.0 / 3.0 * math.sqrt(h * (1 - h)) * (1 - h) * (3 - 2 * h),
                                                  abs=1e-10)


def _one_spin(orc, D, H, lam, dt, integrator=1):
    return orc.Params(1, 1, 1, J=0.0, D=D, H=(H, 0.0, 0.0), lam=lam, T=0.0, dt=dt, R=10 ** 6,
                      integrator=integrator)


def test_F_separatrix_is_half_the_dissipation_per_revolution(orc):
    """Physical meaning of the contour integral: started just inside the
    lobe at h = 1/2 (the pole lies on the separatrix there), the C oracle's
    noiseless LLG with small lambda loses 2 lambda D F_separatrix(1/2)
    of energy per revolution."""
    D, h, lam, dt = 1.0, 0.5, 3e-5, 0.01
    p = _one_spin(orc, D, 2 * h * D, lam, dt)
    d = 1e-6
    s = np.array([d, 0.0, math.sqrt(1 - d * d)]).reshape(3, 1, 1, 1)
    crossings, prev = [], s.copy()
    for n in range(4000):
        s, _ = orc.run(p, s, 1, n0=n, noise=False)
        if prev[1].item() < 0.0 <= s[1].item() and s[2].item() > 0.5:
            w = -prev[1].item() / (s[1].item() - prev[1].item())
            crossings.append((1 - w) * es.energy(D, 2 * h * D, prev.reshape(3))
                             + w * es.energy(D, 2 * h * D, s.reshape(3)))
        prev = s.copy()
    assert len(crossings) >= 3
    dE = np.diff(crossings)
    assert np.all(dE < 0)
    assert -dE[1] / (lam * D) == pytest.approx(2.0 * es.F_ld_separatrix(h), rel=5e-3)


def test_barrier_and_stationary_points(orc):
    """E(saddle) - E(well) = D (1-h)^2 with the C oracle's energy; the well
    bottom and the saddle (1, 0, 0) are stationary (H_eff parallel to s)."""
    for D, h in [(1.0, 0.5), (0.7, 0.2), (2.0, 0.8)]:
        p = orc.Params(1, 1, 1, J=0.0, D=D, H=(2 * h * D, 0.0, 0.0))
        well = np.array(es.well_state(h)).reshape(3, 1, 1, 1)
        saddle = np.array([1.0, 0.0, 0.0]).reshape(3, 1, 1, 1)
        Ew, Es = orc.observables(p, well)[3], orc.observables(p, saddle)[3]
        assert Es - Ew == pytest.approx(es.barrier(D, h), abs=1e-14)
        for st in (well, saddle):
            Hf = orc.heff(p, st).reshape(3)
            assert np.linalg.norm(np.cross(st.reshape(3), Hf)) < 1e-14


def test_fmr_frequency_from_small_oscillations(orc):
    """omega_0 = 2 D sqrt(1-h^2): the period of small precession about the
    well bottom in the C oracle's noiseless, undamped dynamics."""
    for D, h in [(1.0, 0.5), (0.6, 0.3)]:
        dt = 0.005
        p = _one_spin(orc, D, 2 * h * D, 0.0, dt)
        w = np.array(es.well_state(h))
        s = w + np.array([0.0, 1e-4, 0.0])
        s = (s / np.linalg.norm(s)).reshape(3, 1, 1, 1)
        ups, prev = [], s[1].item()
        for n in range(int(3.5 * 2 * math.pi / es.fmr_frequency(D, h) / dt)):
            s, _ = orc.run(p, s, 1, n0=n, noise=False)
            y = s[1].item()
            if prev < 0.0 <= y:
                ups.append((n + prev / (prev - y)) * dt)
            prev = y
        period = np.mean(np.diff(ups))
        assert 2 * math.pi / period == pytest.approx(es.fmr_frequency(D, h), rel=1e-6)


def test_escape_rate_regimes():
    D, h, T = 1.0, 0.5, 0.05
    F = es.F_ld_reduced(h)
    base = es.fmr_frequency(D, h) / (2 * math.pi) * math.exp(-D * (1 - h) ** 2 / T)
    assert es.escape_rate(T, D, h, 0.01, "ID") == pytest.approx(base, rel=1e-14)
    assert es.escape_rate(T, D, h, 0.01, "LD") == pytest.approx(base * 0.01 * (D / T) * F, rel=1e-14)
    # the interpolation tends to LD for small A and to ID for large A
    assert es.escape_rate(T, D, h, 1e-7, "ILD") / es.escape_rate(T, D, h, 1e-7, "LD") == pytest.approx(1, abs=1e-5)
    assert es.escape_rate(T, D, h, 1e5, "ILD") / es.escape_rate(T, D, h, 1e5, "ID") == pytest.approx(1, abs=1e-5)
    # Arrhenius: d ln(Gamma_ID)/d(1/T) = -Delta U
    g1, g2 = es.escape_rate(0.05, D, h, 0.1, "ID"), es.escape_rate(0.04, D, h, 0.1, "ID")
    assert math.log(g2 / g1) / (25.0 - 20.0) == pytest.approx(-es.barrier(D, h), rel=1e-12)
