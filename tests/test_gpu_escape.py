"""Single-spin physics of Sec. III on the GPU kernels, against the oracle's
closed forms (oracle/escape.py):
  * escape of a uniaxial spin in a transverse field (Sec. III.B, Fig. 6):
    h = 1/2, D = 1, spins start at the well bottom, Butcher's RK5, first
    passage = first step that leaves s_z < 0; the rate is the number of
    passages per unit time of the renewal runs (unfinished trials included);
  * the accuracy statements about the parameter sets (delta t, Delta t);
  * the spin in a field H = 1 (Fig. 4): <s_z> against the Langevin function
    and the sign and growth of its deviation with Delta t.
Tolerances are statistical (standard errors quoted in each test) plus the
asymptotic accuracy of the rate formulas at these barriers (Delta U/T = 3-6),
with the measured values recorded beside each assertion."""
import math

import numpy as np
import pytest
import torch

from oracle import escape as es

pytestmark = pytest.mark.gpu

D, HX, H_RED = 1.0, 1.0, 0.5
REF_POINTS = [(0.0003, 20), (0.001, 25), (0.001, 12), (0.003, 12), (0.01, 15), (0.01, 12), (0.03, 15), (0.03, 12),
              (0.1, 20), (0.1, 15)]


def _rates(gpu, points, dt, R, t_budget, nper=8192, seed=1, prec=32):
    T, L, groups = [], [], []
    for lam, inv_t in points:
        groups.append(list(range(len(T), len(T) + nper)))
        T += [1.0 / inv_t] * nper
        L += [lam] * nper
    p = gpu.Params(1, 1, 1, J=0.0, D=D, H=(HX, 0.0, 0.0), lam=0.0, T=0.0, dt=dt, R=R,
                   integrator=gpu.RK5_BUTCHER, precession=1, seed=seed, precision=prec)
    e = gpu.EscapeReplicas(p, T, es.well_state(H_RED), lam=L)
    left = int(round(t_budget / dt))
    while left > 0:
        c = min(left, 400000)
        e.run(c)
        left -= c
    return {pt: (r[3], r[2]) for pt, r in zip(points, e.mfpt(groups))}


@pytest.fixture(scope="module")
def ref(gpu):
    """The paper's reference set delta t = 1/6, Delta t = 1."""
    return _rates(gpu, REF_POINTS, 1.0 / 6.0, 6, 4e5)


def _base(inv_t):
    return es.fmr_frequency(D, H_RED) / (2 * math.pi) * math.exp(-es.barrier(D, H_RED) * inv_t)


def _F_eff(rate, lam, inv_t):
    """F that makes the interpolation A_LD/(1+A_LD) reproduce the rate."""
    A = rate / _base(inv_t)
    return A / (1.0 - A) / (lam * D * inv_t)


def test_low_damping_follows_LD_with_printed_F(ref):
    """lambda = 0.0003 and 0.001 (energy-diffusion regime): the measured
    prefactor gives F within 5% of the paper's 1.90 (measured 1.91 and
    1.87, statistical error < 0.5%), and far from the separatrix
    circulation 4/3 of F's contour definition."""
    Fr, Fs = es.F_ld_reduced(H_RED), es.F_ld_separatrix(H_RED)
    for pt in [(0.0003, 20), (0.001, 25)]:
        rate, n = ref[pt]
        assert n > 20000, (pt, n)
        F = _F_eff(rate, *pt)
        assert abs(F / Fr - 1.0) < 0.05, (pt, F)
        assert abs(F - Fr) < abs(F - Fs)


def test_crossover_damping_follows_interpolation(ref):
    """lambda = 0.01: the ILD interpolation with F = 1.90 within -20%..+10%
    (measured 0.90 and 0.93 of it at 1/T = 15, 12)."""
    for pt in [(0.01, 15), (0.01, 12)]:
        rate, _ = ref[pt]
        g = es.escape_rate(1.0 / pt[1], D, H_RED, pt[0], "ILD")
        assert 0.8 < rate / g < 1.1, (pt, rate / g)


def test_moderate_damping_approaches_transition_state(ref):
    """lambda = 0.1: below the transition-state rate A = 1 and approaching
    it as the barrier grows (measured 0.81 at 1/T = 15, 0.89 at 20)."""
    r15 = ref[(0.1, 15)][0] / es.escape_rate(1 / 15, D, H_RED, 0.1, "ID")
    r20 = ref[(0.1, 20)][0] / es.escape_rate(1 / 20, D, H_RED, 0.1, "ID")
    assert 0.7 < r15 < r20 < 1.0, (r15, r20)


def test_rates_order_with_damping(ref):
    """At fixed T the rate grows with lambda through LD and ILD."""
    for inv_t in (12, 15):
        lams = sorted(l for l, t in REF_POINTS if t == inv_t)
        rates = [ref[(l, inv_t)][0] for l in lams]
        assert all(a < b for a, b in zip(rates, rates[1:])), (inv_t, rates)


def test_parameter_sets(gpu, ref):
    """Sec. III.B: delta t = 0.2, Delta t = 2 gives the reference result
    for lambda = 0.01 and 0.03 (measured within 0.6%); Delta t = 4 gives
    rates that are too high (measured +14% for lambda = 0.03 and +2.7% for
    0.01 at 1/T = 15); for lambda = 0.001 and 0.003, delta t = 0.25,
    Delta t = 4 is accurate (measured within 1%)."""
    pts = [(0.01, 15), (0.01, 12), (0.03, 15), (0.03, 12)]
    s2 = _rates(gpu, pts, 0.2, 10, 6e4, seed=2)
    for pt in pts:
        assert abs(s2[pt][0] / ref[pt][0] - 1.0) < 0.03, (pt, s2[pt][0] / ref[pt][0])
    s4 = _rates(gpu, [(0.01, 15), (0.03, 15)], 0.2, 20, 6e4, seed=3)
    assert s4[(0.03, 15)][0] / ref[(0.03, 15)][0] > 1.08
    assert s4[(0.01, 15)][0] / ref[(0.01, 15)][0] > 1.012  # ratio error ~0.15%
    low = _rates(gpu, [(0.001, 12), (0.003, 12)], 0.25, 16, 6e4, seed=4)
    for pt in [(0.001, 12), (0.003, 12)]:
        assert abs(low[pt][0] / ref[pt][0] - 1.0) < 0.03, (pt, low[pt][0] / ref[pt][0])


def _mz(gpu, T, Dt, dt=0.25, nper=16384, t_therm=2000.0, t_avg=20000.0, seed=9):
    R = int(round(Dt / dt))
    R += R % 2
    p = gpu.Params(1, 1, 1, J=0.0, D=0.0, H=(0.0, 0.0, 1.0), lam=0.01, T=T, dt=Dt / R, R=R,
                   integrator=gpu.RK5_BUTCHER, precession=1, seed=seed, precision=32)
    s0 = torch.zeros(3, nper, dtype=torch.float64)
    s0[2] = 1.0
    s = gpu.SingleSpins(p, [T] * nper, s0)
    s.run(int(t_therm / Dt) * R)
    s.run(int(t_avg / Dt) * R, average=True)
    torch.cuda.synchronize()
    per = (s.sz_sum / s.sz_count.double()).cpu().numpy()
    return float(per.mean()) - es.langevin_mz(1.0, T), float(per.std() / math.sqrt(nper))


def test_spin_in_field_bias_vs_delta_t(gpu):
    """Fig. 4 (H = 1, lambda = 0.01): at Lambda_N Delta t = 0.02 <s_z> is
    the Langevin function within statistics; at Lambda_N Delta t = 0.1 the
    deviation is below 0.005 and negative at T = 1 (measured -0.0026 +-
    0.0003), positive at T = 0.1 (measured +0.0022 +- 0.00006), and at
    T = 1 it grows with Delta t."""
    d1, e1 = _mz(gpu, 1.0, 1.0)
    d5, e5 = _mz(gpu, 1.0, 5.0)
    assert abs(d1) < 4 * e1 + 5e-4, (d1, e1)
    assert -0.005 < d5 < -3 * e5, (d5, e5)
    assert d5 < d1 - 3 * math.hypot(e1, e5)
    c10, f10 = _mz(gpu, 0.1, 10.0)
    c50, f50 = _mz(gpu, 0.1, 50.0)
    assert abs(c10) < 4 * f10 + 2e-4, (c10, f10)
    assert 3 * f50 < c50 < 0.005, (c50, f50)
