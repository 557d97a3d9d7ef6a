"""Equilibrium pins for the whole oracle step (integrator + pulse noise) and
for the oracle's Metropolis Monte Carlo: the Langevin function of independent
spins (Sec. III.A's exact m_z) and, on a small lattice, agreement of the
pulse-noise dynamics with Metropolis (Sec. IV)."""
import json
import math
import os

import numpy as np
import pytest

import spin_inputs

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def langevin(xi):
    return 1.0 / math.tanh(xi) - 1.0 / xi


def test_langevin_printed_values():
    g = GOLDEN["langevin_examples"]
    for xi, v in zip(g["xi"], g["value"]):
        assert abs(langevin(xi) - v) < g["abs_tol"]


def _binned_mean(x, nbins=10):
    b = np.array_split(np.asarray(x), nbins)
    m = np.array([v.mean() for v in b])
    return m.mean(), m.std(ddof=1) / math.sqrt(nbins)


@pytest.mark.parametrize("precession", [1, 0])
def test_independent_spins_reach_langevin(orc, precession):
    """J = 0: every spin is a spin in a field; pulse-noise dynamics must
    sample <s_z> = L(H/T) up to a bias that is small for Lambda_N Delta t << 1
    (here 0.04).  A wrong noise variance (factor 2 in T) moves <s_z> by > 0.1."""
    n = 16
    H, T, lam = 1.0, 1.0, 0.1
    p = orc.Params(n, n, n, J=0.0, D=0.0, H=(0, 0, H), lam=lam, T=T, dt=0.1, R=2,
                   seed=31, precession=precession)
    s = spin_inputs.random_spins(n, n, n, seed=12)
    s, _ = orc.run(p, s, 400)                      # t = 40 ~ 8 relaxation times
    _, smp = orc.run(p, s, 2000, n0=400)           # t = 200
    m, err = _binned_mean(smp[:, 3])
    assert abs(m - langevin(H / T)) < max(5 * err, 0.01)


def test_metropolis_independent_spins_reach_langevin(orc):
    """Metropolis with the paper's trial move samples the Boltzmann weight:
    independent spins give <s_z> = L(H/T); the acceptance rate with
    R = 1.55 sqrt(T/6J) (here at J = 1 scale) is about 50%."""
    n = 16
    H, T = 1.0, 0.5
    p = orc.Params(n, n, n, J=0.0, D=0.0, H=(0, 0, H), T=T)
    s = spin_inputs.random_spins(n, n, n, seed=13)
    s, _, _ = orc.metropolis(p, s, 60, mc_seed=5, R_trial=1.55 * math.sqrt(T / 6.0))
    s, ser, acc = orc.metropolis(p, s, 300, mc_seed=5, R_trial=1.55 * math.sqrt(T / 6.0), sweep0=60)
    m, err = _binned_mean(ser[:, 2])
    assert abs(m - langevin(H / T)) < max(5 * err, 0.004)


def test_metropolis_acceptance_near_half(orc):
    """Sec. IV: R = 1.55 sqrt(T/(6J)) gives about 50% acceptance on the
    Heisenberg lattice over a wide temperature range."""
    g = GOLDEN["mc_trial_length"]
    n = 8
    for T in (0.5, 1.0):
        p = orc.Params(n, n, n, J=1.0, T=T)
        s = spin_inputs.random_spins(n, n, n, seed=14)
        s, _, _ = orc.metropolis(p, s, 100, mc_seed=6)
        _, _, acc = orc.metropolis(p, s, 100, mc_seed=6, sweep0=100)
        rate = acc / (100 * p.N)
        assert abs(rate - g["acceptance"]) < g["acceptance_tol"], (T, rate)


def test_lattice_pulse_noise_matches_metropolis(orc):
    """Heisenberg ferromagnet 6^3 at T = 1 < T_c: the slow (precession-free)
    pulse-noise equation at the paper's working ratio (lambda dt = 0.04,
    lambda Delta t = 0.08, Sec. IV) samples the same <|M|> and <E> as
    Metropolis within statistical error plus a small pulse bias."""
    n = 6
    T = 1.0
    p = orc.Params(n, n, n, J=1.0, D=0.0, H=(0, 0, 0), lam=1.0, T=T, dt=0.04, R=2,
                   seed=41, precession=0)
    s0 = spin_inputs.aligned_spins(n, n, n)
    s, _ = orc.run(p, s0, 500)
    _, smp = orc.run(p, s, 20000, n0=500)
    Mabs = np.linalg.norm(smp[:, 1:4], axis=1)
    m_ld, e_m_ld = _binned_mean(Mabs, 20)
    E_ld, e_E_ld = _binned_mean(smp[:, 4], 20)

    q = orc.Params(n, n, n, J=1.0, T=T)
    s, _, _ = orc.metropolis(q, s0, 300, mc_seed=7)
    _, ser, _ = orc.metropolis(q, s, 6000, mc_seed=7, sweep0=300)
    m_mc, e_m_mc = _binned_mean(np.linalg.norm(ser[:, :3], axis=1), 20)
    E_mc, e_E_mc = _binned_mean(ser[:, 3], 20)
    assert abs(m_ld - m_mc) < 5 * math.hypot(e_m_ld, e_m_mc) + 0.02, (m_ld, m_mc, e_m_ld, e_m_mc)
    assert abs(E_ld - E_mc) < 5 * math.hypot(e_E_ld, e_E_mc) + 0.02, (E_ld, E_mc, e_E_ld, e_E_mc)
