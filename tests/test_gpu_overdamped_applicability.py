"""The pulse condition of Sec. III.A on the slow (overdamped) workload: the
256^3 workload's settings (lambda = 1, T = 1.2, dt = 0.2, Delta t = 1.0, so
Lambda_N Delta t = 2.4, phi_RMS = 1.55) against the paper's working setting
(lambda dt = 0.04, lambda Delta t = 0.08; Lambda_N Delta t = 0.19) and half of
it, compared like with like against the GPU Metropolis on the same 32^3
lattice (J = 1, H = 0.01 along z).

Measured (Metropolis <|M|> 0.568, E -1.545 at 32^3 and at 256^3):

    Lambda_N Delta t   <|M|> 32^3 / 256^3   E
    2.4                0.027 / 0.013        -1.747
    0.19               0.548 / 0.544        -1.500
    0.096              0.562 / 0.559        -1.525

At 2.4 the kicks destroy the long-range order (|M| near its finite-size
floor) while the relaxation between them keeps the local order; in the valid
settings the bias is "hotter" and shrinks with Lambda_N Delta t."""
import math

import numpy as np
import pytest
import torch

import spin_inputs

pytestmark = pytest.mark.gpu

L = 32
T = 1.2
PHYS = dict(J=1.0, D=0.0, H=(0.0, 0.0, 0.01))


def _binned(x, nb=10):
    b = np.array_split(np.asarray(x), nb)
    m = np.array([v.mean() for v in b])
    return m.mean(), m.std(ddof=1) / math.sqrt(nb)


def _slow_equation(gpu, dt, R, t_eq=100.0, t_meas=500.0):
    p = gpu.Params(L, L, L, lam=1.0, T=T, dt=dt, R=R, integrator=gpu.RK4, precision=32, seed=3, precession=0,
                   **PHYS)
    lat = gpu.Lattice(p, torch.from_numpy(spin_inputs.aligned_spins(L, L, L)))
    chunk = 400 * R                        # the sample ring holds 512 records
    n = int(round(t_eq / dt))
    while n > 0:
        lat.step(min(chunk, n))
        lat.samples()
        n -= chunk
    recs, n = [], int(round(t_meas / dt))
    while n > 0:
        lat.step(min(chunk, n))
        recs.append(np.array(lat.samples()))
        n -= chunk
    lat.close()
    rec = np.concatenate(recs)
    return _binned(np.linalg.norm(rec[:, 1:4], axis=1)), _binned(rec[:, 4])


def _metropolis(gpu):
    p = gpu.Params(L, L, L, T=T, precision=32, **PHYS)
    lat = gpu.Lattice(p, torch.from_numpy(spin_inputs.aligned_spins(L, L, L)))
    gpu.spin_metropolis_sweeps(p, lat.state, 2000, mc_seed=9)
    m, e = [], []
    for k in range(800):
        gpu.spin_metropolis_sweeps(p, lat.state, 5, mc_seed=9, sweep0=2000 + 5 * k)
        M, E = lat.observables()
        m.append(float(np.linalg.norm(M)))
        e.append(E)
    lat.close()
    return _binned(m), _binned(e)


def test_pulse_condition_on_the_slow_workload(gpu):
    (m_mc, em_mc), (E_mc, eE_mc) = _metropolis(gpu)
    (m_bad, _), (E_bad, _) = _slow_equation(gpu, 0.2, 5)      # Lambda_N Delta t = 2.4
    (m_ok, em_ok), (E_ok, eE_ok) = _slow_equation(gpu, 0.04, 2)    # 0.19
    (m_half, em_half), (E_half, eE_half) = _slow_equation(gpu, 0.02, 2)  # 0.096
    assert m_mc > 0.5, m_mc
    assert m_bad < 0.1, (m_bad, m_mc)                          # long-range order destroyed
    # hotter than Boltzmann, by less at the smaller Delta t
    assert 0 < m_mc - m_ok < 0.04 and 0 < E_ok - E_mc < 0.08, (m_ok, E_ok, m_mc, E_mc)
    assert abs(m_half - m_mc) < 0.015 and 0 < E_half - E_mc < 0.04, (m_half, E_half, m_mc, E_mc)
    assert (m_mc - m_half) < (m_mc - m_ok) - 3 * math.hypot(em_ok, em_half), (m_ok, m_half)
    assert (E_half - E_mc) < (E_ok - E_mc) - 3 * math.hypot(eE_ok, eE_half), (E_ok, E_half)
