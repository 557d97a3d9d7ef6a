"""Pins for the oracle's rectangular noise, Eq. (zeta_n): a random field
zeta_n = sqrt(2 lambda T / Delta t) G_n added to H_eff in the precession term
of Eq. (LLL) and held over each noise interval of length Delta t = R dt."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import spin_inputs
from oracle import escape as es


def test_zero_field_interval_is_an_exact_rotation(orc):
    """With H_eff = 0 the equation is ds/dt = s x zeta, a rotation about
    -zeta by |zeta| Delta t over one interval; each site of a J = 0 lattice
    turns about its own field, interval after interval (k = 0, 1, 2)."""
    p = orc.Params(3, 1, 1, J=0.0, D=0.0, H=(0, 0, 0), lam=0.05, T=0.8, dt=0.01, R=50,
                   integrator=orc.RK5_BUTCHER, seed=7, replica=3)
    s = spin_inputs.random_spins(3, 1, 1, seed=2)
    want = s.reshape(3, 3).T.copy()
    Dt = p.R * p.dt
    for k in range(3):
        s, _ = orc.run(p, s, p.R, n0=k * p.R, noise=2)
        z = orc.rect_field(p, k).reshape(3, 3).T
        for i in range(3):
            want[i] = Rotation.from_rotvec(-z[i] * Dt).apply(want[i])
        assert np.max(np.abs(s.reshape(3, 3).T - want)) < 1e-12


def test_rect_field_scale_and_sum_rule(orc):
    """zeta_i = sqrt(2 lambda T / Delta t) G(seed, i, k, replica): the same
    Gaussian triple as pulse k; Delta t <zeta_a zeta_b> = 2 lambda T delta_ab
    (the sum rule that fixes the coefficient)."""
    lam, T, dt, R = 0.03, 0.7, 0.1, 4
    p = orc.Params(8, 8, 8, J=0.0, lam=lam, T=T, dt=dt, R=R, seed=11, replica=2)
    Dt = R * dt
    z = orc.rect_field(p, 5)
    g = orc.noise_gauss(11, 3 + 8 * (2 + 8 * 1), 5, 2)  # site (x=3, y=2, z=1)
    assert np.allclose(z[:, 1, 2, 3], math.sqrt(2 * lam * T / Dt) * g, rtol=0, atol=1e-15)
    zs = np.concatenate([orc.rect_field(p, k).reshape(3, -1) for k in range(20)], axis=1)
    C = Dt * (zs @ zs.T) / zs.shape[1]
    assert np.allclose(C, 2 * lam * T * np.eye(3), atol=2 * lam * T * 0.03)


def test_noise_constant_within_an_interval(orc):
    """A call that starts mid-interval uses that interval's field: two calls
    of 3 + 5 steps equal one call of 8 (R = 4)."""
    p = orc.Params(2, 2, 1, J=0.4, D=0.2, H=(0.1, 0, 0.5), lam=0.1, T=1.0, dt=0.05, R=4,
                   integrator=orc.HEUN, seed=5)
    s0 = spin_inputs.random_spins(2, 2, 1, seed=9)
    a, _ = orc.run(p, s0, 8, noise=2)
    b, _ = orc.run(p, s0, 3, noise=2)
    b, _ = orc.run(p, b, 5, n0=3, noise=2)
    assert np.array_equal(a, b)


def test_rect_needs_precession(orc):
    p = orc.Params(1, 1, 1, precession=0)
    with pytest.raises(ValueError):
        orc.run(p, np.array([0, 0, 1.0]).reshape(3, 1, 1, 1), 2, noise=2)


def test_rect_equilibrium_is_the_langevin_function(orc):
    """Independent spins (J = 0 lattice) in H = 1 along z under rectangular
    noise with a short interval (Delta t = delta t = 0.05, lambda = 0.1,
    T = 1, Heun): <s_z> -> coth(1) - 1 (the Boltzmann value; standard error
    0.004 over 64 spins x 6000 time units after 100 of relaxation, relaxation
    time ~10)."""
    n = 4
    p = orc.Params(n, n, n, J=0.0, D=0.0, H=(0, 0, 1.0), lam=0.1, T=1.0, dt=0.05, R=1,
                   integrator=orc.HEUN, seed=23)
    s = spin_inputs.aligned_spins(n, n, n, (0, 0, 1.0))
    s, _ = orc.run(p, s, 2000, noise=2)
    acc, cnt = 0.0, 0
    for k in range(240):
        s, _ = orc.run(p, s, 500, n0=2000 + 500 * k, noise=2)
        acc += s[2].mean()
        cnt += 1
    assert acc / cnt == pytest.approx(es.langevin_mz(1.0, 1.0), abs=0.015)
