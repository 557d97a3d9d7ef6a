"""Pins for the oracle's discrete adjoint (pathwise gradients with the noise
fixed): dot-product tests of each transposed primitive against central finite
differences of the forward map, and gradients of the full loss
L = dLdE E(s_n) + dLdM . M(s_n) against central finite differences of the
forward oracle."""
import numpy as np
import pytest

import spin_inputs


def _rand(shape, seed):
    return np.random.default_rng(seed).standard_normal((3, shape[2], shape[1], shape[0]))


@pytest.mark.parametrize("precession", [1, 0])
def test_rhs_vjp_dot_product(orc, precession):
    """<v, J_f(x) u> = <J_f(x)^T v, u>, J_f u by central differences of the
    right-hand side (a cubic polynomial, so the difference is exact to O(eps^2))."""
    shape = (4, 3, 5)
    p = orc.Params(*shape, J=0.8, D=0.35, H=(0.1, -0.2, 0.4), lam=0.3, precession=precession)
    x = spin_inputs.random_spins(*shape, seed=1) * 1.05
    hs = spin_inputs.site_fields(*shape, 0.2, seed=2)
    u, v = _rand(shape, 3), _rand(shape, 4)
    e = 1e-5
    Ju = (orc.rhs(p, x + e * u, hs) - orc.rhs(p, x - e * u, hs)) / (2 * e)
    JTv, gJ, gD, gH, gh = orc.rhs_vjp(p, x, v, hs)
    assert np.sum(v * Ju) == pytest.approx(np.sum(JTv * u), rel=1e-8)
    # parameter directions: <v, df/dtheta>
    for name, val, got in (("J", p.J, gJ), ("D", p.D, gD)):
        pp = orc.Params(**{**p.__dict__, name: val + e})
        pm = orc.Params(**{**p.__dict__, name: val - e})
        fd = np.sum(v * (orc.rhs(pp, x, hs) - orc.rhs(pm, x, hs))) / (2 * e)
        assert got == pytest.approx(fd, rel=1e-7)
    dh = _rand(shape, 5)
    fd = np.sum(v * (orc.rhs(p, x, hs + e * dh) - orc.rhs(p, x, hs - e * dh))) / (2 * e)
    assert np.sum(gh * dh) == pytest.approx(fd, rel=1e-7)
    assert np.allclose(gH, gh.reshape(3, -1).sum(axis=1), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("integrator", [0, 1, 2, 3])
@pytest.mark.parametrize("pulse", [False, True])
def test_step_vjp_dot_product(orc, integrator, pulse):
    """One full step (RK stages, renormalisation, pulse rotation): the adjoint
    map is the transpose of the step's Jacobian."""
    shape = (3, 4, 3)
    p = orc.Params(*shape, J=1.0, D=0.2, H=(0.05, 0.0, 0.3), lam=0.15, T=0.9, dt=0.1, R=4,
                   integrator=integrator, seed=8)
    s = spin_inputs.random_spins(*shape, seed=6)
    hs = spin_inputs.site_fields(*shape, 0.1, seed=7)
    u, lam = _rand(shape, 9), _rand(shape, 10)

    def step(x):
        y = orc.renormalise(p, orc.integrate(p, x, hs))
        return orc.pulse(p, y, 3) if pulse else y

    e = 1e-6
    Ju = (step(s + e * u) - step(s - e * u)) / (2 * e)
    back, *_ = orc.step_vjp(p, s, lam, pulse=pulse, k=3, h_site=hs)
    assert np.sum(lam * Ju) == pytest.approx(np.sum(back * u), rel=1e-7)


def _loss(orc, p, s0, n, dLdM, dLdE, hs):
    out, _ = orc.run(p, s0, n, h_site=hs)
    o = orc.observables(p, out, hs)
    return dLdE * o[3] + np.dot(dLdM, o[:3])


@pytest.mark.parametrize("integrator,precession", [(0, 1), (0, 0), (1, 1), (2, 0)])
def test_adjoint_matches_finite_differences(orc, integrator, precession):
    """Gradients of L = dLdE E + dLdM.M after 9 steps with pulses (R = 4)
    w.r.t. J, D, H, the per-site field and the initial spins, against central
    finite differences of the forward oracle (noise fixed)."""
    shape = (4, 3, 3)
    base = dict(J=0.9, D=0.25, H=(0.05, -0.1, 0.2), lam=0.1, T=0.8, dt=0.1, R=4, integrator=integrator,
                precession=precession, seed=12)
    p = orc.Params(*shape, **base)
    s0 = spin_inputs.random_spins(*shape, seed=11)
    hs = spin_inputs.site_fields(*shape, 0.1, seed=13)
    dLdM, dLdE, n = np.array([0.3, -0.2, 0.7]), 1.0, 9
    g = orc.adjoint(p, s0, n, dLdM, dLdE, h_site=hs)
    e = 1e-5

    def L(**kw):
        q = orc.Params(*shape, **{**base, **{k: v for k, v in kw.items() if k in base}})
        return _loss(orc, q, kw.get("s0", s0), n, dLdM, dLdE, kw.get("hs", hs))

    assert g["J"] == pytest.approx((L(J=base["J"] + e) - L(J=base["J"] - e)) / (2 * e), rel=1e-6)
    assert g["D"] == pytest.approx((L(D=base["D"] + e) - L(D=base["D"] - e)) / (2 * e), rel=1e-6)
    for a in range(3):
        Hp, Hm = list(base["H"]), list(base["H"])
        Hp[a] += e
        Hm[a] -= e
        assert g["H"][a] == pytest.approx((L(H=tuple(Hp)) - L(H=tuple(Hm))) / (2 * e), rel=1e-6, abs=1e-9)
    rng = np.random.default_rng(0)
    for _ in range(4):
        c, z, y, x = (int(rng.integers(0, m)) for m in (3, shape[2], shape[1], shape[0]))
        d = np.zeros_like(hs)
        d[c, z, y, x] = e
        fd = (L(hs=hs + d) - L(hs=hs - d)) / (2 * e)
        assert g["h"][c, z, y, x] == pytest.approx(fd, rel=1e-5, abs=1e-10)
        d = np.zeros_like(s0)
        d[c, z, y, x] = e
        fd = (L(s0=s0 + d) - L(s0=s0 - d)) / (2 * e)
        assert g["s0"][c, z, y, x] == pytest.approx(fd, rel=1e-5, abs=1e-10)
    assert np.allclose(g["H"], g["h"].reshape(3, -1).sum(axis=1), rtol=1e-10, atol=1e-12)
