"""Pins for the oracle's deterministic part: effective field, the right-hand
side of Eq. (LLL), the Appendix integrators, renormalisation and the energy."""
import itertools
import math

import numpy as np
import pytest

import spin_inputs


def _frame(Hvec):
    """Right-handed orthonormal frame (e1, e2, h) with h along H."""
    h = np.asarray(Hvec, float) / np.linalg.norm(Hvec)
    a = np.array([1.0, 0, 0]) if abs(h[0]) < 0.9 else np.array([0, 1.0, 0])
    e1 = a - h * (a @ h)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(h, e1)
    return e1, e2, h


def _uniform(shape, v):
    nx, ny, nz = shape
    return spin_inputs.aligned_spins(nx, ny, nz, v)


@pytest.mark.parametrize("integrator,tol", [(0, 1e-9), (1, 1e-10), (2, 2e-5), (3, 2e-5)])
@pytest.mark.parametrize("precession", [1, 0])
def test_uniform_state_follows_single_spin_map(orc, integrator, tol, precession):
    """With D = 0 a uniform state stays uniform (the exchange field is parallel
    to s) and each spin follows the closed-form map of Eq. (s_evolution_anal):
    the component along H obeys s_h' = tanh(lambda |H| t + artanh s_h) and the
    transverse part precesses by -|H| t about H (dropped in the slow equation)."""
    Hvec = (0.3, -0.2, 0.6)
    lam, dt, nsteps = 0.2, 0.01, 300
    e1, e2, h = _frame(Hvec)
    th, psi0 = math.radians(150.0), 0.4
    s0 = math.cos(th) * h + math.sin(th) * (math.cos(psi0) * e1 + math.sin(psi0) * e2)
    shape = (5, 4, 3)
    p = orc.Params(*shape, J=1.3, D=0.0, H=Hvec, lam=lam, dt=dt, R=nsteps + 1,
                   integrator=integrator, precession=precession)
    s, _ = orc.run(p, _uniform(shape, s0), nsteps, noise=False)
    t = nsteps * dt
    Hn = np.linalg.norm(Hvec)
    sh = math.tanh(lam * Hn * t + math.atanh(math.cos(th)))
    psi = psi0 - (Hn * t if precession else 0.0)
    ref = sh * h + math.sqrt(1 - sh * sh) * (math.cos(psi) * e1 + math.sin(psi) * e2)
    err = np.max(np.abs(s.reshape(3, -1) - ref[:, None]))
    assert err < tol


def test_magnon_dispersion(orc):
    """Linear spin waves about +z at lambda = 0: psi = s_x + i s_y = eps e^{i k.r}
    evolves as e^{-i omega t} with omega = H + 2D + 2J sum_a (1 - cos k_a).
    This fixes the J, D and H factors of H_eff and the sign of precession."""
    L = 8
    J, D, Hz = 1.0, 0.3, 0.5
    k = 2 * math.pi * np.array([1, 2, 3]) / L
    z, y, x = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    ph = k[0] * x + k[1] * y + k[2] * z
    eps = 1e-4
    s = np.stack([eps * np.cos(ph), eps * np.sin(ph), np.full(ph.shape, math.sqrt(1 - eps * eps))])
    dt, nsteps = 0.01, 200
    p = orc.Params(L, L, L, J=J, D=D, H=(0, 0, Hz), lam=0.0, dt=dt, R=nsteps + 1)
    out, _ = orc.run(p, s, nsteps, noise=False)
    omega = Hz + 2 * D + 2 * J * np.sum(1 - np.cos(k))
    psi = (out[0] + 1j * out[1]) / eps
    ref = np.exp(1j * (ph - omega * nsteps * dt))
    assert np.max(np.abs(psi - ref)) < 1e-4


@pytest.mark.parametrize("integrator,order", [(0, 4), (1, 5), (2, 2), (3, 2)])
def test_convergence_order(orc, integrator, order):
    """Global error at fixed time falls as dt^order (RK4: 4; Butcher RK5: 5;
    RK2 midpoint and Heun: 2)."""
    shape = (4, 4, 4)
    s0 = spin_inputs.random_spins(*shape, seed=7)
    kw = dict(J=1.0, D=0.3, H=(0.1, 0.2, 0.5), lam=0.1, renorm=0, R=10 ** 6)
    tend = 1.6
    ref_p = orc.Params(*shape, dt=tend / 1280, integrator=1, **kw)
    ref, _ = orc.run(ref_p, s0, 1280, noise=False)
    errs = []
    for dt in (0.1, 0.05, 0.025):
        p = orc.Params(*shape, dt=dt, integrator=integrator, **kw)
        out, _ = orc.run(p, s0, int(round(tend / dt)), noise=False)
        errs.append(np.max(np.abs(out - ref)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    for r in rates:
        assert order - 0.35 < r < order + 0.6, (errs, rates)


def _energy(orc, p, s, h=None):
    return orc.observables(p, s, h)[3]


def test_energy_derivative_is_minus_lambda_torque_squared(orc):
    """E is a Lyapunov function of Eq. (LLL): dE/dt = -lambda sum_i |s_i x H_eff,i|^2 / N
    when H_eff = -dE/ds.  A central difference of E along the integrated
    trajectory checks the bond counting of E against the J factor of H_eff,
    the 2D factor of the anisotropy field and the sign of every term."""
    shape = (5, 3, 4)
    s0 = spin_inputs.random_spins(*shape, seed=2)
    hs = spin_inputs.site_fields(*shape, sigma=0.3, seed=4)
    for precession in (1, 0):
        kw = dict(J=0.7, D=0.45, H=(0.2, -0.3, 0.5), lam=0.3, renorm=0, R=10 ** 6,
                  precession=precession)
        dt = 1e-3
        fwd, _ = orc.run(orc.Params(*shape, dt=dt, **kw), s0, 1, h_site=hs, noise=False)
        bwd, _ = orc.run(orc.Params(*shape, dt=-dt, **kw), s0, 1, h_site=hs, noise=False)
        p = orc.Params(*shape, dt=dt, **kw)
        dEdt = (_energy(orc, p, fwd, hs) - _energy(orc, p, bwd, hs)) / (2 * dt)
        Hf = orc.heff(p, s0, hs).reshape(3, -1)
        sv = s0.reshape(3, -1)
        torque2 = np.sum(np.cross(sv.T, Hf.T) ** 2) / p.N
        assert dEdt == pytest.approx(-0.3 * torque2, rel=1e-5)


def test_precession_conserves_energy_and_sz(orc):
    """lambda = 0 with D and H along z: E is conserved (drift falls ~2^4 per
    dt halving for RK4) and sum_i s_z is a linear invariant that RK methods
    keep to rounding (Sec. II: S_z is an integral of motion)."""
    shape = (6, 5, 4)
    s0 = spin_inputs.random_spins(*shape, seed=3)
    drifts = []
    for dt in (0.1, 0.05):
        p = orc.Params(*shape, J=1.0, D=0.4, H=(0, 0, 0.3), lam=0.0, dt=dt, R=10 ** 6, renorm=0)
        n = int(round(2.0 / dt))
        out, _ = orc.run(p, s0, n, noise=False)
        o0, o1 = orc.observables(p, s0), orc.observables(p, out)
        assert abs(o1[2] - o0[2]) < 1e-13
        drifts.append(abs(o1[3] - o0[3]))
    assert drifts[0] / drifts[1] > 10.0


def test_rk5_energy_drift_order(orc):
    """lambda = 0: Butcher's RK5 (Appendix) conserves the energy to order 5 —
    the drift over 2 time units falls ~2^5 per halving of dt once dt is small
    (measured 28.5 from dt = 0.05 to 0.025) and lies far below RK4's at the
    same dt (1.1e-7 against 7.6e-6 at dt = 0.05)."""
    shape = (6, 5, 4)
    s0 = spin_inputs.random_spins(*shape, seed=3)

    def drift(integrator, dt):
        p = orc.Params(*shape, J=1.0, D=0.4, H=(0, 0, 0.3), lam=0.0, dt=dt, R=10 ** 6, renorm=0,
                       integrator=integrator)
        out, _ = orc.run(p, s0, int(round(2.0 / dt)), noise=False)
        return abs(orc.observables(p, out)[3] - orc.observables(p, s0)[3])

    d5 = [drift(orc.RK5_BUTCHER, dt) for dt in (0.05, 0.025)]
    assert d5[0] / d5[1] > 20.0, d5
    assert d5[0] < drift(orc.RK4, 0.05) / 20.0, d5


def test_isotropic_exchange_rigid_rotation(orc):
    """D = 0, lambda = 0: internal exchange torques cancel pairwise, so
    dM/dt = M x H and M rotates rigidly about H by -|H| t."""
    shape = (4, 6, 5)
    s0 = spin_inputs.random_spins(*shape, seed=8)
    Hz = 0.7
    p = orc.Params(*shape, J=1.0, D=0.0, H=(0, 0, Hz), lam=0.0, dt=0.02, R=10 ** 6, renorm=0)
    out, _ = orc.run(p, s0, 100, noise=False)
    M0 = orc.observables(p, s0)[:3]
    M1 = orc.observables(p, out)[:3]
    a = -Hz * 2.0
    ref = np.array([M0[0] * math.cos(a) - M0[1] * math.sin(a), M0[0] * math.sin(a) + M0[1] * math.cos(a), M0[2]])
    assert np.max(np.abs(M1 - ref)) < 1e-9


def test_energy_uniform_closed_form(orc):
    """Aligned state: E/N = -3J - D d_z^2 - H.d (three bonds per site)."""
    d = np.array([0.36, -0.48, 0.8])
    for shape in [(4, 4, 4), (3, 5, 2), (1, 1, 1), (2, 1, 3)]:
        p = orc.Params(*shape, J=1.3, D=0.25, H=(0.1, 0.2, -0.4))
        E = _energy(orc, p, _uniform(shape, d))
        assert E == pytest.approx(-3 * 1.3 - 0.25 * d[2] ** 2 - np.dot([0.1, 0.2, -0.4], d), abs=1e-13)


def test_energy_brute_force_bond_list(orc):
    """Energy by explicit enumeration of the nearest-neighbour pairs of a
    periodic lattice (a size-2 direction gives two bonds between the same
    pair; a size-1 direction gives a bond of a site with itself)."""
    shape = (3, 2, 4)
    nx, ny, nz = shape
    s = spin_inputs.random_spins(*shape, seed=5)
    hs = spin_inputs.site_fields(*shape, sigma=0.2, seed=6)
    J, D, H = 0.8, 0.3, np.array([0.1, -0.2, 0.3])
    p = orc.Params(*shape, J=J, D=D, H=tuple(H))
    E = 0.0
    for x, y, z in itertools.product(range(nx), range(ny), range(nz)):
        si = s[:, z, y, x]
        for dx, dy, dz in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
            sj = s[:, (z + dz) % nz, (y + dy) % ny, (x + dx) % nx]
            E -= J * si @ sj
        E -= D * si[2] ** 2 + (H + hs[:, z, y, x]) @ si
    assert _energy(orc, p, s, hs) == pytest.approx(E / (nx * ny * nz), abs=1e-14)


def test_heff_is_minus_energy_gradient(orc):
    """H_eff,i = -dE_total/ds_i, checked component by component by central
    differences of the energy (E is quadratic, so the difference is exact up
    to rounding)."""
    shape = (3, 4, 2)
    s = spin_inputs.random_spins(*shape, seed=9)
    hs = spin_inputs.site_fields(*shape, sigma=0.2, seed=1)
    p = orc.Params(*shape, J=0.9, D=0.35, H=(0.2, 0.1, -0.3))
    Hf = orc.heff(p, s, hs)
    N = p.N
    g = np.random.default_rng(1)
    for _ in range(12):
        a, z, y, x = (int(g.integers(0, m)) for m in (3, shape[2], shape[1], shape[0]))
        e = 1e-4
        sp, sm = s.copy(), s.copy()
        sp[a, z, y, x] += e
        sm[a, z, y, x] -= e
        dE = (_energy(orc, p, sp, hs) - _energy(orc, p, sm, hs)) * N / (2 * e)
        assert -dE == pytest.approx(Hf[a, z, y, x], abs=1e-9)


def test_renormalisation(orc):
    shape = (3, 3, 3)
    s = 1.7 * spin_inputs.random_spins(*shape, seed=2)
    out = orc.renormalise(orc.Params(*shape), s)
    assert np.max(np.abs(np.sum(out ** 2, axis=0) - 1.0)) < 1e-15
    assert np.allclose(out * 1.7, s, atol=1e-15)


def test_renormalised_step_keeps_unit_length(orc):
    shape = (5, 5, 5)
    s = spin_inputs.random_spins(*shape, seed=11)
    p = orc.Params(*shape, J=1.0, D=0.1, H=(0, 0, 0.2), lam=0.1, dt=0.1, R=10, seed=3)
    out, _ = orc.run(p, s, 25)
    assert np.max(np.abs(np.sum(out ** 2, axis=0) - 1.0)) < 1e-15
    p0 = orc.Params(*shape, J=1.0, D=0.1, H=(0, 0, 0.2), lam=0.1, dt=0.1, R=10, seed=3, renorm=0)
    raw = orc.integrate(p0, s)
    dev = np.max(np.abs(np.sum(raw ** 2, axis=0) - 1.0))
    assert 1e-12 < dev < 1e-3   # RK4 drifts off the sphere by O(dt^5) per step


@pytest.mark.parametrize("k", [2.0, 4.0, 3.0])
def test_slow_equation_lambda_scales_out(orc, k):
    """Sec. IV: without precession, (lambda, dt, Delta t) and (lambda/k, k dt,
    k Delta t) give the same trajectory with the same noise (bit-identical for
    k a power of two, since scaling by 2 is exact)."""
    shape = (4, 5, 3)
    s = spin_inputs.random_spins(*shape, seed=4)
    base = dict(J=1.0, D=0.2, H=(0.1, 0, 0.3), T=1.1, R=4, seed=17, precession=0)
    a, sa = orc.run(orc.Params(*shape, lam=0.5, dt=0.05, **base), s, 40)
    b, sb = orc.run(orc.Params(*shape, lam=0.5 / k, dt=0.05 * k, **base), s, 40)
    if k in (2.0, 4.0):
        assert np.array_equal(a, b)
    else:
        assert np.max(np.abs(a - b)) < 1e-12
    assert np.allclose(sa[:, 1:], sb[:, 1:], atol=1e-12)


def test_precession_step_limit_on_the_lattice(orc):
    """Sec. III.B: with the precession term the integration step must keep
    gamma H_eff dt at or below about 0.25, larger steps lose accuracy.  On the
    simple-cubic lattice the exchange field is up to 6 J, so dt = 0.2 gives
    gamma H_eff dt ~ 1.2: started from a T = 1.3 Metropolis state, the
    noiseless, undamped, renormalised RK4 step then changes the energy (an
    integral of motion at lambda = 0) by more than one J per spin in 200 time
    units, while dt = 0.04 (gamma H_eff dt ~ 0.24) keeps it within 0.02."""
    n = 8
    q = orc.Params(n, n, n, J=1.0, D=0.05, H=(0, 0, 0.02), T=1.3)
    s, _, _ = orc.metropolis(q, spin_inputs.aligned_spins(n, n, n), 500, mc_seed=3)
    drift = {}
    for dt in (0.2, 0.04):
        p = orc.Params(n, n, n, J=1.0, D=0.05, H=(0, 0, 0.02), lam=0.0, dt=dt, R=10 ** 6)
        out, _ = orc.run(p, s, int(round(200 / dt)), noise=False)
        drift[dt] = abs(orc.observables(p, out)[3] - orc.observables(p, s)[3])
    assert drift[0.04] < 0.02, drift
    assert drift[0.2] > 1.0, drift
