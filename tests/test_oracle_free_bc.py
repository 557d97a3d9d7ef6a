"""Pins for the oracle with free boundaries (the paper's 64^3 particle of
Sec. IV, Fig. 7): sites on a face have fewer neighbours, bonds end at the
surface."""
import itertools
import math

import numpy as np
import pytest

import spin_inputs


def test_aligned_energy_counts_interior_bonds(orc):
    """E/N of an aligned state = -J n_bonds/N - D d_z^2 - H.d with
    n_bonds = (nx-1) ny nz + nx (ny-1) nz + nx ny (nz-1)."""
    d = np.array([0.36, -0.48, 0.8])
    for shape in [(4, 4, 4), (3, 5, 2), (1, 1, 1), (2, 1, 3)]:
        nx, ny, nz = shape
        p = orc.Params(*shape, J=1.3, D=0.25, H=(0.1, 0.2, -0.4), bc=1)
        nb = (nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1)
        E = orc.observables(p, spin_inputs.aligned_spins(*shape, d))[3]
        ref = -1.3 * nb / (nx * ny * nz) - 0.25 * d[2] ** 2 - np.dot([0.1, 0.2, -0.4], d)
        assert E == pytest.approx(ref, abs=1e-13)


def test_energy_bond_list_free(orc):
    shape = (3, 4, 2)
    nx, ny, nz = shape
    s = spin_inputs.random_spins(*shape, seed=5)
    hs = spin_inputs.site_fields(*shape, sigma=0.2, seed=6)
    J, D, H = 0.8, 0.3, np.array([0.1, -0.2, 0.3])
    p = orc.Params(*shape, J=J, D=D, H=tuple(H), bc=1)
    E = 0.0
    for x, y, z in itertools.product(range(nx), range(ny), range(nz)):
        si = s[:, z, y, x]
        for dx, dy, dz in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
            if x + dx < nx and y + dy < ny and z + dz < nz:
                E -= J * si @ s[:, z + dz, y + dy, x + dx]
        E -= D * si[2] ** 2 + (H + hs[:, z, y, x]) @ si
    assert orc.observables(p, s, hs)[3] == pytest.approx(E / (nx * ny * nz), abs=1e-14)


def test_heff_is_minus_gradient_free(orc):
    shape = (3, 4, 3)
    s = spin_inputs.random_spins(*shape, seed=9)
    hs = spin_inputs.site_fields(*shape, sigma=0.2, seed=1)
    p = orc.Params(*shape, J=0.9, D=0.35, H=(0.2, 0.1, -0.3), bc=1)
    Hf = orc.heff(p, s, hs)
    g = np.random.default_rng(2)
    for _ in range(12):
        a, z, y, x = (int(g.integers(0, m)) for m in (3, shape[2], shape[1], shape[0]))
        e = 1e-4
        sp, sm = s.copy(), s.copy()
        sp[a, z, y, x] += e
        sm[a, z, y, x] -= e
        dE = (orc.observables(p, sp, hs)[3] - orc.observables(p, sm, hs)[3]) * p.N / (2 * e)
        assert -dE == pytest.approx(Hf[a, z, y, x], abs=1e-9)
    # a corner site of a free lattice sees three neighbours, not six
    aligned = spin_inputs.aligned_spins(*shape, (0, 0, 1))
    q = orc.Params(*shape, J=1.0, bc=1)
    H0 = orc.heff(q, aligned)
    assert H0[2, 0, 0, 0] == pytest.approx(3.0) and H0[2, 1, 1, 1] == pytest.approx(6.0)


@pytest.mark.parametrize("precession", [1, 0])
def test_lyapunov_free(orc, precession):
    shape = (5, 3, 4)
    s0 = spin_inputs.random_spins(*shape, seed=2)
    kw = dict(J=0.7, D=0.45, H=(0.2, -0.3, 0.5), lam=0.3, renorm=0, R=10 ** 6, precession=precession, bc=1)
    dt = 1e-3
    fwd, _ = orc.run(orc.Params(*shape, dt=dt, **kw), s0, 1, noise=False)
    bwd, _ = orc.run(orc.Params(*shape, dt=-dt, **kw), s0, 1, noise=False)
    p = orc.Params(*shape, dt=dt, **kw)
    dEdt = (orc.observables(p, fwd)[3] - orc.observables(p, bwd)[3]) / (2 * dt)
    Hf = orc.heff(p, s0).reshape(3, -1)
    torque2 = np.sum(np.cross(s0.reshape(3, -1).T, Hf.T) ** 2) / p.N
    assert dEdt == pytest.approx(-0.3 * torque2, rel=1e-5)


def test_uniform_state_single_spin_map_free(orc):
    """A uniform state stays uniform with free boundaries too (every site's
    exchange field is parallel to s) and follows the closed-form map of
    Eq. (s_evolution_anal)."""
    shape = (4, 3, 5)
    lam, dt, n = 0.2, 0.01, 300
    th = math.radians(150.0)
    s0 = spin_inputs.aligned_spins(*shape, (math.sin(th), 0.0, math.cos(th)))
    p = orc.Params(*shape, J=1.3, D=0.0, H=(0, 0, 0.7), lam=lam, dt=dt, R=n + 1, bc=1)
    out, _ = orc.run(p, s0, n, noise=False)
    sz = math.tanh(lam * 0.7 * n * dt + math.atanh(math.cos(th)))
    assert np.max(np.abs(out[2] - sz)) < 1e-9


def test_adjoint_free_matches_fd(orc):
    shape = (4, 3, 3)
    base = dict(J=0.9, D=0.25, H=(0.05, -0.1, 0.2), lam=0.1, T=0.8, dt=0.1, R=4, seed=12, bc=1)
    p = orc.Params(*shape, **base)
    s0 = spin_inputs.random_spins(*shape, seed=11)
    dLdM, dLdE, n = np.array([0.3, -0.2, 0.7]), 1.0, 9
    g = orc.adjoint(p, s0, n, dLdM, dLdE)
    e = 1e-5

    def L(J):
        q = orc.Params(*shape, **{**base, "J": J})
        out, _ = orc.run(q, s0, n)
        o = orc.observables(q, out)
        return dLdE * o[3] + np.dot(dLdM, o[:3])

    assert g["J"] == pytest.approx((L(0.9 + e) - L(0.9 - e)) / (2 * e), rel=1e-6)
