"""Pins for the oracle's noise path: Philox4x64-10, Box-Muller, the pulse
angle of Eq. (phi_n) and the rotation of Eq. (s_rotation)."""
import json
import math
import os

import numpy as np
import pytest

import spin_inputs

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
M64 = (1 << 64) - 1


@pytest.mark.parametrize("key,ctr", [
    (0, 0), (1, 0), (12345, 7), ((1 << 64) + 5, (3 << 64) + 9),
    (0xDEADBEEFCAFEF00D, (1 << 191) + (77 << 64) + 3), (M64, M64 - 1),
])
def test_philox_matches_numpy(orc, key, ctr):
    """numpy.random.Philox is the same Philox4x64-10 generator.  It advances
    its 256-bit counter by one before producing its first block, so its first
    four words are the block of counter ctr + 1."""
    raw = [int(v) for v in np.random.Philox(key=key, counter=ctr).random_raw(4)]
    c = ctr + 1
    words = [(c >> (64 * i)) & M64 for i in range(4)]
    out = orc.philox4x64(words, [key & M64, (key >> 64) & M64])
    assert [int(v) for v in out] == raw


def test_philox_many_counters_match_numpy(orc):
    g = np.random.default_rng(3)
    for _ in range(50):
        key = int(g.integers(0, 1 << 63)) * 2 + 1
        ctr = int(g.integers(0, 1 << 62))
        raw = [int(v) for v in np.random.Philox(key=key, counter=ctr).random_raw(4)]
        out = orc.philox4x64([ctr + 1, 0, 0, 0], [key & M64, key >> 64])
        assert [int(v) for v in out] == raw


def _gauss_sample(orc, n, seed=11):
    return np.array([orc.noise_gauss(seed, i, 3, 0) for i in range(n)])


def test_box_muller_moments(orc):
    """G components are independent unit normals: mean 0, variance 1, fourth
    moment 3, no cross-correlation (bounds are ~5 standard errors)."""
    G = _gauss_sample(orc, 60000)
    n = len(G)
    for a in range(3):
        g = G[:, a]
        assert abs(g.mean()) < 5 / math.sqrt(n)
        assert abs(g.var() - 1.0) < 5 * math.sqrt(2.0 / n)
        assert abs((g ** 4).mean() - 3.0) < 5 * math.sqrt(96.0 / n)
    for a, b in [(0, 1), (0, 2), (1, 2)]:
        assert abs((G[:, a] * G[:, b]).mean()) < 5 / math.sqrt(n)


def test_box_muller_distribution_ks(orc):
    """Kolmogorov-Smirnov distance to the normal CDF (erf) per component."""
    G = _gauss_sample(orc, 20000, seed=5)
    n = len(G)
    for a in range(3):
        x = np.sort(G[:, a])
        cdf = 0.5 * (1.0 + np.array([math.erf(v / math.sqrt(2.0)) for v in x]))
        ks = max(np.max(np.arange(1, n + 1) / n - cdf), np.max(cdf - np.arange(n) / n))
        assert ks < 1.63 / math.sqrt(n) * 1.3  # ~1% level with margin


def test_box_muller_textbook_form(orc):
    """Box-Muller on hand-made words: u = ((w>>11)+1/2) 2^-53, G0 = r cos(2 pi u1),
    G1 = r sin(2 pi u1), r = sqrt(-2 ln u0), G2 = sqrt(-2 ln u2) cos(2 pi u3)."""
    w = [1 << 62, 3 << 61, 5 << 59, 1 << 63]
    u = [((v >> 11) + 0.5) / 2.0 ** 53 for v in w]
    G = orc.gauss3(w)
    r0 = math.sqrt(-2 * math.log(u[0]))
    assert G[0] == pytest.approx(r0 * math.cos(2 * math.pi * u[1]), abs=1e-15)
    assert G[1] == pytest.approx(r0 * math.sin(2 * math.pi * u[1]), abs=1e-15)
    assert G[2] == pytest.approx(math.sqrt(-2 * math.log(u[2])) * math.cos(2 * math.pi * u[3]), abs=1e-15)


def test_pulse_angle_printed_values(orc):
    """phi_RMS = sqrt(Lambda_N Delta t) with Lambda_N = 2 gamma lambda T / mu0
    reproduces the numbers printed in Sec. III.A."""
    g = GOLDEN["phi_rms_fig1"]
    R = int(round(g["Delta_t"] / g["dt"]))
    p = orc.Params(1, 1, 1, lam=g["lambda"], T=g["T"], dt=g["dt"], R=R)
    assert abs(orc.pulse_sigma(p) - g["value"]) < g["abs_tol"]
    for name in ("LambdaN_Dt_T1", "LambdaN_Dt_T01"):
        g = GOLDEN[name]
        p = orc.Params(1, 1, 1, lam=g["lambda"], T=g["T"], dt=g["Delta_t"], R=1)
        assert abs(orc.pulse_sigma(p) ** 2 - g["value"]) < 1e-12


def test_rotation_matches_scipy_rotvec(orc):
    """Eq. (s_rotation) is the rotation by the rotation vector phi (Rodrigues)."""
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    g = np.random.default_rng(0)
    for _ in range(200):
        phi = g.normal(size=3) * g.uniform(0.01, 3.0)
        s = g.normal(size=3)
        s /= np.linalg.norm(s)
        ref = Rot.from_rotvec(phi).apply(s)
        assert np.max(np.abs(orc.rotate(phi, s) - ref)) < 1e-14
    s = np.array([0.3, -0.4, np.sqrt(1 - 0.25)])
    assert np.array_equal(orc.rotate([0.0, 0.0, 0.0], s), s)


def test_rotation_right_handed(orc):
    s = orc.rotate([0.0, 0.0, 0.5], [1.0, 0.0, 0.0])
    assert np.allclose(s, [math.cos(0.5), math.sin(0.5), 0.0], atol=1e-15)


def one_pulse_decay(sig2):
    """<s_z'> / s_z after one pulse of isotropic Gaussian angle variance sig2 per
    component: (1 + 2 E[cos phi])/3 with E[cos(sigma|G|)] = (1-sig2) e^{-sig2/2}."""
    return (1.0 + 2.0 * (1.0 - sig2) * math.exp(-sig2 / 2.0)) / 3.0


@pytest.mark.parametrize("lam,T,dt,R", [(0.01, 1.0, 0.25, 40), (0.1, 1.0, 0.1, 10), (0.05, 0.8, 0.1, 10)])
def test_one_pulse_exact_decay(orc, lam, T, dt, R):
    """Pure-noise relaxation (Sec. III.A, Fig. 1): with J = D = H = 0 each pulse
    multiplies the mean s_z of aligned spins by the exact factor above, which
    tends to exp(-Lambda_N Delta t) for small angles."""
    n = 48
    p = orc.Params(n, n, n, J=0.0, D=0.0, H=(0, 0, 0), lam=lam, T=T, dt=dt, R=R, seed=9)
    s = spin_inputs.aligned_spins(n, n, n)
    s1 = orc.pulse(p, s, 0)
    sig2 = 2 * lam * T * R * dt
    mz = s1[2].mean()
    se = s1[2].std() / math.sqrt(p.N)
    assert abs(mz - one_pulse_decay(sig2)) < 5 * se
    assert np.max(np.abs(np.sum(s1 ** 2, axis=0) - 1.0)) < 1e-14
    assert abs(one_pulse_decay(sig2) - math.exp(-sig2)) < sig2 ** 2


def test_noise_only_run_decays_geometrically(orc):
    """m(t) = m0 prod of per-pulse factors, sampled at the end of each Delta t."""
    n = 32
    p = orc.Params(n, n, n, J=0.0, D=0.0, H=(0, 0, 0), lam=0.01, T=1.0, dt=0.25, R=40, seed=3)
    s = spin_inputs.aligned_spins(n, n, n)
    _, smp = orc.run(p, s, 40 * 6)
    c = one_pulse_decay(2 * 0.01 * 1.0 * 10.0)
    assert list(smp[:, 0]) == [40.0 * k for k in range(1, 7)]
    for k, row in enumerate(smp, start=1):
        assert abs(row[3] - c ** k) < 6 / math.sqrt(p.N)


def test_pulse_schedule(orc):
    """Pulse after step n when n mod R == floor(R/2) (R = 1: every step);
    pulse number floor((n-1)/R); middle of each interval (Eq. ST-expansion)."""
    for R in (1, 2, 5, 6, 10):
        pulses = [n for n in range(1, 4 * R + 1) if orc.is_pulse_step(n, R)]
        assert len(pulses) == 4
        assert [orc.pulse_number(n, R) for n in pulses] == [0, 1, 2, 3]
        for k, n in enumerate(pulses):
            assert k * R < n <= (k + 1) * R
            if R % 2 == 0:
                assert n - k * R == R // 2   # exactly mid-interval for even R


def test_pulses_only_at_scheduled_steps(orc):
    """With J = D = H = 0 the integrator is the identity, so the state changes
    exactly at the pulse steps and the pulse number picks the noise."""
    p = orc.Params(4, 3, 2, J=0.0, H=(0, 0, 0), lam=0.1, T=1.0, dt=0.1, R=6, seed=21, renorm=0)
    s = spin_inputs.random_spins(4, 3, 2, seed=1)
    prev = s.copy()
    for n in range(1, 19):
        cur, _ = orc.run(p, prev, 1, n0=n - 1)
        changed = not np.array_equal(cur, prev)
        assert changed == orc.is_pulse_step(n, 6)
        if changed:
            assert np.allclose(cur, orc.pulse(p, prev, orc.pulse_number(n, 6)), atol=1e-15)
        prev = cur


def test_openmp_build_is_bitwise_serial(orc):
    """The OpenMP build of the oracle (whole-lattice loops over z-planes on all
    host cores, used for the all-cores CPU baseline) computes every site with
    the same expression as the serial build: bitwise equal states and samples
    over 25 steps with two pulses, and for the slow equation and RK5."""
    import spin_inputs
    if orc.build_omp() is None:
        pytest.skip("gcc without OpenMP")
    for kw in (dict(), dict(precession=0, integrator=orc.RK2_MIDPOINT), dict(integrator=orc.RK5_BUTCHER, bc=1)):
        p = orc.Params(16, 12, 10, J=1.0, D=0.05, H=(0, 0, 0.1), lam=0.1, T=1.0, dt=0.1, R=10, seed=1, **kw)
        s0 = spin_inputs.random_spins(16, 12, 10, seed=0)
        a, sa = orc.run(p, s0, 25)
        b, sb = orc.run(p, s0, 25, threads=True)
        assert np.array_equal(a, b) and np.array_equal(sa, sb)
