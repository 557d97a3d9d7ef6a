"""Single-spin replica kernels (spin_single_run, spin_single_escape) against
the oracle: replica r of the GPU kernels is the oracle's one-site lattice
with J = 0 and replica index r (trial j of the escape kernel: replica index
r + j nrep, pulse schedule counted from the trial's start).  The energy is
E = -D s_z^2 - H.s of Sec. III (spin in a field; uniaxial spin in a
transverse field)."""
import math

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

H_ESC = 0.5  # h = H/(2D) of the escape problem, Sec. III.B
S_WELL = (H_ESC, 0.0, math.sqrt(1.0 - H_ESC ** 2))  # bottom of the well phi = 0, sin(theta) = h


def _orc_one(orc, p, r, T, lam, **over):
    kw = dict(J=0.0, D=p.D, H=tuple(p.H), lam=lam, T=T, dt=p.dt, R=p.R, integrator=p.integrator,
              precession=p.precession, renorm=p.renorm, seed=p.seed, replica=r)
    kw.update(over)
    return orc.Params(1, 1, 1, **kw)


def _start(nrep, seed):
    g = np.random.default_rng(seed)
    v = g.normal(size=(3, nrep))
    return v / np.linalg.norm(v, axis=0)


def _input(prec, a):
    a = np.asarray(a, dtype=np.float64)
    return a.astype(np.float32).astype(np.float64) if prec == 32 else a


CASES = [  # precision, integrator, precession, R, nsteps
    (64, 1, 1, 6, 60),
    (64, 0, 1, 4, 41),
    (64, 2, 0, 2, 33),
    (64, 3, 1, 5, 25),
    (32, 1, 1, 6, 36),
    (32, 0, 0, 4, 40),
]


@pytest.mark.parametrize("prec,integ,precession,R,nsteps", CASES)
def test_run_matches_oracle(gpu, orc, prec, integ, precession, R, nsteps):
    nrep = 67  # one full block of 128 threads is not filled: ragged tail
    T = np.linspace(0.05, 2.0, nrep)
    lam = np.linspace(0.001, 0.3, nrep)[::-1].copy()
    p = gpu.Params(1, 1, 1, J=0.0, D=0.8, H=(0.3, -0.2, 0.4), lam=0.0, T=0.0, dt=0.11, R=R, integrator=integ,
                   precession=precession, seed=21, precision=prec)
    s0 = _start(nrep, 4)
    ss = gpu.SingleSpins(p, T, torch.from_numpy(s0), lam=lam)
    ss.run(nsteps // 2).run(nsteps - nsteps // 2, average=True)
    torch.cuda.synchronize()
    got = ss.state.double().cpu().numpy()
    sz_sum = ss.sz_sum.cpu().numpy()
    cnt = ss.sz_count.cpu().numpy()
    tol = 1e-12 if prec == 64 else 2e-5
    s0i = _input(prec, s0)
    for r in range(nrep):
        op = _orc_one(orc, p, r, T[r], lam[r])
        a, _ = orc.run(op, s0i[:, r].reshape(3, 1, 1, 1), nsteps // 2)
        acc, k = 0.0, 0
        for n in range(nsteps // 2, nsteps):
            a, _ = orc.run(op, a, 1, n0=n)
            if (n + 1) % R == 0:
                acc += a[2].item()
                k += 1
        assert np.max(np.abs(got[:, r] - a.reshape(3))) < tol, r
        assert cnt[r] == k
        assert abs(sz_sum[r] - acc) < tol * max(k, 1)


RECT_CASES = [  # precision, integrator, R, nsteps, first call
    (64, 1, 4, 30, 13),
    (64, 3, 1, 40, 17),
    (64, 0, 3, 25, 10),
    (32, 1, 4, 24, 9),
    (32, 3, 1, 40, 21),
]


@pytest.mark.parametrize("prec,integ,R,nsteps,first", RECT_CASES)
def test_run_rectangular_noise_matches_oracle(gpu, orc, prec, integ, R, nsteps, first):
    """Rectangular noise, Eq. (zeta_n) (noise = 2): the field of interval k
    uses the counter of pulse k; calls that end mid-interval resume with the
    same field."""
    nrep = 45
    T = np.linspace(0.1, 1.5, nrep)
    lam = np.linspace(0.002, 0.2, nrep)
    p = gpu.Params(1, 1, 1, J=0.0, D=0.6, H=(0.2, 0.1, 0.7), lam=0.0, T=0.0, dt=0.07, R=R, integrator=integ,
                   precession=1, noise=2, seed=41, precision=prec)
    s0 = _start(nrep, 6)
    ss = gpu.SingleSpins(p, T, torch.from_numpy(s0), lam=lam)
    ss.run(first).run(nsteps - first)
    torch.cuda.synchronize()
    got = ss.state.double().cpu().numpy()
    tol = 1e-12 if prec == 64 else 2e-5
    s0i = _input(prec, s0)
    for r in range(nrep):
        op = _orc_one(orc, p, r, T[r], lam[r])
        a, _ = orc.run(op, s0i[:, r].reshape(3, 1, 1, 1), nsteps, noise=2)
        assert np.max(np.abs(got[:, r] - a.reshape(3))) < tol, r


def test_rectangular_noise_needs_precession(gpu):
    p = gpu.Params(1, 1, 1, J=0.0, D=1.0, lam=0.1, T=0.3, dt=0.1, R=2, precession=0, noise=2, precision=64)
    with pytest.raises(gpu.SpinError):
        gpu.SingleSpins(p, [0.3], torch.tensor([[0.0], [0.0], [1.0]])).run(3)
    q = gpu.Params(4, 4, 4, noise=2)
    with pytest.raises(gpu.SpinError):
        gpu.Lattice(q, torch.from_numpy(np.ascontiguousarray(_start(64, 1).reshape(3, 4, 4, 4))))


def test_first_passage_matches_oracle(gpu, orc):
    """Stop at the first step that leaves s_z < 0 (FP64): the recorded step
    equals the oracle's, replica by replica."""
    nrep, R, dt = 24, 6, 1.0 / 6.0
    T = [0.4] * nrep
    p = gpu.Params(1, 1, 1, J=0.0, D=1.0, H=(1.0, 0, 0), lam=0.1, T=0.4, dt=dt, R=R, integrator=gpu.RK5_BUTCHER,
                   seed=8, precision=64)
    init = np.tile(np.array(S_WELL).reshape(3, 1), (1, nrep))
    ss = gpu.SingleSpins(p, T, torch.from_numpy(init))
    for _ in range(4):
        ss.run(150, stop_on_crossing=True)
    torch.cuda.synchronize()
    fp = ss.first_passage.cpu().numpy()
    got = ss.state.cpu().numpy()
    crossed = 0
    for r in range(nrep):
        op = _orc_one(orc, p, r, 0.4, 0.1)
        a = init[:, r].reshape(3, 1, 1, 1).copy()
        want, prev = -1, None
        for n in range(600):
            prev = a[2].item()
            a, _ = orc.run(op, a, 1, n0=n)
            if a[2].item() < 0:
                want = n + 1
                break
        if want > 0 and (abs(a[2].item()) < 1e-9 or abs(prev) < 1e-9):
            continue  # a crossing within rounding of s_z = 0: not decidable
        assert fp[r] == want, (r, fp[r], want)
        if want > 0:
            crossed += 1
            assert np.max(np.abs(got[:, r] - a.reshape(3))) < 1e-12
    assert crossed >= nrep // 2  # at T = 0.4 most replicas cross within 100 time units


@pytest.mark.parametrize("prec,noise", [(64, 1), (32, 1), (64, 2)])
def test_escape_renewal_matches_oracle(gpu, orc, prec, noise):
    """The renewal kernel: each finished trial's passage step, the trial
    count, the waiting state and the running trial agree with the oracle run
    trial by trial (trial j of replica r = oracle replica r + j nrep, started
    at the first global step n >= the passage with n mod R == 0)."""
    nrep, R, dt, nsteps = 8, 6, 1.0 / 6.0, 400
    T, lam = [0.35 + 0.05 * r for r in range(nrep)], [0.05 + 0.02 * r for r in range(nrep)]
    p = gpu.Params(1, 1, 1, J=0.0, D=1.0, H=(1.0, 0, 0), lam=0.0, T=0.0, dt=dt, R=R,
                   integrator=gpu.RK5_BUTCHER, seed=31, precision=prec, noise=noise)
    e = gpu.EscapeReplicas(p, T, S_WELL, lam=lam)
    e.run(151).run(nsteps - 151)  # a call boundary inside an interval
    torch.cuda.synchronize()
    fsum, fcnt = e.fpt_sum.cpu().numpy(), e.fpt_count.cpu().numpy()
    trial, local = e.trial.cpu().numpy(), e.local_step.cpu().numpy()
    fsq = e.fpt_sq.cpu().numpy()
    init = _input(prec, np.array(S_WELL)).reshape(3, 1, 1, 1)
    total = 0
    for r in range(nrep):
        j, m, a, steps = 0, 0, init.copy(), []
        tie = False
        for n in range(1, nsteps + 1):
            if m >= 0:
                op = _orc_one(orc, p, r + j * nrep, T[r], lam[r])
                a, _ = orc.run(op, a, 1, n0=m, noise=noise)
                m += 1
                if abs(a[2].item()) < (1e-9 if prec == 64 else 1e-4):
                    tie = True
                if a[2].item() < 0:
                    steps.append(m)
                    j, m = j + 1, -1
            if m < 0 and n % R == 0:
                m, a = 0, init.copy()
        if tie and prec == 32:
            continue  # FP32 rounding may decide a marginal crossing differently
        assert not tie
        assert fcnt[r] == len(steps) and trial[r] == j and local[r] == m, r
        assert fsum[r] == sum(steps) and fsq[r] == float(sum(x * x for x in steps))
        if m > 0 and prec == 64:
            assert np.max(np.abs(e.state[:, r].cpu().numpy() - a.reshape(3))) < 1e-12
        total += len(steps)
    assert total > 0


def test_escape_mfpt_estimators(gpu):
    """mfpt(): the mean of finished trials and the rate estimate (finished
    trials / total time, unfinished trials included) agree for a long run,
    and the per-group split adds up."""
    nrep = 2048
    p = gpu.Params(1, 1, 1, J=0.0, D=1.0, H=(1.0, 0, 0), lam=0.1, T=0.25, dt=1.0 / 6.0, R=6,
                   integrator=gpu.RK5_BUTCHER, seed=3, precision=32)
    e = gpu.EscapeReplicas(p, [0.25] * nrep, S_WELL)
    e.run(30000)
    m, se, n, rate = e.mfpt()
    assert n > 20 * nrep
    assert abs(1.0 / m - rate) / rate < 5 * se / m
    halves = e.mfpt([list(range(0, nrep, 2)), list(range(1, nrep, 2))])
    assert halves[0][2] + halves[1][2] == n


def test_single_rejects_bad_arguments(gpu):
    import ctypes

    from paper_1610_04914_gb300 import _binding as B

    L = B.load()
    p = gpu.Params(1, 1, 1, J=0.0, D=1.0, H=(1.0, 0, 0), lam=0.1, T=0.3, dt=0.1, R=2, precision=64)
    s = torch.zeros(3, 4, dtype=torch.float64, device="cuda")
    sc = torch.zeros(8, dtype=torch.float64, device="cuda")
    T = (ctypes.c_double * 4)(0.3, 0.3, -0.1, 0.3)
    assert L.spin_single_prepare(ctypes.byref(p.c()), 4, T, None, sc.data_ptr(), None) == B.SPIN_EINVAL
    lam = (ctypes.c_double * 4)(0.1, float("nan"), 0.1, 0.1)
    T = (ctypes.c_double * 4)(0.3, 0.3, 0.3, 0.3)
    assert L.spin_single_prepare(ctypes.byref(p.c()), 4, T, lam, sc.data_ptr(), None) == B.SPIN_EINVAL
    assert L.spin_single_prepare(ctypes.byref(p.c()), 4, T, None, sc.data_ptr(), None) == B.SPIN_OK
    assert L.spin_single_run(ctypes.byref(p.c()), 0, s.data_ptr(), sc.data_ptr(), 0, 5, 0, None, None, None,
                             None) == B.SPIN_EINVAL
    # stop requested without a first_passage array
    assert L.spin_single_run(ctypes.byref(p.c()), 4, s.data_ptr(), sc.data_ptr(), 0, 5, 1, None, None, None,
                             None) == B.SPIN_EINVAL
    init = (ctypes.c_double * 3)(0.0, 0.0, -1.0)  # a trial must start with s_z >= 0
    z = torch.zeros(4, dtype=torch.int64, device="cuda")
    assert L.spin_single_escape(ctypes.byref(p.c()), 4, init, s.data_ptr(), sc.data_ptr(), 0, 5, z.data_ptr(),
                                z.data_ptr(), z.data_ptr(), None, z.data_ptr(), None) == B.SPIN_EINVAL
