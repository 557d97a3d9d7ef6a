"""GPU (sm_103a, through the C-ABI) against the FP64 oracle on identical seeded
inputs and identical Philox noise.

Tolerances.  FP64 path: one step agrees to a few ulps (1e-13 per step).
FP32 path: one step from the same float32 input agrees with the FP64 oracle to
2e-6 (float rounding of the stage states, ~10 eps).  Whole trajectories are
compared over the horizon where the oracle's own sensitivity keeps rounding
differences below the tolerance: the 16^3 workload at T=1 amplifies a
perturbation by ~2.5x per unit time, so 1e-16 reaches 1e-11 after ~120 steps
of dt=0.1 and 1e-7 reaches 1e-5 after ~50 steps.  Longer runs are checked step
by step (oracle restarted from the GPU state at every step) over all 200
steps, and statistically elsewhere."""
import numpy as np
import pytest
import torch

import spin_inputs
from gpu_helpers import as_input, gpu_state, orc_params, run_gpu, run_oracle

pytestmark = pytest.mark.gpu
M64 = (1 << 64) - 1


# ----------------------------------------------------------------- noise draw
@pytest.mark.parametrize("seed,k,replica", [(1, 0, 0), ((1 << 63) + 5, 17, 3), (123, 999, 511)])
def test_noise_words_bit_exact(gpu, orc, seed, k, replica):
    n = 3000
    words, g64 = gpu.spin_noise_draw(seed, k, replica, n, precision=64)
    _, g32 = gpu.spin_noise_draw(seed, k, replica, n, precision=32)
    torch.cuda.synchronize()
    w = words.cpu().numpy().view(np.uint64)
    g64 = g64.cpu().numpy()
    g32 = g32.double().cpu().numpy()
    for i in range(0, n, 7):
        ref = orc.philox4x64([i, k, replica, 0], [seed & M64, orc.STREAM_NOISE])
        assert [int(v) for v in w[i]] == [int(v) for v in ref]
    ref_g = np.array([orc.noise_gauss(seed, i, k, replica) for i in range(n)])
    assert np.max(np.abs(g64 - ref_g)) < 2e-14
    assert np.max(np.abs(g32 - ref_g)) < 1e-5


# ----------------------------------------------------------------- short runs
CASES = [
    # size, precision, integrator, precession, with h_site, path
    ((16, 16, 16), 64, 0, 1, False, 0),
    ((16, 16, 16), 32, 0, 1, False, 0),
    ((37, 21, 13), 32, 0, 1, True, 0),
    ((37, 21, 13), 64, 0, 0, True, 0),
    ((2, 3, 5), 64, 0, 1, False, 0),
    ((2, 3, 5), 32, 0, 1, True, 0),
    ((1, 1, 1), 64, 0, 1, False, 0),
    ((64, 8, 9), 32, 0, 0, False, 0),
    ((20, 19, 18), 64, 2, 1, False, 0),
    ((20, 19, 18), 32, 2, 0, True, 0),
    ((20, 19, 18), 32, 3, 1, False, 0),
    ((11, 12, 7), 64, 3, 0, True, 0),
    ((20, 19, 18), 64, 1, 1, False, 0),
    ((20, 19, 18), 32, 1, 1, True, 0),
    ((9, 10, 11), 64, 1, 0, False, 0),
    ((20, 19, 18), 64, 0, 1, True, 1),
    ((20, 19, 18), 32, 0, 0, False, 1),
    # rows of 64 and 128 columns (2 and 4 tiles of the fused step along x,
    # the benchmark's row length)
    ((128, 10, 7), 32, 0, 1, False, 0),
    ((64, 30, 21), 32, 0, 0, False, 0),
    ((64, 17, 40), 32, 0, 1, False, 0),
    # Butcher RK5 on the fused two-segment path (FP32, no h_i): ragged, tiny,
    # one site, several tiles along x and y, and a 128-column row
    ((20, 19, 18), 32, 1, 0, False, 0),
    ((37, 21, 13), 32, 1, 1, False, 0),
    ((2, 3, 5), 32, 1, 1, False, 0),
    ((1, 1, 1), 32, 1, 0, False, 0),
    ((64, 30, 21), 32, 1, 1, False, 0),
    ((128, 10, 7), 32, 1, 0, False, 0),
    # rows of 26 and 52 columns: the last tile along x outputs one column
    ((26, 9, 5), 32, 1, 1, False, 0),
    ((52, 7, 6), 32, 1, 0, False, 0),
    ((20, 19, 18), 32, 1, 1, False, 1),
    # RK4 on lattices whose x and y sides are multiples of 4 (x >= 24,
    # y >= 16), the shapes that also qualify for TMA staging
    ((24, 16, 9), 32, 0, 1, False, 0),
    ((48, 40, 20), 32, 0, 1, True, 0),
    ((128, 36, 17), 32, 0, 0, False, 0),
    ((28, 20, 11), 32, 0, 1, True, 0),
]


@pytest.mark.parametrize("shape,prec,integ,precession,hsite,path", CASES)
def test_three_steps_with_pulse(gpu, orc, shape, prec, integ, precession, hsite, path):
    """Three steps with R = 3: a pulse after step 1 (mid-interval), a sample
    after step 3; fused kernels (RK4, RK2, Heun; RK5 in two segments) and
    per-stage kernels (RK5 with h_i or in FP64, forced path 1), ragged and tiny
    lattices, with and without h_i."""
    nx, ny, nz = shape
    p = gpu.Params(nx, ny, nz, J=0.9, D=0.15, H=(0.05, -0.1, 0.2), lam=0.1, T=0.7, dt=0.07, R=3,
                   integrator=integ, precession=precession, seed=77, replica=2, precision=prec, path=path)
    s0 = spin_inputs.random_spins(nx, ny, nz, seed=3)
    hs = spin_inputs.site_fields(nx, ny, nz, 0.1, seed=4) if hsite else None
    got, lat = run_gpu(gpu, p, s0, 3, h_site=hs)
    ref, smp = run_oracle(orc, p, s0, 3, h_site=hs)
    tol = 1e-13 if prec == 64 else 2e-6
    assert np.max(np.abs(got - ref)) < tol
    rec = lat.samples()
    assert len(rec) == 1 and rec[0][0] == 3.0
    assert np.max(np.abs(np.array(rec[0][1:]) - smp[0, 1:])) < (1e-13 if prec == 64 else 5e-6)


@pytest.mark.parametrize("prec", [64, 32])
def test_step_by_step_200_steps(gpu, orc, prec):
    """The 16^3 workload (J=1, H=0.1 z, lambda=0.1, T=1, RK4 dt=0.1, pulses
    every 10 steps): at every one of 200 steps the oracle, restarted from the
    GPU state, reproduces the GPU's next state (pulse steps included)."""
    n = 16
    p = gpu.Params(n, n, n, J=1.0, D=0.0, H=(0, 0, 0.1), lam=0.1, T=1.0, dt=0.1, R=10, seed=1, precision=prec)
    s0 = spin_inputs.random_spins(n, n, n, seed=0)
    lat = gpu.Lattice(p, torch.from_numpy(s0))
    cur = gpu_state(lat)
    worst = 0.0
    op = orc_params(orc, p)
    for step in range(200):
        lat.step(1)
        nxt = gpu_state(lat)
        ref, _ = orc.run(op, cur, 1, n0=step)
        worst = max(worst, float(np.max(np.abs(nxt - ref))))
        cur = nxt
    assert worst < (1e-13 if prec == 64 else 2e-6), worst


def test_fp64_trajectory_16cubed(gpu, orc):
    """Whole-trajectory parity of the FP64 path on the 16^3 workload: 1e-11
    over the first 100 steps (the stated FP64 tolerance, within the chaos
    horizon) and the measured sensitivity envelope (1e-8) at 200 steps."""
    n = 16
    p = gpu.Params(n, n, n, J=1.0, D=0.0, H=(0, 0, 0.1), lam=0.1, T=1.0, dt=0.1, R=10, seed=1, precision=64)
    s0 = spin_inputs.random_spins(n, n, n, seed=0)
    lat = gpu.Lattice(p, torch.from_numpy(s0))
    lat.step(100)
    got100 = gpu_state(lat)
    ref100, smp100 = run_oracle(orc, p, s0, 100)
    assert np.max(np.abs(got100 - ref100)) < 1e-11
    lat.step(100)
    got200 = gpu_state(lat)
    ref200, smp200 = run_oracle(orc, p, ref100, 100, n0=100)
    assert np.max(np.abs(got200 - ref200)) < 1e-8
    rec = np.array(lat.samples())
    assert rec.shape == (20, 5)
    assert np.array_equal(rec[:, 0], np.arange(10, 201, 10, dtype=float))
    allsmp = np.vstack([smp100, smp200])
    assert np.max(np.abs(rec[:10, 1:] - allsmp[:10, 1:])) < 1e-12


def test_fp32_trajectory_16cubed(gpu, orc):
    """FP32 state against the FP64 oracle on the 16^3 workload: 1e-5 max-abs
    over 20 steps, and the two samples (steps 10, 20) to 5e-6.  FP32 rounding
    (~1e-7 per component and step, at every site) compounds with the system's
    ~2.5x-per-unit-time sensitivity; at 40 steps the measured gap is ~1.2e-5
    and by 200 steps the microscopic trajectories have decorrelated (sample
    energies then differ by ~1e-3), so longer horizons are compared
    statistically (equilibrium averages), not pointwise."""
    n = 16
    p = gpu.Params(n, n, n, J=1.0, D=0.0, H=(0, 0, 0.1), lam=0.1, T=1.0, dt=0.1, R=10, seed=1, precision=32)
    s0 = spin_inputs.random_spins(n, n, n, seed=0)
    got, lat = run_gpu(gpu, p, s0, 20)
    ref, smp = run_oracle(orc, p, s0, 20)
    assert np.max(np.abs(got - ref)) < 1e-5
    rec = np.array(lat.samples())
    assert rec.shape == smp.shape == (2, 5)
    assert np.max(np.abs(rec[:, 1:] - smp[:, 1:])) < 5e-6


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("shape", [(16, 16, 16), (5, 7, 3), (1, 1, 1), (2, 2, 2), (130, 64, 96)])
def test_observables(gpu, orc, prec, shape):
    """M and E against the oracle on the same values.  FP64 states: FP64
    arithmetic throughout (1e-13).  FP32 states: each lane pre-sums its
    k = ceil(nx/32) sites of a row in FP32 (the spin components exactly as
    stored, and each site's energy term formed in FP32 like the stencil), and
    everything longer is summed in FP64.  M: a pre-sum of k values of size <= 1
    carries at most (k-1) k 2^-24 absolute error, so M per spin is off by at
    most (k-1) 2^-24 <= 2.4e-7 for rows up to 160 sites: bound 1e-6.  E: each
    site's term (|e_i| < 7 here, ~8 roundings) is off by at most 3.3e-6 and the
    pre-sums add (k-1) k 7 2^-24 / k per site: bound 5e-6.  (130, 64, 96):
    rows of 130 sites, five sites per lane of which the last is ragged."""
    nx, ny, nz = shape
    p = gpu.Params(nx, ny, nz, J=0.8, D=0.3, H=(0.1, -0.2, 0.3), precision=prec)
    s0 = spin_inputs.random_spins(nx, ny, nz, seed=9)
    hs = spin_inputs.site_fields(nx, ny, nz, 0.2, seed=8)
    lat = gpu.Lattice(p, torch.from_numpy(s0), h_site=torch.from_numpy(hs))
    M, E = lat.observables()
    ref = orc.observables(orc_params(orc, p), as_input(p, s0), as_input(p, hs))
    tm, te = (1e-13, 1e-13) if prec == 64 else (1e-6, 5e-6)
    assert np.max(np.abs(np.array(M) - ref[:3])) < tm
    assert abs(E - ref[3]) < te


@pytest.mark.parametrize("shape,hsite,bc", [((48, 40, 20), False, 0), ((28, 20, 11), True, 1),
                                             ((128, 36, 17), True, 0), ((72, 64, 33), False, 1)])
def test_tma_staging_bitwise(gpu, shape, hsite, bc, monkeypatch):
    """RK4 lattices that qualify for TMA staging (SPIN_TMA=1) give bitwise the
    same states (20 steps, two pulses) as with the spin planes staged per
    thread by cp.async (the default): the two stagings move the same values
    into the tile and every output site keeps its arithmetic."""
    nx, ny, nz = shape
    p = gpu.Params(nx, ny, nz, J=1.0, D=0.05, H=(0.01, -0.02, 0.02), lam=0.05, T=1.0, dt=0.1, R=10, seed=3,
                   precision=32, bc=bc)
    s0 = spin_inputs.random_spins(nx, ny, nz, seed=2)
    hs = spin_inputs.site_fields(nx, ny, nz, 0.1, seed=4) if hsite else None
    monkeypatch.setenv("SPIN_TMA", "1")
    a, la = run_gpu(gpu, p, s0, 20, h_site=hs)
    monkeypatch.delenv("SPIN_TMA", raising=False)
    b, lb = run_gpu(gpu, p, s0, 20, h_site=hs)
    monkeypatch.delenv("SPIN_TMA", raising=False)
    la.close()
    lb.close()
    assert np.array_equal(a, b)


@pytest.mark.parametrize("shape,precession,bc", [((128, 128, 40), 1, 0), ((64, 57, 33), 0, 1), ((37, 21, 13), 1, 0),
                                                  ((2, 3, 5), 1, 1), ((1, 1, 1), 0, 0), ((96, 100, 70), 1, 1)])
def test_tmem_rings_bitwise(gpu, shape, precession, bc, monkeypatch):
    """The RK4 step with its older spin planes and accumulators in tensor
    memory (28-row tiles; SPIN_TMEM=1 forces it) gives bitwise the states of
    the register-ring step (SPIN_TMEM=0) over 20 steps with two pulses, on
    ragged, tiny and free-boundary lattices and both equations: the same
    arithmetic per site, only where the values wait between iterations
    differs."""
    nx, ny, nz = shape
    p = gpu.Params(nx, ny, nz, J=1.0, D=0.05, H=(0.01, -0.02, 0.02), lam=0.05, T=1.0, dt=0.1, R=10, seed=3,
                   precision=32, bc=bc, precession=precession)
    s0 = spin_inputs.random_spins(nx, ny, nz, seed=2)
    monkeypatch.setenv("SPIN_TMEM", "1")
    a, la = run_gpu(gpu, p, s0, 20)
    monkeypatch.setenv("SPIN_TMEM", "0")
    b, lb = run_gpu(gpu, p, s0, 20)
    monkeypatch.delenv("SPIN_TMEM", raising=False)
    la.close()
    lb.close()
    assert np.array_equal(a, b)


# ----------------------------------------------------------------- graph path, resume
@pytest.mark.parametrize("R", [10, 5, 1])
def test_graph_replay_equals_eager(gpu, R):
    """Whole intervals replayed from the cached CUDA graph give bitwise the
    same state and samples as step-by-step launches (odd R flips buffers)."""
    n = 24
    p = gpu.Params(n, n, n, J=1.0, D=0.05, H=(0, 0, 0.02), lam=0.05, T=1.0, dt=0.1, R=R, seed=5, precision=32)
    s0 = spin_inputs.random_spins(n, n, n, seed=2)
    a, la = run_gpu(gpu, p, s0, 5 * R)
    b, lb = run_gpu(gpu, p, s0, 5 * R, calls=[1] * (5 * R))
    assert np.array_equal(a, b)
    assert la.samples() == lb.samples()


def test_resume_is_bitwise(gpu):
    """Noise is a pure function of (seed, site, pulse number, replica): a run
    restarted from a saved state and step count reproduces the uninterrupted
    run bit for bit."""
    n = 20
    p = gpu.Params(n, n, n, J=1.0, D=0.05, H=(0, 0, 0.02), lam=0.05, T=1.0, dt=0.1, R=10, seed=5, precision=32)
    s0 = spin_inputs.random_spins(n, n, n, seed=2)
    full, _ = run_gpu(gpu, p, s0, 47)
    half, _ = run_gpu(gpu, p, s0, 23)
    lat = gpu.Lattice(p, torch.from_numpy(half))
    lat.set_step(23)
    lat.step(24)
    assert np.array_equal(gpu_state(lat), full)


# ----------------------------------------------------------------- full sizes, sampled
def _oracle_one_step_at(orc, p, s, sites, pulse, k):
    """One oracle step at sampled sites: the RK4 dependency cone of a site is
    its 9^3 neighbourhood, so each site's new value is the centre of a 9^3
    periodic oracle run on that neighbourhood, then renormalised and rotated by
    the noise of its global index."""
    nx, ny, nz = p.nx, p.ny, p.nz
    op9 = orc_params(orc, p)
    op9 = orc.Params(9, 9, 9, J=op9.J, D=op9.D, H=op9.H, lam=op9.lam, T=op9.T, dt=op9.dt, R=op9.R,
                     integrator=op9.integrator, precession=op9.precession, seed=op9.seed, replica=op9.replica)
    sig = orc.pulse_sigma(op9)
    out = []
    for (x, y, z) in sites:
        xs, ys, zs = (np.arange(c - 4, c + 5) % m for c, m in ((x, nx), (y, ny), (z, nz)))
        cube = s[:, zs][:, :, ys][:, :, :, xs]
        c1 = orc.renormalise(op9, orc.integrate(op9, cube))
        v = c1[:, 4, 4, 4].copy()
        if pulse:
            G = orc.noise_gauss(p.seed, x + nx * (y + ny * z), k, p.replica)
            v = orc.rotate(sig * G, v)
        out.append(v)
    return np.array(out)


@pytest.mark.parametrize("name", ["lattice128", "overdamped256"])
def test_full_size_sampled(gpu, orc, name):
    """The benchmark workloads at full size in the benchmark's launch
    configuration: 2000 sampled sites of a pulse step and of a plain step
    against the oracle; unit length everywhere."""
    w = spin_inputs.WORKLOADS[name]
    nx, ny, nz = w["n"]
    p = gpu.Params(nx, ny, nz, J=w["J"], D=w["D"], H=w["H"], lam=w["lam"], T=w["T"], dt=w["dt"], R=w["R"],
                   precession=w["precession"], seed=w["noise_seed"], precision=32)
    s0 = spin_inputs.random_spins(nx, ny, nz, seed=w["spin_seed"])
    lat = gpu.Lattice(p, torch.from_numpy(s0))
    R = p.R
    pulse_step = R // 2 if R > 1 else 1
    lat.step(pulse_step - 1)
    before = gpu_state(lat)
    lat.step(1)                     # the pulse step (pulse number 0)
    after = gpu_state(lat)
    g = np.random.default_rng(0)
    sites = list(zip(g.integers(0, nx, 2000), g.integers(0, ny, 2000), g.integers(0, nz, 2000)))
    ref = _oracle_one_step_at(orc, p, before, sites, True, 0)
    got = np.array([after[:, z, y, x] for (x, y, z) in sites])
    assert np.max(np.abs(got - ref)) < 2e-6
    lat.step(1)                     # a plain step
    after2 = gpu_state(lat)
    ref2 = _oracle_one_step_at(orc, p, after, sites, False, 0)
    got2 = np.array([after2[:, z, y, x] for (x, y, z) in sites])
    assert np.max(np.abs(got2 - ref2)) < 2e-6
    assert np.max(np.abs(np.sum(after2 ** 2, axis=0) - 1.0)) < 1e-6


# ----------------------------------------------------------------- failure detection
def test_nonfinite_spin_reported(gpu):
    """A NaN planted from the host is reported by the observables call."""
    n = 8
    p = gpu.Params(n, n, n, precision=32)
    s0 = spin_inputs.random_spins(n, n, n, seed=1)
    lat = gpu.Lattice(p, torch.from_numpy(s0))
    lat.state[1, 2, 3, 4] = float("nan")
    M, E, rc = gpu.spin_observables(lat.handle)
    assert rc == gpu.SPIN_ENONFINITE


def test_applicability_warning(gpu):
    """The 256^3 slow-equation workload has Lambda_N Delta t = 2.4 > 0.2
    (Eq. phi_condition): create succeeds and returns the warning status."""
    n = 4
    p = gpu.Params(n, n, n, lam=1.0, T=1.2, dt=0.2, R=5, precession=0, precision=32)
    lat = gpu.Lattice(p, torch.from_numpy(spin_inputs.random_spins(n, n, n, seed=1)))
    assert lat.status == gpu.SPIN_WARN_APPLICABILITY
    q = gpu.Params(n, n, n, lam=0.01, T=1.0, dt=0.2, R=10, precision=32)
    assert gpu.Lattice(q, torch.from_numpy(spin_inputs.random_spins(n, n, n, seed=1))).status == gpu.SPIN_OK


@pytest.mark.parametrize("bc", [0, 1])
def test_rk5_fused_trajectory(gpu, orc, bc):
    """Butcher RK5 in FP32 on the fused two-segment path, 40^3 (several tiles
    and z-chunks), dt = 0.15, pulses every 10 steps.  Each of the first 10
    steps, restarted in the oracle from the GPU state, within 5e-6 (measured
    3.5e-6 for this path and for the per-stage FP32 path alike); after 30
    steps the fused path, the per-stage FP32 path (forced path 1) and the
    oracle within 6e-5 of each other (measured 3.2e-5: the FP32 step error
    grows by about 10x over 30 steps, the same for both FP32 paths)."""
    n = 40
    kw = dict(J=1.0, D=0.05, H=(0.02, 0.0, 0.1), lam=0.05, T=0.9, dt=0.15, R=10, seed=21, integrator=gpu.RK5_BUTCHER,
              precision=32, bc=bc)
    p = gpu.Params(n, n, n, **kw)
    s0 = spin_inputs.random_spins(n, n, n, seed=5)
    lat = gpu.Lattice(p, torch.from_numpy(s0))
    cur = gpu_state(lat)
    worst = 0.0
    for step in range(10):
        lat.step(1)
        nxt = gpu_state(lat)
        ref1, _ = run_oracle(orc, p, cur, 1, n0=step)
        worst = max(worst, float(np.max(np.abs(nxt - ref1))))
        cur = nxt
    assert worst < 5e-6, worst
    lat.step(20)
    got = gpu_state(lat)
    per_stage, _ = run_gpu(gpu, gpu.Params(n, n, n, path=1, **kw), s0, 30)
    ref, smp = run_oracle(orc, p, s0, 30)
    assert np.max(np.abs(got - ref)) < 6e-5
    assert np.max(np.abs(per_stage - ref)) < 6e-5
    assert np.max(np.abs(got - per_stage)) < 6e-5
    rec = np.array(lat.samples())
    assert rec.shape == (3, 5) and np.max(np.abs(rec[:, 1:] - smp[:, 1:])) < 5e-6
