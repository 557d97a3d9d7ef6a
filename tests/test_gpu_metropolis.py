"""GPU checkerboard Metropolis (spin_metropolis_sweeps) against the oracle's
checkerboard Metropolis (same trials, same counter-based random numbers,
Sec. IV's trial length and acceptance rule)."""
import numpy as np
import pytest
import torch

import spin_inputs
from gpu_helpers import as_input

pytestmark = pytest.mark.gpu


def _gpu_state(p, s):
    return torch.from_numpy(np.ascontiguousarray(as_input(p, s))).to("cuda", p.dtype)


CASES = [  # shape, bc, T, with h_site
    ((4, 6, 2), 0, 1.0, True),
    ((5, 3, 7), 1, 0.7, False),
    ((8, 8, 8), 0, 0.3, False),
    ((10, 4, 6), 0, 1.6, True),
    ((1, 1, 3), 1, 0.5, False),
]


@pytest.mark.parametrize("shape,bc,T,hsite", CASES)
def test_fp64_sweeps_match_oracle(gpu, orc, shape, bc, T, hsite):
    """FP64: after 3 + 4 sweeps (two calls) the state equals the oracle's to
    1e-12 and the accepted counts are equal."""
    nx, ny, nz = shape
    p = gpu.Params(nx, ny, nz, J=1.0, D=0.2, H=(0.05, -0.1, 0.3), T=T, bc=bc, replica=3, precision=64)
    s0 = spin_inputs.random_spins(nx, ny, nz, seed=5)
    hs = spin_inputs.site_fields(nx, ny, nz, 0.1, seed=6) if hsite else None
    st = _gpu_state(p, s0)
    hg = None if hs is None else _gpu_state(p, hs)
    acc = torch.zeros(1, dtype=torch.int64, device="cuda")
    gpu.spin_metropolis_sweeps(p, st, 3, mc_seed=77, h_site=hg, accepted=acc)
    gpu.spin_metropolis_sweeps(p, st, 4, mc_seed=77, sweep0=3, h_site=hg, accepted=acc)
    q = orc.Params(nx, ny, nz, J=1.0, D=0.2, H=(0.05, -0.1, 0.3), T=T, bc=bc, replica=3)
    ref, _, nacc = orc.metropolis_checkerboard(q, s0, 7, mc_seed=77, h_site=hs)
    got = st.cpu().numpy()
    assert np.max(np.abs(got - ref)) < 1e-12
    assert int(acc.item()) == nacc > 0


def test_fp32_half_sweeps_match_oracle(gpu, orc):
    """FP32 decides acceptance in FP32: half-sweep by half-sweep from the
    same state, the sites whose decision agrees match the oracle to 2e-6; a
    decision may differ only where dE/T + ln(u) is within FP32 rounding of 0,
    which happens at a rate ~1e-6 per trial (at most 2 of ~16k trials per
    half-sweep are allowed)."""
    n = 32
    p = gpu.Params(n, n, n, J=1.0, D=0.05, H=(0, 0, 0.02), T=1.0, precision=32)
    q = orc.Params(n, n, n, J=1.0, D=0.05, H=(0, 0, 0.02), T=1.0)
    st = _gpu_state(p, spin_inputs.random_spins(n, n, n, seed=9))
    z, y, x = np.indices((n, n, n))
    flips = 0
    for sweep in range(4):
        for color in (0, 1):
            before = st.double().cpu().numpy()
            ref, _ = orc.metropolis_color(q, before, sweep, color, mc_seed=13)
            gpu.spin_metropolis_color(p, st, sweep, color, mc_seed=13)
            got = st.double().cpu().numpy()
            moved_g = np.any(got != before, axis=0)
            moved_o = np.any(ref != before, axis=0)
            assert not np.any(moved_g & (((x + y + z) & 1) != color))
            differ = moved_g != moved_o
            assert int(differ.sum()) <= 2
            flips += int(differ.sum())
            assert np.max(np.abs((got - ref)[:, ~differ])) < 2e-6
            assert moved_g.sum() > 0.4 * n ** 3 / 2  # about half the trials accepted
    assert flips <= 4


def test_sweep_is_two_colours(gpu):
    n = 8
    p = gpu.Params(n, n, n, J=1.0, T=0.8, precision=64)
    s0 = _gpu_state(p, spin_inputs.random_spins(n, n, n, seed=2))
    a, b = s0.clone(), s0.clone()
    gpu.spin_metropolis_sweeps(p, a, 2, mc_seed=4, sweep0=5)
    for w in (5, 6):
        for c in (0, 1):
            gpu.spin_metropolis_color(p, b, w, c, mc_seed=4)
    assert torch.equal(a, b)


def test_rejects_odd_periodic_and_bad_arguments(gpu):
    p = gpu.Params(5, 4, 4, J=1.0, T=1.0, precision=32, bc=0)
    st = torch.zeros(3, 4, 4, 5, dtype=torch.float32, device="cuda")
    with pytest.raises(gpu.SpinError):
        gpu.spin_metropolis_sweeps(p, st, 1, mc_seed=1)
    q = gpu.Params(4, 4, 4, J=0.0, T=1.0, precision=32)  # paper's trial length needs J > 0
    st = torch.zeros(3, 4, 4, 4, dtype=torch.float32, device="cuda")
    with pytest.raises(gpu.SpinError):
        gpu.spin_metropolis_sweeps(q, st, 1, mc_seed=1)
    with pytest.raises(gpu.SpinError):
        gpu.spin_metropolis_color(gpu.Params(4, 4, 4, T=1.0), st, 0, 2, mc_seed=1)


def test_equilibrium_matches_sequential_oracle(gpu, orc):
    """8^3 periodic ferromagnet at T = 1: the GPU checkerboard chain (FP32,
    20000 sweeps) and the oracle's sequential chain (6000 sweeps) sample
    the same <|M|> and <E> within binned errors."""
    n = 8
    p = gpu.Params(n, n, n, J=1.0, T=1.0, precision=32)
    st = _gpu_state(p, spin_inputs.aligned_spins(n, n, n, (0, 0, 1.0)))
    gpu.spin_metropolis_sweeps(p, st, 1000, mc_seed=3)
    ms, es = [], []
    for k in range(200):
        gpu.spin_metropolis_sweeps(p, st, 100, mc_seed=3, sweep0=1000 + 100 * k)
        v = st.double()
        ms.append(float(v.mean(dim=(1, 2, 3)).norm()))
        E = 0.0
        for ax in (1, 2, 3):
            E -= float((v * torch.roll(v, 1, dims=ax)).sum())
        es.append(E / n ** 3)
    q = orc.Params(n, n, n, J=1.0, T=1.0)
    _, ser, _ = orc.metropolis(q, spin_inputs.aligned_spins(n, n, n, (0, 0, 1.0)), 6000, mc_seed=5)
    mo = np.linalg.norm(ser[1000:, :3], axis=1).reshape(50, -1).mean(1)
    eo = ser[1000:, 3].reshape(50, -1).mean(1)
    mg, eg = np.array(ms).reshape(50, -1).mean(1), np.array(es).reshape(50, -1).mean(1)
    dm = np.hypot(mo.std(), mg.std()) / np.sqrt(50)
    de = np.hypot(eo.std(), eg.std()) / np.sqrt(50)
    assert abs(mo.mean() - mg.mean()) < 4 * dm + 0.003, (mo.mean(), mg.mean(), dm)
    assert abs(eo.mean() - eg.mean()) < 4 * de + 0.005, (eo.mean(), eg.mean(), de)
