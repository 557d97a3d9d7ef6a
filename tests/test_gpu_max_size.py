"""The largest lattice the library accepts (N < 2^31 sites: 1290^3 =
2,146,689,000 sites, 25.8 GB per FP32 copy) in the benchmark's launch
configuration: a pulse step and a plain step at sampled sites against the
oracle (sites near the last index included, so the noise counter and every
offset run up to 2^31 - 1), unit length, and the FP64 observables against a
plain FP64 reduction of the same state in PyTorch."""
import numpy as np
import pytest
import torch

import spin_inputs
from gpu_helpers import orc_params

pytestmark = pytest.mark.gpu

L = 1290
NEED = 120 * 2 ** 30      # initial state, the lattice's copy, its workspace and temporaries


def _cubes(state, sites):
    """9^3 periodic neighbourhoods of the sites, gathered on the device: (n, 3, 9, 9, 9) float64."""
    dev = state.device
    nz, ny, nx = state.shape[1:]
    off = torch.arange(-4, 5, device=dev)
    out = []
    flat = state.reshape(3, -1)
    for (x, y, z) in sites:
        xs = (x + off) % nx
        ys = (y + off) % ny
        zs = (z + off) % nz
        idx = (zs[:, None, None] * ny + ys[None, :, None]) * nx + xs[None, None, :]
        out.append(flat[:, idx.reshape(-1)].reshape(3, 9, 9, 9))
    return torch.stack(out).double().cpu().numpy()


def _values(state, sites):
    nz, ny, nx = state.shape[1:]
    idx = torch.tensor([(z * ny + y) * nx + x for (x, y, z) in sites], device=state.device)
    return state.reshape(3, -1)[:, idx].double().cpu().numpy().T


def _oracle_step(orc, p, cubes, sites, pulse, k):
    q = orc_params(orc, p)
    q9 = orc.Params(9, 9, 9, J=q.J, D=q.D, H=q.H, lam=q.lam, T=q.T, dt=q.dt, R=q.R, integrator=q.integrator,
                    precession=q.precession, seed=q.seed, replica=q.replica)
    sig = orc.pulse_sigma(q9)
    out = []
    for cube, (x, y, z) in zip(cubes, sites):
        v = orc.renormalise(q9, orc.integrate(q9, cube))[:, 4, 4, 4].copy()
        if pulse:
            v = orc.rotate(sig * orc.noise_gauss(p.seed, x + L * (y + L * z), k, p.replica), v)
        out.append(v)
    return np.array(out)


def _torch_observables(s, p):
    """M and E per spin in FP64 by plain tensor operations, z-slab by z-slab
    (each bond once through the three forward neighbours)."""
    nz = s.shape[1]
    M = torch.zeros(3, dtype=torch.float64, device=s.device)
    E = torch.zeros((), dtype=torch.float64, device=s.device)
    H = torch.tensor(p.H, dtype=torch.float64, device=s.device)
    for z0 in range(0, nz, 32):
        z1 = min(nz, z0 + 32)
        c = s[:, z0:z1].double()
        zn = s[:, [(z + 1) % nz for z in range(z0, z1)]].double()
        nb = torch.roll(c, -1, dims=3) + torch.roll(c, -1, dims=2) + zn
        E -= p.J * (c * nb).sum()
        E -= p.D * (c[2] * c[2]).sum()
        E -= (c * H[:, None, None, None]).sum()
        M += c.sum(dim=(1, 2, 3))
        del c, zn, nb
    n = float(s.shape[1] * s.shape[2] * s.shape[3])
    return (M / n).cpu().numpy(), float(E / n)


def test_largest_lattice(gpu, orc):
    free, _ = torch.cuda.mem_get_info()
    if free < NEED:
        pytest.skip(f"needs {NEED / 2 ** 30:.0f} GiB of free device memory, {free / 2 ** 30:.0f} GiB free")
    w = spin_inputs.WORKLOADS["lattice128"]
    p = gpu.Params(L, L, L, J=w["J"], D=w["D"], H=w["H"], lam=w["lam"], T=w["T"], dt=w["dt"], R=w["R"],
                   precession=w["precession"], seed=w["noise_seed"], precision=32)
    s0 = spin_inputs.random_spins_device(L, L, L, seed=7)
    lat = gpu.Lattice(p, s0)
    del s0
    torch.cuda.empty_cache()
    g = np.random.default_rng(1)
    sites = [(L - 1, L - 1, L - 1), (0, 0, 0), (L - 1, 0, L - 1), (0, L - 1, L - 1), (L - 2, L - 1, L - 1)]
    sites += list(zip(g.integers(0, L, 195).tolist(), g.integers(0, L, 195).tolist(), g.integers(0, L, 195).tolist()))
    pulse_step = p.R // 2
    lat.step(pulse_step - 1)
    torch.cuda.synchronize()
    cubes = _cubes(lat.state, sites)
    lat.step(1)                                   # the pulse step (pulse number 0)
    torch.cuda.synchronize()
    got = _values(lat.state, sites)
    ref = _oracle_step(orc, p, cubes, sites, True, 0)
    assert np.max(np.abs(got - ref)) < 2e-6
    cubes = _cubes(lat.state, sites)
    lat.step(1)                                   # a plain step
    torch.cuda.synchronize()
    got = _values(lat.state, sites)
    ref = _oracle_step(orc, p, cubes, sites, False, 0)
    assert np.max(np.abs(got - ref)) < 2e-6
    n2 = (lat.state * lat.state).sum(dim=0)
    assert float((n2 - 1.0).abs().max()) < 1e-6
    del n2
    M, E = lat.observables()
    Mt, Et = _torch_observables(lat.state, p)
    assert np.max(np.abs(np.array(M) - Mt)) < 1e-6
    assert abs(E - Et) < 5e-6
    lat.close()
    del lat
    torch.cuda.empty_cache()
