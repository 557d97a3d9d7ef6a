"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the
benchmark.

This module only draws inputs (initial spin fields, per-site random fields,
replica sizes and temperatures) and states the workload parameters.  It holds
none of the method's arithmetic and imports neither the oracle nor the GPU
library.  Every draw uses numpy's Philox-based ``Generator`` with an explicit
seed, so a given seed gives the same array on every machine.

Workloads (the paper's lattice set-up of Sec. IV with periodic boundaries;
units J = gamma = mu0 = 1):

* ``small_fp64``   16^3, J=1, D=0, H=(0,0,0.1), lambda=0.1, T=1, RK4 dt=0.1, R=10
* ``lattice128``   128^3, J=1, D=0.05, H=(0,0,0.02), lambda=0.01, T in {0.5,1,1.4},
                   RK4 dt=0.2, R=10, spins seed 2
* ``overdamped256`` 256^3 slow equation, J=1, D=0, H=(0,0,0.01), lambda=1, T=1.2,
                   dt=0.2, R=5, spins seed 3
* ``batch512``     512 replicas, L in {16,24,32,48,64}, T in [0.2, 2], D=0.02, H=0,
                   lambda=0.02, RK4 dt=0.2, R=10, seed 4
* ``adjoint64``    64^3, J=1, D=0.05, h_i ~ N(0, 0.01^2) per component (seed 5),
                   lambda=0.05, T=0.8, RK4 dt=0.1, R=10, checkpoint every 50 steps
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[seed & 0xFFFFFFFFFFFFFFFF, stream]))


def random_spins(nx: int, ny: int, nz: int, seed: int, stream: int = 0) -> np.ndarray:
    """Unit vectors uniform on the sphere, shape (3, nz, ny, nx), float64.

    z = 2u - 1 and azimuth 2 pi u' with u, u' uniform on [0, 1)."""
    g = _rng(seed, stream)
    n = nx * ny * nz
    cz = 2.0 * g.random(n) - 1.0
    ph = 2.0 * np.pi * g.random(n)
    st = np.sqrt(np.maximum(0.0, 1.0 - cz * cz))
    s = np.stack([st * np.cos(ph), st * np.sin(ph), cz])
    return s.reshape(3, nz, ny, nx)


def random_spins_device(nx: int, ny: int, nz: int, seed: int, device="cuda", chunk_planes: int = 64):
    """Unit vectors uniform on the sphere drawn directly in device memory as a
    float32 tensor (3, nz, ny, nx), for lattices too large to draw on the
    host: z = 2u - 1 and azimuth 2 pi u' from torch's seeded generator on the
    device, chunk by chunk along z (same recipe as ``random_spins``, another
    random stream)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    s = torch.empty((3, nz, ny, nx), dtype=torch.float32, device=device)
    for z0 in range(0, nz, chunk_planes):
        z1 = min(nz, z0 + chunk_planes)
        shape = (z1 - z0, ny, nx)
        cz = 2.0 * torch.rand(shape, generator=g, device=device, dtype=torch.float64) - 1.0
        ph = 2.0 * np.pi * torch.rand(shape, generator=g, device=device, dtype=torch.float64)
        st = torch.sqrt(torch.clamp(1.0 - cz * cz, min=0.0))
        s[0, z0:z1] = (st * torch.cos(ph)).float()
        s[1, z0:z1] = (st * torch.sin(ph)).float()
        s[2, z0:z1] = cz.float()
    return s


def aligned_spins(nx: int, ny: int, nz: int, direction=(0.0, 0.0, 1.0)) -> np.ndarray:
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    return np.broadcast_to(d[:, None, None, None], (3, nz, ny, nx)).copy()


def site_fields(nx: int, ny: int, nz: int, sigma: float, seed: int, stream: int = 1) -> np.ndarray:
    """Per-site random field h_i with independent N(0, sigma^2) components."""
    g = _rng(seed, stream)
    return (sigma * g.standard_normal(3 * nx * ny * nz)).reshape(3, nz, ny, nx)


def replica_draws(nrep: int, seed: int, sizes=(16, 24, 32, 48, 64), Tmin=0.2, Tmax=2.0):
    """Replica lattice sizes (uniform over ``sizes``) and temperatures (uniform
    in [Tmin, Tmax]), drawn in replica order."""
    g = _rng(seed, 2)
    L = np.array([sizes[i] for i in g.integers(0, len(sizes), nrep)], dtype=np.int32)
    T = Tmin + (Tmax - Tmin) * g.random(nrep)
    return L, T


WORKLOADS = {
    "small_fp64": dict(n=(16, 16, 16), J=1.0, D=0.0, H=(0.0, 0.0, 0.1), lam=0.1, T=1.0,
                       dt=0.1, R=10, spin_seed=0, noise_seed=1, steps=2000, precision=64,
                       precession=1),
    "lattice128": dict(n=(128, 128, 128), J=1.0, D=0.05, H=(0.0, 0.0, 0.02), lam=0.01,
                       T=1.0, Ts=(0.5, 1.0, 1.4), dt=0.2, R=10, spin_seed=2, noise_seed=2,
                       steps=10000, precision=32, precession=1),
    "overdamped256": dict(n=(256, 256, 256), J=1.0, D=0.0, H=(0.0, 0.0, 0.01), lam=1.0,
                          T=1.2, dt=0.2, R=5, spin_seed=3, noise_seed=3, steps=2000,
                          precision=32, precession=0),
    "batch512": dict(nrep=512, J=1.0, D=0.02, H=(0.0, 0.0, 0.0), lam=0.02, dt=0.2, R=10,
                     seed=4, steps=5000, precision=32, precession=1),
    "adjoint64": dict(n=(64, 64, 64), J=1.0, D=0.05, H=(0.0, 0.0, 0.0), lam=0.05, T=0.8,
                      dt=0.1, R=10, spin_seed=5, noise_seed=5, field_sigma=0.01, steps=500,
                      checkpoint=50, precision=32, precession=1, m_target=(0.0, 0.0, 0.5)),
}
