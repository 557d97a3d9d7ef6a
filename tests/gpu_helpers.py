"""Shared helpers of the GPU parity tests: run the CUDA path through the C-ABI
and the oracle on the same seeded inputs."""
import numpy as np
import torch


def orc_params(orc, p, **over):
    """Oracle parameters for the same problem as GPU parameters p."""
    kw = dict(J=p.J, D=p.D, H=tuple(p.H), lam=p.lam, T=p.T, dt=p.dt, R=p.R,
              integrator=p.integrator, precession=p.precession, renorm=p.renorm,
              seed=p.seed, replica=p.replica, bc=p.bc)
    kw.update(over)
    return orc.Params(p.nx, p.ny, p.nz, **kw)


def as_input(p, s):
    """The exact values the GPU receives (rounded to float32 for precision 32)."""
    a = np.asarray(s, dtype=np.float64)
    if p.precision == 32:
        a = a.astype(np.float32).astype(np.float64)
    return a.reshape(3, p.nz, p.ny, p.nx)


def gpu_state(lat):
    torch.cuda.synchronize()
    return lat.state.double().cpu().numpy()


def run_gpu(sp, p, s0, nsteps, h_site=None, calls=None):
    lat = sp.Lattice(p, torch.from_numpy(np.ascontiguousarray(s0)), h_site=None if h_site is None else torch.from_numpy(h_site))
    if calls is None:
        lat.step(nsteps)
    else:
        for c in calls:
            lat.step(c)
    return gpu_state(lat), lat


def run_oracle(orc, p, s0, nsteps, h_site=None, n0=0):
    op = orc_params(orc, p)
    return orc.run(op, as_input(p, s0), nsteps, n0=n0, h_site=None if h_site is None else as_input(p, h_site),
                   noise=bool(p.noise))
