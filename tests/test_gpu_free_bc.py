"""Free boundary conditions (the paper's particle, Sec. IV) on the GPU against
the oracle: fused FP32 and FP64 steps, per-stage kernels, observables and the
adjoint; same tolerances as the periodic tests."""
import numpy as np
import pytest
import torch

import spin_inputs
from gpu_helpers import as_input, gpu_state, orc_params, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

CASES = [  # size, precision, integrator, precession, h_site, path
    ((16, 16, 16), 32, 0, 1, False, 0),
    ((37, 21, 13), 32, 0, 0, True, 0),
    ((2, 3, 5), 32, 0, 1, False, 0),
    ((1, 1, 1), 32, 0, 1, False, 0),
    ((20, 19, 18), 64, 0, 1, True, 0),
    ((20, 19, 18), 32, 2, 0, False, 0),
    ((20, 19, 18), 64, 1, 1, False, 0),
    ((11, 12, 7), 32, 0, 1, True, 1),
    # rows of 64 / 128 columns: no spin beyond the first and last column
    ((64, 19, 9), 32, 0, 1, False, 0),
    ((128, 9, 11), 32, 0, 0, False, 0),
    # Butcher RK5, fused two-segment FP32 path
    ((20, 19, 18), 32, 1, 1, False, 0),
    ((2, 3, 5), 32, 1, 0, False, 0),
    ((64, 19, 9), 32, 1, 1, False, 0),
    # RK4 on shapes that qualify for TMA staging (sides multiples of 4, x >= 24, y >= 16)
    ((24, 16, 9), 32, 0, 1, True, 0),
    ((52, 36, 10), 32, 0, 0, False, 0),
]


@pytest.mark.parametrize("shape,prec,integ,precession,hsite,path", CASES)
def test_three_steps_free(gpu, orc, shape, prec, integ, precession, hsite, path):
    nx, ny, nz = shape
    p = gpu.Params(nx, ny, nz, J=0.9, D=0.15, H=(0.05, -0.1, 0.2), lam=0.1, T=0.7, dt=0.07, R=3,
                   integrator=integ, precession=precession, seed=77, replica=2, precision=prec, path=path, bc=1)
    s0 = spin_inputs.random_spins(nx, ny, nz, seed=3)
    hs = spin_inputs.site_fields(nx, ny, nz, 0.1, seed=4) if hsite else None
    got, lat = run_gpu(gpu, p, s0, 3, h_site=hs)
    ref, smp = run_oracle(orc, p, s0, 3, h_site=hs)
    assert np.max(np.abs(got - ref)) < (1e-13 if prec == 64 else 2e-6)
    rec = lat.samples()
    assert np.max(np.abs(np.array(rec[0][1:]) - smp[0, 1:])) < (1e-13 if prec == 64 else 5e-6)


def test_trajectory_free_32cubed(gpu, orc):
    """32^3 free-boundary lattice, 20 steps with two pulses (FP32)."""
    n = 32
    p = gpu.Params(n, n, n, J=1.0, D=0.05, H=(0, 0, 0.05), lam=0.05, T=1.0, dt=0.1, R=10, seed=3, precision=32,
                   bc=1)
    s0 = spin_inputs.random_spins(n, n, n, seed=8)
    got, _ = run_gpu(gpu, p, s0, 20)
    ref, _ = run_oracle(orc, p, s0, 20)
    assert np.max(np.abs(got - ref)) < 1e-5


@pytest.mark.parametrize("prec", [64, 32])
def test_adjoint_free(gpu, orc, prec):
    shape = (6, 5, 4)
    p = gpu.Params(*shape, J=0.9, D=0.25, H=(0.05, -0.1, 0.2), lam=0.1, T=0.8, dt=0.1, R=4, seed=12,
                   precision=prec, bc=1)
    s0 = spin_inputs.random_spins(*shape, seed=11)
    hs = spin_inputs.site_fields(*shape, 0.1, seed=13)
    lat = gpu.Lattice(p, torch.from_numpy(s0), h_site=torch.from_numpy(hs))
    lat.record(8, 20)
    lat.step(20)
    g = lat.backward([0.3, -0.2, 0.7], 1.0, field_grad=True)
    ref = orc.adjoint(orc_params(orc, p), as_input(p, s0), 20, [0.3, -0.2, 0.7], 1.0, h_site=as_input(p, hs))
    # same bounds as the periodic adjoint tests (test_gpu_adjoint.py): FP32
    # 1e-5 of the largest entry and 2e-4 |r_i| + 1e-5 max|r| per element
    tol = 1e-9 if prec == 64 else 1e-5
    for key in ("J", "D", "H"):
        a, b = np.asarray(g[key], float), np.asarray(ref[key], float)
        assert np.max(np.abs(a - b)) / np.max(np.abs(b)) < tol, key
    hg = g["h"].cpu().numpy()
    assert np.max(np.abs(hg - ref["h"])) / np.max(np.abs(ref["h"])) < tol
    if prec == 32:
        r = ref["h"]
        assert np.all(np.abs(hg - r) <= 2e-4 * np.abs(r) + 1e-5 * np.max(np.abs(r)))
