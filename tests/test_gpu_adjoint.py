"""GPU checkpointed adjoint (spin_backward through the C-ABI) against the
oracle's own discrete adjoint on identical inputs and noise.

Tolerances.  FP64 state: the GPU recomputes the same steps, so gradients agree
to rounding (relative 1e-9 of each gradient's largest entry).  FP32 state and
adjoint against the FP64 oracle: every forward stage and every transposed
stage rounds its result to float (relative 2^-24 = 6e-8), so over 20 steps of
4 stages the gradients carry at most ~80 such roundings, accumulated
linearly: ~5e-6 of the largest entry.  The bound used is 1e-5 (the measured
errors over these cases are 1e-8..5.4e-7 for J, D, H and 6e-7..1.9e-6 for
dL/dh_i and dL/ds_0).  dL/dh_i and dL/ds_0 are also checked element by element:
|g_i - r_i| <= 2e-4 |r_i| + 1e-5 max|r| (measured: at most 6e-5 |r_i| +
6e-7 max|r|), so a dropped term that is small against the largest entry but
not against its own element fails."""
import numpy as np
import pytest
import torch

import spin_inputs
from gpu_helpers import as_input, orc_params

pytestmark = pytest.mark.gpu


def _rel(a, b):
    a, b = np.asarray(a, dtype=float), np.asarray(b, dtype=float)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


TOL32 = 1e-5


def _elementwise_ok(a, b, rtol=2e-4, atol_rel=1e-5):
    """|a_i - b_i| <= rtol |b_i| + atol_rel max|b| for every element."""
    a, b = np.asarray(a, dtype=float).ravel(), np.asarray(b, dtype=float).ravel()
    return bool(np.all(np.abs(a - b) <= rtol * np.abs(b) + atol_rel * np.max(np.abs(b))))


CASES = [  # precision, integrator, precession, K
    (64, 0, 1, 8), (64, 1, 1, 8), (64, 0, 0, 5), (64, 3, 1, 20),
    (32, 0, 1, 8), (32, 2, 0, 8), (32, 1, 1, 4),
]


@pytest.mark.parametrize("prec,integ,precession,K", CASES)
def test_adjoint_matches_oracle(gpu, orc, prec, integ, precession, K):
    shape = (6, 5, 4)
    nsteps = 20
    p = gpu.Params(*shape, J=0.9, D=0.25, H=(0.05, -0.1, 0.2), lam=0.1, T=0.8, dt=0.1, R=4, integrator=integ,
                   precession=precession, seed=12, precision=prec)
    s0 = spin_inputs.random_spins(*shape, seed=11)
    hs = spin_inputs.site_fields(*shape, 0.1, seed=13)
    lat = gpu.Lattice(p, torch.from_numpy(s0), h_site=torch.from_numpy(hs))
    lat.record(K, nsteps)
    lat.step(nsteps)
    dLdM, dLdE = [0.3, -0.2, 0.7], 1.0
    g = lat.backward(dLdM, dLdE, field_grad=True, state_grad=True)
    ref = orc.adjoint(orc_params(orc, p), as_input(p, s0), nsteps, dLdM, dLdE, h_site=as_input(p, hs))
    tol = 1e-9 if prec == 64 else TOL32
    assert _rel(g["J"], ref["J"]) < tol
    assert _rel(g["D"], ref["D"]) < tol
    assert _rel(g["H"], ref["H"]) < tol
    assert _rel(g["h"].cpu().numpy(), ref["h"]) < tol
    assert _rel(g["s0"].double().cpu().numpy(), ref["s0"]) < tol
    if prec == 32:
        assert _elementwise_ok(g["h"].cpu().numpy(), ref["h"])
        assert _elementwise_ok(g["s0"].double().cpu().numpy(), ref["s0"])


def test_adjoint_full_size_64cubed(gpu, orc):
    """The 64^3 differentiation workload (J=1, D=0.05, h_i ~ N(0, 0.01^2),
    lambda=0.05, T=0.8, RK4 dt=0.1, pulses every 10 steps, FP32 forward, FP64
    gradient accumulation) over 10 steps with checkpoints every 5, against the
    oracle's adjoint at full size; loss E + |M - m*|^2, m* = (0, 0, 0.5)."""
    w = spin_inputs.WORKLOADS["adjoint64"]
    nx, ny, nz = w["n"]
    p = gpu.Params(nx, ny, nz, J=w["J"], D=w["D"], H=w["H"], lam=w["lam"], T=w["T"], dt=w["dt"], R=w["R"],
                   seed=w["noise_seed"], precision=32)
    s0 = spin_inputs.random_spins(nx, ny, nz, seed=w["spin_seed"])
    hs = spin_inputs.site_fields(nx, ny, nz, w["field_sigma"], seed=w["noise_seed"])
    nsteps = 10
    lat = gpu.Lattice(p, torch.from_numpy(s0), h_site=torch.from_numpy(hs))
    lat.record(5, nsteps)
    lat.step(nsteps)
    M, E = lat.observables()
    dLdM = [2.0 * (M[a] - w["m_target"][a]) for a in range(3)]
    g = lat.backward(dLdM, 1.0, field_grad=True)
    ref = orc.adjoint(orc_params(orc, p), as_input(p, s0), nsteps, dLdM, 1.0, h_site=as_input(p, hs))
    assert _rel(g["J"], ref["J"]) < TOL32
    assert _rel(g["D"], ref["D"]) < TOL32
    assert _rel(g["H"], ref["H"]) < TOL32
    assert _rel(g["h"].cpu().numpy(), ref["h"]) < TOL32
    assert _elementwise_ok(g["h"].cpu().numpy(), ref["h"])


def test_autograd_function(gpu):
    """SpinRunFn wraps the forward run and spin_backward as a
    torch.autograd.Function: its gradients w.r.t. J, D, H and h equal the
    direct call's, and dL/dH is the sum of dL/dh_i."""
    shape = (8, 8, 8)
    p = gpu.Params(*shape, J=1.0, D=0.05, H=(0, 0, 0), lam=0.05, T=0.8, dt=0.1, R=10, seed=5, precision=32)
    s0 = torch.from_numpy(spin_inputs.random_spins(*shape, seed=5)).float().cuda()
    hs = torch.from_numpy(spin_inputs.site_fields(*shape, 0.01, seed=5)).float().cuda()
    J = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    D = torch.tensor(0.05, dtype=torch.float64, requires_grad=True)
    H = torch.tensor([0.01, -0.02, 0.03], dtype=torch.float64, requires_grad=True)
    h = hs.clone().requires_grad_(True)
    E, M = gpu.SpinRunFn.apply(J, D, H, h, s0, p, 30, 10)
    m_target = torch.tensor([0.0, 0.0, 0.5], dtype=torch.float64, device=M.device)
    loss = E + ((M - m_target) ** 2).sum()
    loss.backward()
    import dataclasses
    lat = gpu.Lattice(dataclasses.replace(p, H=(0.01, -0.02, 0.03)), s0, h_site=hs)
    lat.record(10, 30)
    lat.step(30)
    Md, Ed = lat.observables()
    assert abs(Ed - E.item()) < 1e-12
    dLdM = [2.0 * (Md[a] - [0.0, 0.0, 0.5][a]) for a in range(3)]
    g = lat.backward(dLdM, 1.0)
    assert abs(J.grad.item() - g["J"]) <= 1e-12 * max(1.0, abs(g["J"]))
    assert abs(D.grad.item() - g["D"]) <= 1e-12 * max(1.0, abs(g["D"]))
    for a in range(3):
        assert abs(H.grad[a].item() - g["H"][a]) <= 1e-12 * max(1.0, abs(g["H"][a]))
    assert torch.allclose(h.grad.double(), g["h"].float().double(), rtol=1e-6, atol=1e-9)
    # dL/dH = sum_i dL/dh_i (the uniform field enters H_eff like every h_i)
    hsum = g["h"].reshape(3, -1).sum(dim=1).cpu().numpy()
    assert np.max(np.abs(hsum - np.array(g["H"]))) <= 1e-9 * max(1.0, float(np.max(np.abs(hsum))))
