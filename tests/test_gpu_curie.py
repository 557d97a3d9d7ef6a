"""The bulk Curie temperature the paper quotes for the simple-cubic classical
Heisenberg ferromagnet (Sec. IV: T_c/J = 1.444), as a check of the many-spin
Hamiltonian's convention (each bond counted once; counting bonds twice would
put T_c near 2.9): Binder cumulants U4 = 1 - <m^4> / (3 <m^2>^2) of the GPU
checkerboard Metropolis (which matches the oracle's sweeps) grow with the
lattice size below T_c and fall with it above.  Measured: at T = 1.41
U4(L=12) = 0.645 +- 0.002, U4(L=24) = 0.661 +- 0.0003; at T = 1.47
0.593 +- 0.006 and 0.536 +- 0.011, so the curves cross between 1.41 and 1.47."""
import numpy as np
import pytest
import torch

import spin_inputs

pytestmark = pytest.mark.gpu


def _binder(gpu, L, T, sweeps=12000, every=2, therm=2000):
    p = gpu.Params(L, L, L, J=1.0, T=T, precision=32)
    st = torch.from_numpy(spin_inputs.random_spins(L, L, L, seed=L)).to("cuda", torch.float32).contiguous()
    seed = L * 100 + int(round(T * 100))
    gpu.spin_metropolis_sweeps(p, st, therm, mc_seed=seed)
    m2, w = [], therm
    for _ in range(sweeps // every):
        gpu.spin_metropolis_sweeps(p, st, every, mc_seed=seed, sweep0=w)
        w += every
        m = st.mean(dim=(1, 2, 3))
        m2.append((m * m).sum())
    a = torch.stack(m2).double().cpu().numpy()
    u4 = 1.0 - np.mean(a * a) / (3.0 * np.mean(a) ** 2)
    bins = [1.0 - np.mean(x * x) / (3.0 * np.mean(x) ** 2) for x in a.reshape(30, -1)]
    return u4, np.std(bins) / np.sqrt(30)


def test_binder_cumulants_bracket_the_quoted_curie_temperature(gpu):
    lo12, e_lo12 = _binder(gpu, 12, 1.41)
    lo24, e_lo24 = _binder(gpu, 24, 1.41)
    hi12, e_hi12 = _binder(gpu, 12, 1.47)
    hi24, e_hi24 = _binder(gpu, 24, 1.47)
    assert lo24 - lo12 > 3 * np.hypot(e_lo12, e_lo24), (lo12, lo24)   # ordered side: T_c > 1.41
    assert hi12 - hi24 > 3 * np.hypot(e_hi12, e_hi24), (hi12, hi24)   # disordered side: T_c < 1.47
