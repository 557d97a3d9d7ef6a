"""spin_observables_noalloc: the observables of caller-owned arrays for callers
that cannot allocate device memory where they need M and E (a fixed memory
budget, a thread that must not enter the allocator, a plug-in handed only
existing arrays).  Its reduction scratch is a file-scope device array inside
the library, so the call allocates nothing.

Checked through the C-ABI against the handle-based spin_observables, on two
calls in a row (the shared scratch keeps the previous call's contents).  This
file is collected last so that a stop-at-first-failure run has already run
every other test."""
import numpy as np
import pytest
import torch

import spin_inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("with_field", [False, True])
@pytest.mark.parametrize("bc", [0, 1])
def test_noalloc_matches_handle_observables(gpu, prec, with_field, bc):
    shapes = [(16, 16, 16), (37, 21, 13)]
    for call, (nx, ny, nz) in enumerate(shapes):      # two calls in a row, different sizes
        p = gpu.Params(nx, ny, nz, J=0.8, D=0.3, H=(0.1, -0.2, 0.3), precision=prec, bc=bc)
        s0 = spin_inputs.random_spins(nx, ny, nz, seed=20 + call)
        hs = spin_inputs.site_fields(nx, ny, nz, 0.2, seed=30 + call) if with_field else None
        lat = gpu.Lattice(p, torch.from_numpy(s0), h_site=None if hs is None else torch.from_numpy(hs))
        M, E = lat.observables()
        out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
        gpu.spin_observables_noalloc(lat.state, p.J, p.D, p.H, out, h_site=lat.h_site, bc=bc)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        assert np.max(np.abs(o[:3] - np.array(M))) < 1e-13
        assert abs(o[3] - E) < 1e-13
        assert o[4] == 0.0
        lat.close()


def test_noalloc_wrapper_rejects_bad_tensors(gpu):
    """The Python wrapper refuses tensors whose dtype, shape, layout or device
    would make the kernel read or write outside them."""
    s = torch.zeros((3, 4, 4, 4), device="cuda")
    ok = torch.zeros(5, dtype=torch.float64, device="cuda")
    bad = [
        dict(state=s, out5=torch.zeros(5, dtype=torch.float32, device="cuda")),
        dict(state=s, out5=torch.zeros(4, dtype=torch.float64, device="cuda")),
        dict(state=s, out5=torch.zeros(5, dtype=torch.float64)),
        dict(state=s.half(), out5=ok),
        dict(state=s.cpu(), out5=ok),
        dict(state=s.transpose(1, 3), out5=ok),
        dict(state=s[0], out5=ok),
        dict(state=s, out5=ok, h_site=torch.zeros((3, 4, 4, 4), dtype=torch.float64, device="cuda")),
        dict(state=s, out5=ok, h_site=torch.zeros((3, 4, 4), device="cuda")),
        dict(state=s, out5=ok, bc=2),
    ]
    for kw in bad:
        with pytest.raises(ValueError):
            gpu.spin_observables_noalloc(J=1.0, D=0.0, H=(0, 0, 0), **kw)


def test_noalloc_rejects_beyond_maximum(gpu):
    from paper_1610_04914_gb300 import _binding as B
    L = B.load()
    x = torch.zeros(4, device="cuda")
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    H = (B.ctypes.c_double * 3)(0, 0, 0)
    big = 2048  # 2048^3 sites > SPIN_NOALLOC_MAX_SITES
    rc = L.spin_observables_noalloc(32, x.data_ptr(), x.data_ptr(), x.data_ptr(), None, big, big, big,
                                    1.0, 0.0, H, 0, out.data_ptr(), None)
    assert rc == B.SPIN_EINVAL
    rc = L.spin_observables_noalloc(32, x.data_ptr(), x.data_ptr(), x.data_ptr(), None, 0, 1, 1,
                                    1.0, 0.0, H, 0, out.data_ptr(), None)
    assert rc == B.SPIN_EINVAL
    rc = L.spin_observables_noalloc(32, x.data_ptr(), x.data_ptr(), x.data_ptr(), None, 1, 1, 1,
                                    1.0, 0.0, H, 3, out.data_ptr(), None)
    assert rc == B.SPIN_EINVAL
