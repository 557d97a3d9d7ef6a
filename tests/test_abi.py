"""The C-ABI library builds, loads and exports every entry point declared in
include/*.h (no compute calls: runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?(?:int|void|char|size_t|double)\s*\*?\s*(spin_\w+)\s*\(", text, re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1610_04914_gb300 import build as b
    path = b.build()
    return ctypes.CDLL(path)


def test_header_declares_the_four_calls():
    names = declared_symbols()
    for n in ("spin_lattice_create", "spin_step_pulse", "spin_observables", "spin_backward"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(declared_symbols()) if not hasattr(lib, n)]
    assert not missing, missing


def test_params_struct_layout_matches_header():
    from paper_1610_04914_gb300._binding import spin_params
    # 12 int32 fields, 8 doubles, 1 uint64
    assert ctypes.sizeof(spin_params) == 12 * 4 + 8 * 8 + 8
    assert spin_params.J.offset == 48


def test_validation_without_gpu(lib):
    """Parameter validation is host logic and runs without a device."""
    import paper_1610_04914_gb300 as sp
    from paper_1610_04914_gb300 import _binding as B
    L = B.load()
    p = sp.Params(16, 16, 16)
    n = ctypes.c_size_t()
    assert L.spin_workspace_size(ctypes.byref(p.c()), ctypes.byref(n)) == 0
    assert n.value >= 3 * 4 * 16 ** 3
    for bad in (dict(nx=0), dict(precision=16), dict(R=0), dict(dt=0.0), dict(lam=-1.0), dict(integrator=9)):
        q = sp.Params(**{**dict(nx=16, ny=16, nz=16), **bad})
        assert L.spin_workspace_size(ctypes.byref(q.c()), ctypes.byref(n)) == B.SPIN_EINVAL
    assert L.spin_workspace_size(None, ctypes.byref(n)) == B.SPIN_EINVAL
    # the largest lattice: N < 2^31 sites (1290^3 = 2146689000 is accepted)
    assert L.spin_workspace_size(ctypes.byref(sp.Params(1290, 1290, 1290).c()), ctypes.byref(n)) == 0
    assert n.value >= 3 * 4 * 1290 ** 3
    assert L.spin_workspace_size(ctypes.byref(sp.Params(1290, 1290, 1291).c()), ctypes.byref(n)) == B.SPIN_EINVAL
    assert L.spin_step_pulse(None, 1) == B.SPIN_EINVAL
    assert L.spin_strerror(B.SPIN_ENONFINITE).decode().startswith("non-finite")


def test_generic_path_needs_more_workspace():
    import paper_1610_04914_gb300 as sp
    fused = sp.spin_workspace_size(sp.Params(32, 32, 32, integrator=sp.RK4))
    generic = sp.spin_workspace_size(sp.Params(32, 32, 32, integrator=sp.RK5_BUTCHER))
    assert generic >= fused + 7 * 3 * 4 * 32 ** 3


def test_backward_workspace_holds_the_stage_store_when_it_applies(lib):
    """The adjoint keeps a checkpoint segment's stage inputs, stage neighbour
    sums and unnormalised RK results (2 x stages x K arrays of 3N) only for
    FP32 chain tableaus on the fused path and while they take at most 8 GiB
    (host logic, no device)."""
    import paper_1610_04914_gb300 as sp

    def ws(**kw):
        q = {**dict(nx=64, ny=64, nz=64, integrator=sp.RK4, precision=32), **kw}
        K = q.pop("K", 50)
        return sp.spin_backward_workspace_size(sp.Params(q.pop("nx"), q.pop("ny"), q.pop("nz"), **q), K)

    arr = lambda n, elt: (3 * n * elt + 255) // 256 * 256
    n64 = 64 ** 3
    base32 = ws(path=1)                          # per-stage forward path: no stage store
    assert ws() - base32 == 8 * 50 * arr(n64, 4)
    assert ws(K=10) - ws(K=10, path=1) == 8 * 10 * arr(n64, 4)
    assert ws(integrator=sp.RK2_MIDPOINT) - ws(integrator=sp.RK2_MIDPOINT, path=1) == 4 * 50 * arr(n64, 4)
    assert ws(precision=64) == ws(precision=64, path=1)                     # FP64: stages recomputed
    assert ws(integrator=sp.RK5_BUTCHER) == ws(integrator=sp.RK5_BUTCHER, path=1)   # not a chain tableau
    big = dict(nx=256, ny=256, nz=256)                # 8 x 50 x 201 MB > 8 GiB
    assert ws(**big) == ws(**big, path=1)
