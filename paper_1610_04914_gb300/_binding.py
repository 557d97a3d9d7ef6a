"""ctypes binding of ``libspinpulse.so`` (declared in include/spinpulse.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Loading fails loudly when the library has not been built; there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libspinpulse.so")

SPIN_OK = 0
SPIN_WARN_APPLICABILITY = 1
SPIN_EINVAL = -1
SPIN_ECUDA = -2
SPIN_ENONFINITE = -3
SPIN_ETIMEOUT = -4
SPIN_EUNSUPPORTED = -5
SPIN_ENOSPACE = -6
SPIN_SAMPLE_RING = 4096
SPIN_NOALLOC_MAX_BLOCKS = 1024
SPIN_BATCH_SAMPLE_RING = 512
SPIN_NOALLOC_MAX_SITES = 2147483647

RK4, RK5_BUTCHER, RK2_MIDPOINT, HEUN = 0, 1, 2, 3


class SpinError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"spinpulse error {code}: {msg}")
        self.code = code


class spin_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("integrator", ctypes.c_int32),
        ("precession", ctypes.c_int32), ("steps_per_pulse", ctypes.c_int32),
        ("renorm", ctypes.c_int32), ("noise", ctypes.c_int32), ("replica", ctypes.c_int32),
        ("path", ctypes.c_int32), ("bc", ctypes.c_int32),
        ("J", ctypes.c_double), ("D", ctypes.c_double), ("H", ctypes.c_double * 3),
        ("lambda_", ctypes.c_double), ("T", ctypes.c_double), ("dt", ctypes.c_double),
        ("seed", ctypes.c_uint64),
    ]


EXPORTS = [
    "spin_workspace_size", "spin_lattice_create", "spin_step_pulse", "spin_observables",
    "spin_samples", "spin_get_step", "spin_set_step", "spin_lattice_destroy", "spin_strerror",
    "spin_last_error", "spin_noise_draw", "spin_observables_noalloc", "spin_record_store_size",
    "spin_record_begin", "spin_record_end", "spin_backward_workspace_size", "spin_backward",
    "spin_batch_offsets", "spin_batch_workspace_size", "spin_batch_create", "spin_batch_tuning",
    "spin_batch_tile_rows", "spin_batch_tiling", "spin_batch_set_tiling", "spin_batch_autotune",
    "spin_batch_step_pulse", "spin_batch_observables", "spin_batch_samples", "spin_batch_destroy",
    "spin_batch_last_error", "spin_single_prepare", "spin_single_run", "spin_single_escape", "spin_metropolis_sweeps", "spin_metropolis_color",
]

_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises if it is missing: build it first)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} not found: build it with paper_1610_04914_gb300.build.build() "
                           "(there is no CPU fallback)")
    L = ctypes.CDLL(path)
    P, vp = ctypes.POINTER, ctypes.c_void_p
    i32, i64, u64, sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_size_t
    L.spin_workspace_size.argtypes = [P(spin_params), P(sz)]
    L.spin_lattice_create.argtypes = [P(spin_params), vp, vp, vp, vp, vp, sz, vp, P(vp)]
    L.spin_step_pulse.argtypes = [vp, i64]
    L.spin_observables.argtypes = [vp, P(ctypes.c_double), P(ctypes.c_double)]
    L.spin_samples.argtypes = [vp, P(ctypes.c_double), i64, P(i64)]
    L.spin_get_step.argtypes = [vp, P(i64)]
    L.spin_set_step.argtypes = [vp, i64]
    L.spin_lattice_destroy.argtypes = [vp]
    L.spin_strerror.argtypes = [ctypes.c_int]
    L.spin_strerror.restype = ctypes.c_char_p
    L.spin_last_error.argtypes = [vp]
    L.spin_last_error.restype = ctypes.c_char_p
    L.spin_noise_draw.argtypes = [u64, i64, i64, i64, i32, vp, vp, vp]
    d = ctypes.c_double
    L.spin_observables_noalloc.argtypes = [i32, vp, vp, vp, vp, i32, i32, i32, d, d, P(d), i32, vp, vp]
    L.spin_record_store_size.argtypes = [P(spin_params), i32, i64, P(sz)]
    L.spin_record_begin.argtypes = [vp, i32, i64, vp, sz]
    L.spin_record_end.argtypes = [vp]
    L.spin_backward_workspace_size.argtypes = [P(spin_params), i32, P(sz)]
    L.spin_backward.argtypes = [vp, P(d), d, vp, sz, P(d), P(d), P(d), vp, vp]
    L.spin_batch_offsets.argtypes = [i32, P(i32), P(i64)]
    L.spin_batch_workspace_size.argtypes = [P(spin_params), i32, P(i32), P(sz)]
    L.spin_batch_create.argtypes = [P(spin_params), i32, P(i32), P(d), vp, vp, vp, i32, vp, sz, vp, P(vp)]
    L.spin_batch_tuning.argtypes = [vp, P(i32), P(i32)]
    L.spin_batch_tile_rows.argtypes = [i32, i32, P(i32), P(i32)]
    L.spin_batch_tiling.argtypes = [vp, i32, P(i32), P(i32), P(i32), P(i32)]
    L.spin_batch_set_tiling.argtypes = [vp, i32, P(i32), P(i32), P(i32)]
    L.spin_batch_autotune.argtypes = [vp]
    L.spin_batch_step_pulse.argtypes = [vp, i64]
    L.spin_batch_observables.argtypes = [vp, P(d)]
    L.spin_batch_samples.argtypes = [vp, P(d), i64, P(i64)]
    L.spin_batch_destroy.argtypes = [vp]
    L.spin_metropolis_sweeps.argtypes = [P(spin_params), vp, vp, u64, d, i64, i64, vp, vp]
    L.spin_metropolis_color.argtypes = [P(spin_params), vp, vp, u64, d, i64, i32, vp, vp]
    L.spin_single_prepare.argtypes = [P(spin_params), i32, P(d), P(d), vp, vp]
    L.spin_single_run.argtypes = [P(spin_params), i32, vp, vp, i64, i64, i32, vp, vp, vp, vp]
    L.spin_single_escape.argtypes = [P(spin_params), i32, P(d), vp, vp, i64, i64, vp, vp, vp, vp, vp, vp]
    L.spin_batch_last_error.argtypes = [vp]
    L.spin_batch_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("spin_strerror", "spin_last_error", "spin_batch_last_error"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def check(rc: int, handle=None) -> int:
    if rc < 0:
        L = load()
        detail = L.spin_last_error(handle).decode() if handle else ""
        raise SpinError(rc, f"{L.spin_strerror(rc).decode()} {detail}".strip())
    return rc
