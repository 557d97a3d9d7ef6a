"""FP64 CPU oracle for the pulse-noise many-spin step (arXiv:1610.04914).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the GPU library never
does, and this package never imports the GPU library.

The arithmetic lives in ``spin_oracle.c`` (plain C, double precision, one site
at a time, compiled with ``-ffp-contract=off``).  This module only builds it
with gcc, loads it with ctypes and marshals numpy arrays.

Spin states are numpy arrays of shape (3, nz, ny, nx) (component, z, y, x),
i.e. structure-of-arrays with x fastest.

Parity status (what pins each function) is stated in the C source and in the
``-m "not gpu"`` tests under ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spin_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")

RK4, RK5_BUTCHER, RK2_MIDPOINT, HEUN = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile spin_oracle.c into liboracle.so next to it (gcc, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def build_omp(force: bool = False):
    """The same source compiled with -fopenmp into liboracle_omp.so: its
    whole-lattice loops run on all host cores with unchanged per-site
    arithmetic.  Returns the path, or None if the compiler has no OpenMP."""
    if force or not os.path.exists(_LIB_OMP) or os.path.getmtime(_LIB_OMP) < os.path.getmtime(_SRC):
        tmp = _LIB_OMP + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            return None
        os.replace(tmp, _LIB_OMP)
    return _LIB_OMP


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("integrator", ctypes.c_int32), ("precession", ctypes.c_int32),
        ("R", ctypes.c_int32), ("renorm", ctypes.c_int32), ("replica", ctypes.c_int32),
        ("bc", ctypes.c_int32), ("unused", ctypes.c_int32),
        ("J", ctypes.c_double), ("D", ctypes.c_double), ("H", ctypes.c_double * 3),
        ("lambda_", ctypes.c_double), ("T", ctypes.c_double), ("dt", ctypes.c_double),
        ("seed", ctypes.c_uint64),
    ]


@dataclass
class Params:
    """Problem statement of one lattice run (gamma = mu0 = k_B = 1)."""
    nx: int
    ny: int
    nz: int
    J: float = 1.0
    D: float = 0.0
    H: tuple = (0.0, 0.0, 0.0)
    lam: float = 0.1
    T: float = 1.0
    dt: float = 0.1
    R: int = 10                    # steps per noise interval, Delta t = R dt
    integrator: int = RK4
    precession: int = 1            # 0: slow (overdamped) equation
    renorm: int = 1
    seed: int = 1
    replica: int = 0
    bc: int = 0                    # 0: periodic, 1: free

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.nz

    def c(self) -> _Params:
        return _Params(self.nx, self.ny, self.nz, self.integrator, self.precession,
                       self.R, self.renorm, self.replica, self.bc, 0, self.J, self.D,
                       (ctypes.c_double * 3)(*self.H), self.lam, self.T, self.dt,
                       self.seed & 0xFFFFFFFFFFFFFFFF)


_lib = None
_lib_omp = None


def lib(threads: bool = False):
    """The serial build (default) or, with threads=True, the OpenMP build."""
    global _lib, _lib_omp
    if threads:
        if _lib_omp is None:
            path = build_omp()
            if path is None:
                raise RuntimeError("gcc could not build the OpenMP oracle")
            _lib_omp = _declare(ctypes.CDLL(path))
        return _lib_omp
    if _lib is None:
        _lib = _declare(ctypes.CDLL(build()))
    return _lib


def _declare(L):
    if True:
        P = ctypes.POINTER
        d, u64, i64 = ctypes.c_double, ctypes.c_uint64, ctypes.c_int64
        L.orc_philox4x64.argtypes = [P(u64), P(u64), P(u64)]
        L.orc_gauss3.argtypes = [P(u64), P(d)]
        L.orc_noise_gauss.argtypes = [u64, i64, i64, i64, P(d)]
        L.orc_rect_field.argtypes = [P(_Params), i64, P(d)]
        L.orc_heff.argtypes = [P(_Params), P(d), P(d), P(d)]
        L.orc_rhs.argtypes = [P(_Params), P(d), P(d), P(d)]
        L.orc_integrate.argtypes = [P(_Params), P(d), P(d)]
        L.orc_renormalise.argtypes = [P(_Params), P(d)]
        L.orc_pulse_sigma.argtypes = [P(_Params)]
        L.orc_pulse_sigma.restype = d
        L.orc_rotate.argtypes = [P(d), P(d)]
        L.orc_pulse.argtypes = [P(_Params), P(d), i64]
        L.orc_observables.argtypes = [P(_Params), P(d), P(d), P(d)]
        L.orc_is_pulse_step.argtypes = [i64, ctypes.c_int32]
        L.orc_pulse_number.argtypes = [i64, ctypes.c_int32]
        L.orc_pulse_number.restype = i64
        L.orc_run.argtypes = [P(_Params), P(d), P(d), i64, i64, ctypes.c_int, P(d), i64]
        L.orc_run.restype = i64
        L.orc_metropolis.argtypes = [P(_Params), P(d), P(d), u64, d, i64, i64, P(d)]
        L.orc_metropolis.restype = i64
        L.orc_metropolis_color.argtypes = [P(_Params), P(d), P(d), u64, d, i64, ctypes.c_int]
        L.orc_metropolis_color.restype = i64
        L.orc_metropolis_checkerboard.argtypes = [P(_Params), P(d), P(d), u64, d, i64, i64, P(d)]
        L.orc_metropolis_checkerboard.restype = i64
        L.orc_rhs_vjp.argtypes = [P(_Params), P(d), P(d), P(d), P(d), P(d), P(d), P(d), P(d)]
        L.orc_step_vjp.argtypes = [P(_Params), P(d), P(d), ctypes.c_int, i64, P(d), P(d), P(d), P(d), P(d)]
        L.orc_adjoint.argtypes = [P(_Params), P(d), P(d), i64, i64, ctypes.c_int, P(d), d, P(d), P(d), P(d),
                                  P(d), P(d)]
    return L


def omp_threads() -> int:
    """Threads the OpenMP build uses (OMP_NUM_THREADS, else all host cores)."""
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v and v.isdigit() and int(v) > 0 else (os.cpu_count() or 1)


def _dp(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _state(p: Params, s) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(s, dtype=np.float64).reshape(3, p.nz, p.ny, p.nx))
    return a.copy()


def _field(p: Params, h):
    if h is None:
        return None
    return np.ascontiguousarray(np.asarray(h, dtype=np.float64).reshape(3, p.nz, p.ny, p.nx))


# ---------------------------------------------------------------- Philox / noise
def philox4x64(ctr, key) -> np.ndarray:
    c = (ctypes.c_uint64 * 4)(*[int(v) & 0xFFFFFFFFFFFFFFFF for v in ctr])
    k = (ctypes.c_uint64 * 2)(*[int(v) & 0xFFFFFFFFFFFFFFFF for v in key])
    o = (ctypes.c_uint64 * 4)()
    lib().orc_philox4x64(c, k, o)
    return np.array(list(o), dtype=np.uint64)


def gauss3(words) -> np.ndarray:
    w = (ctypes.c_uint64 * 4)(*[int(v) for v in words])
    g = (ctypes.c_double * 3)()
    lib().orc_gauss3(w, g)
    return np.array(list(g))


def noise_gauss(seed: int, site: int, k: int, replica: int = 0) -> np.ndarray:
    g = (ctypes.c_double * 3)()
    lib().orc_noise_gauss(seed & 0xFFFFFFFFFFFFFFFF, site, k, replica, g)
    return np.array(list(g))


STREAM_NOISE = 0x6E6F697365
STREAM_MC = 0x6D6F6E7465


def pulse_sigma(p: Params) -> float:
    return lib().orc_pulse_sigma(ctypes.byref(p.c()))


def rotate(phi_vec, s) -> np.ndarray:
    a = np.array(phi_vec, dtype=np.float64)
    b = np.array(s, dtype=np.float64)
    lib().orc_rotate(_dp(a), _dp(b))
    return b


def is_pulse_step(n: int, R: int) -> bool:
    return bool(lib().orc_is_pulse_step(n, R))


def pulse_number(n: int, R: int) -> int:
    return int(lib().orc_pulse_number(n, R))


# ---------------------------------------------------------------- field / rhs / step
def heff(p: Params, s, h_site=None) -> np.ndarray:
    a = _state(p, s)
    out = np.empty_like(a)
    hs = _field(p, h_site)
    lib().orc_heff(ctypes.byref(p.c()), _dp(a), _dp(hs), _dp(out))
    return out


def rhs(p: Params, s, h_site=None) -> np.ndarray:
    a = _state(p, s)
    out = np.empty_like(a)
    hs = _field(p, h_site)
    lib().orc_rhs(ctypes.byref(p.c()), _dp(a), _dp(hs), _dp(out))
    return out


def integrate(p: Params, s, h_site=None) -> np.ndarray:
    """One noiseless step delta t (no renormalisation, no pulse)."""
    a = _state(p, s)
    hs = _field(p, h_site)
    lib().orc_integrate(ctypes.byref(p.c()), _dp(a), _dp(hs))
    return a


def renormalise(p: Params, s) -> np.ndarray:
    a = _state(p, s)
    lib().orc_renormalise(ctypes.byref(p.c()), _dp(a))
    return a


def pulse(p: Params, s, k: int) -> np.ndarray:
    a = _state(p, s)
    lib().orc_pulse(ctypes.byref(p.c()), _dp(a), k)
    return a


def observables(p: Params, s, h_site=None) -> np.ndarray:
    """(M_x, M_y, M_z, E) per spin."""
    a = _state(p, s)
    hs = _field(p, h_site)
    out = np.zeros(4)
    lib().orc_observables(ctypes.byref(p.c()), _dp(a), _dp(hs), _dp(out))
    return out


NOISE_NONE, NOISE_PULSE, NOISE_RECT = 0, 1, 2


def run(p: Params, s, nsteps: int, n0: int = 0, h_site=None, noise=True, threads: bool = False):
    """Advance nsteps from completed step n0.  Returns (state, samples) with
    samples rows (n, M_x, M_y, M_z, E) taken after steps with n mod R == 0.
    noise: False/0 none, True/1 the pulses (Eq. (phi_n)), 2 rectangular noise
    (Eq. (zeta_n), needs the precession term).  threads: run the OpenMP build
    (same per-site arithmetic on all host cores)."""
    a = _state(p, s)
    hs = _field(p, h_site)
    cap = nsteps // max(p.R, 1) + 2
    smp = np.zeros((cap, 5))
    ns = lib(threads).orc_run(ctypes.byref(p.c()), _dp(a), _dp(hs), n0, nsteps, int(noise), _dp(smp), cap)
    if ns < 0:
        raise ValueError("rectangular noise needs the precession term (precession=1)")
    return a, smp[:ns]


def rect_field(p: Params, k: int) -> np.ndarray:
    """Rectangular-noise field of interval k at every site, shape (3, nz, ny, nx)."""
    z = np.zeros((3, p.nz, p.ny, p.nx))
    lib().orc_rect_field(ctypes.byref(p.c()), k, _dp(z))
    return z


def metropolis(p: Params, s, nsweeps: int, mc_seed: int, R_trial=None, sweep0: int = 0, h_site=None):
    """Sequential Metropolis sweeps.  Returns (state, series[nsweeps,4], accepted)."""
    if R_trial is None:
        R_trial = 1.55 * np.sqrt(p.T / (6.0 * p.J))
    a = _state(p, s)
    hs = _field(p, h_site)
    ser = np.zeros((nsweeps, 4))
    acc = lib().orc_metropolis(ctypes.byref(p.c()), _dp(a), _dp(hs), mc_seed & 0xFFFFFFFFFFFFFFFF,
                               float(R_trial), sweep0, nsweeps, _dp(ser))
    return a, ser, int(acc)


def _trial_length(p: Params, R_trial):
    return 1.55 * np.sqrt(p.T / (6.0 * p.J)) if R_trial is None else R_trial


def metropolis_checkerboard(p: Params, s, nsweeps: int, mc_seed: int, R_trial=None, sweep0: int = 0,
                            h_site=None):
    """Checkerboard Metropolis sweeps (colour 0 = even x+y+z, then colour 1),
    the same trials and random numbers as ``metropolis``.  Returns
    (state, series[nsweeps,4], accepted)."""
    a = _state(p, s)
    hs = _field(p, h_site)
    ser = np.zeros((nsweeps, 4))
    acc = lib().orc_metropolis_checkerboard(ctypes.byref(p.c()), _dp(a), _dp(hs), mc_seed & 0xFFFFFFFFFFFFFFFF,
                                            float(_trial_length(p, R_trial)), sweep0, nsweeps, _dp(ser))
    return a, ser, int(acc)


def metropolis_color(p: Params, s, sweep: int, color: int, mc_seed: int, R_trial=None, h_site=None):
    """One half of checkerboard sweep ``sweep``: the sites of one colour.
    Returns (state, accepted)."""
    a = _state(p, s)
    hs = _field(p, h_site)
    acc = lib().orc_metropolis_color(ctypes.byref(p.c()), _dp(a), _dp(hs), mc_seed & 0xFFFFFFFFFFFFFFFF,
                                     float(_trial_length(p, R_trial)), sweep, color)
    return a, int(acc)


# ---------------------------------------------------------------- adjoint
def rhs_vjp(p: Params, x, v, h_site=None):
    """(J_f(x)^T v, dJ, dD, dH[3], dh[3N]): transpose of the right-hand side's
    Jacobian applied to v, and <v, df/dtheta> for theta = J, D, H, h_i."""
    xa = _state(p, x)
    va = _state(p, v)
    hs = _field(p, h_site)
    out = np.empty_like(xa)
    gJ, gD = ctypes.c_double(0.0), ctypes.c_double(0.0)
    gH = np.zeros(3)
    gh = np.zeros_like(xa)
    lib().orc_rhs_vjp(ctypes.byref(p.c()), _dp(xa), _dp(hs), _dp(va), _dp(out), ctypes.byref(gJ),
                      ctypes.byref(gD), _dp(gH), _dp(gh))
    return out, gJ.value, gD.value, gH, gh


def step_vjp(p: Params, s, lam, pulse: bool = False, k: int = 0, h_site=None):
    """dL/ds_before from dL/ds_after = lam for one step taken from s, with the
    parameter gradients of that step: (lam_before, dJ, dD, dH, dh)."""
    sa = _state(p, s)
    la = _state(p, lam)
    hs = _field(p, h_site)
    gJ, gD = ctypes.c_double(0.0), ctypes.c_double(0.0)
    gH = np.zeros(3)
    gh = np.zeros_like(sa)
    lib().orc_step_vjp(ctypes.byref(p.c()), _dp(sa), _dp(hs), int(pulse), k, _dp(la), ctypes.byref(gJ),
                       ctypes.byref(gD), _dp(gH), _dp(gh))
    return la, gJ.value, gD.value, gH, gh


def adjoint(p: Params, s0, nsteps: int, dLdM, dLdE: float, n0: int = 0, h_site=None, noise: bool = True):
    """Gradients of L = dLdE E(s_n) + dLdM.M(s_n) (E, M per spin) after nsteps
    steps: dict with J, D, H (3,), h (3N field gradient) and s0 (dL/ds_0)."""
    sa = _state(p, s0)
    hs = _field(p, h_site)
    gJ, gD = ctypes.c_double(0.0), ctypes.c_double(0.0)
    gH = np.zeros(3)
    gh = np.zeros_like(sa)
    gs = np.zeros_like(sa)
    dm = np.asarray(dLdM, dtype=np.float64)
    lib().orc_adjoint(ctypes.byref(p.c()), _dp(sa), _dp(hs), n0, nsteps, int(noise), _dp(dm), float(dLdE),
                      ctypes.byref(gJ), ctypes.byref(gD), _dp(gH), _dp(gh), _dp(gs))
    return {"J": gJ.value, "D": gD.value, "H": gH, "h": gh, "s0": gs}
