"""Python face of the C-ABI: functions with the C names (argument marshalling
only) and a ``Lattice`` convenience class.  PyTorch provides device memory
and the CUDA stream; all arithmetic runs in ``libspinpulse.so``.

A state is a torch tensor of shape (3, nz, ny, nx) (components s_x, s_y,
s_z, each an x-fastest array), float32 or float64, on a CUDA device.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

import torch

from . import _binding as B
from ._binding import check


@dataclass
class Params:
    """Problem statement of one lattice (gamma = mu0 = k_B = 1)."""
    nx: int
    ny: int
    nz: int
    J: float = 1.0
    D: float = 0.0
    H: tuple = (0.0, 0.0, 0.0)
    lam: float = 0.1
    T: float = 1.0
    dt: float = 0.1
    R: int = 10
    integrator: int = B.RK4
    precession: int = 1
    renorm: int = 1
    noise: int = 1
    seed: int = 1
    replica: int = 0
    precision: int = 32
    path: int = 0
    bc: int = 0            # 0: periodic, 1: free boundaries

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def dtype(self):
        return torch.float64 if self.precision == 64 else torch.float32

    def c(self) -> B.spin_params:
        return B.spin_params(self.nx, self.ny, self.nz, self.precision, self.integrator,
                             self.precession, self.R, self.renorm, self.noise, self.replica,
                             self.path, self.bc, self.J, self.D, (ctypes.c_double * 3)(*self.H),
                             self.lam, self.T, self.dt, self.seed & 0xFFFFFFFFFFFFFFFF)


def _stream_ptr(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def spin_workspace_size(p: Params) -> int:
    n = ctypes.c_size_t()
    check(B.load().spin_workspace_size(ctypes.byref(p.c()), ctypes.byref(n)))
    return int(n.value)


def spin_lattice_create(p: Params, state: torch.Tensor, h_site: torch.Tensor | None,
                        workspace: torch.Tensor, stream=None):
    """Returns (handle, status); status is SPIN_OK or SPIN_WARN_APPLICABILITY."""
    L = B.load()
    h = ctypes.c_void_p()
    rc = L.spin_lattice_create(ctypes.byref(p.c()), state[0].data_ptr(), state[1].data_ptr(),
                               state[2].data_ptr(), h_site.data_ptr() if h_site is not None else None,
                               workspace.data_ptr(), workspace.numel() * workspace.element_size(),
                               _stream_ptr(stream), ctypes.byref(h))
    check(rc)
    return h, rc


def spin_step_pulse(h, nsteps: int) -> None:
    check(B.load().spin_step_pulse(h, int(nsteps)), h)


def spin_observables(h):
    """Returns (M[3] as a list, E, status)."""
    M = (ctypes.c_double * 3)()
    E = ctypes.c_double()
    rc = B.load().spin_observables(h, M, ctypes.byref(E))
    if rc != B.SPIN_ENONFINITE:
        check(rc, h)
    return [M[0], M[1], M[2]], E.value, rc


def spin_samples(h, max_records: int = B.SPIN_SAMPLE_RING):
    buf = (ctypes.c_double * (5 * max_records))()
    cnt = ctypes.c_int64()
    check(B.load().spin_samples(h, buf, max_records, ctypes.byref(cnt)), h)
    n = cnt.value
    return [tuple(buf[5 * q:5 * q + 5]) for q in range(n)]


def spin_get_step(h) -> int:
    n = ctypes.c_int64()
    check(B.load().spin_get_step(h, ctypes.byref(n)), h)
    return n.value


def spin_set_step(h, n: int) -> None:
    check(B.load().spin_set_step(h, int(n)), h)


def spin_lattice_destroy(h) -> None:
    check(B.load().spin_lattice_destroy(h))


def spin_noise_draw(seed: int, k: int, replica: int, n_sites: int, precision: int = 64,
                    device="cuda", stream=None):
    """Philox words (int64 tensor holding the uint64 bit patterns, shape (n, 4))
    and Box-Muller normals (shape (n, 3)) of pulse k for sites 0..n-1."""
    words = torch.empty((n_sites, 4), dtype=torch.int64, device=device)
    gauss = torch.empty((n_sites, 3), dtype=torch.float64 if precision == 64 else torch.float32,
                        device=device)
    check(B.load().spin_noise_draw(seed & 0xFFFFFFFFFFFFFFFF, k, replica, n_sites, precision,
                                   words.data_ptr(), gauss.data_ptr(), _stream_ptr(stream)))
    return words, gauss


def spin_observables_noalloc(state: torch.Tensor, J: float, D: float, H, out5: torch.Tensor,
                             h_site: torch.Tensor | None = None, bc: int = 0, stream=None) -> None:
    """M and E of a (3, nz, ny, nx) state into the device tensor out5 (5 doubles:
    M_x, M_y, M_z, E, non-finite count) without any allocation; asynchronous.
    For callers that cannot allocate device memory at the call site.  bc: 0
    periodic, 1 free boundaries.  The arguments are checked here before any
    pointer reaches the library (a wrong dtype, shape or device would make the
    kernel read or write outside the tensors)."""
    if not (isinstance(state, torch.Tensor) and state.is_cuda and state.dim() == 4 and state.shape[0] == 3
            and state.is_contiguous() and state.dtype in (torch.float32, torch.float64)):
        raise ValueError("state must be a contiguous CUDA float32/float64 tensor of shape (3, nz, ny, nx)")
    if not (isinstance(out5, torch.Tensor) and out5.is_cuda and out5.dtype == torch.float64
            and out5.is_contiguous() and out5.numel() >= 5 and out5.device == state.device):
        raise ValueError("out5 must be a contiguous CUDA float64 tensor of at least 5 elements on the state's device")
    if h_site is not None and not (isinstance(h_site, torch.Tensor) and h_site.dtype == state.dtype
                                   and h_site.device == state.device and h_site.is_contiguous()
                                   and h_site.numel() == state.numel()):
        raise ValueError("h_site must be a contiguous tensor of the state's dtype, device and size (3N)")
    if int(bc) not in (0, 1):
        raise ValueError("bc must be 0 (periodic) or 1 (free)")
    _, nz, ny, nx = state.shape
    prec = 64 if state.dtype == torch.float64 else 32
    Hc = (ctypes.c_double * 3)(*[float(v) for v in H])
    check(B.load().spin_observables_noalloc(prec, state[0].data_ptr(), state[1].data_ptr(), state[2].data_ptr(),
                                            h_site.data_ptr() if h_site is not None else None, nx, ny, nz,
                                            float(J), float(D), Hc, int(bc), out5.data_ptr(), _stream_ptr(stream)))


def spin_record_store_size(p: Params, K: int, nsteps: int) -> int:
    n = ctypes.c_size_t()
    check(B.load().spin_record_store_size(ctypes.byref(p.c()), int(K), int(nsteps), ctypes.byref(n)))
    return int(n.value)


def spin_record_begin(h, K: int, nsteps: int, store: torch.Tensor) -> None:
    check(B.load().spin_record_begin(h, int(K), int(nsteps), store.data_ptr(),
                                     store.numel() * store.element_size()), h)


def spin_record_end(h) -> None:
    check(B.load().spin_record_end(h), h)


def spin_backward_workspace_size(p: Params, K: int) -> int:
    n = ctypes.c_size_t()
    check(B.load().spin_backward_workspace_size(ctypes.byref(p.c()), int(K), ctypes.byref(n)))
    return int(n.value)


def spin_backward(h, dLdM, dLdE: float, workspace: torch.Tensor, g_h_site: torch.Tensor | None = None,
                  g_s0: torch.Tensor | None = None):
    """Returns (dL/dJ, dL/dD, dL/dH[3]); fills g_h_site (FP64, 3N) and g_s0 if given."""
    dM = (ctypes.c_double * 3)(*[float(v) for v in dLdM])
    gJ, gD = ctypes.c_double(), ctypes.c_double()
    gH = (ctypes.c_double * 3)()
    check(B.load().spin_backward(h, dM, float(dLdE), workspace.data_ptr(),
                                 workspace.numel() * workspace.element_size(), ctypes.byref(gJ), ctypes.byref(gD), gH,
                                 g_h_site.data_ptr() if g_h_site is not None else None,
                                 g_s0.data_ptr() if g_s0 is not None else None), h)
    return gJ.value, gD.value, [gH[0], gH[1], gH[2]]


class Lattice:
    """Owns the device state, the optional per-site field and the workspace of
    one handle.  ``state`` is (3, nz, ny, nx) on the GPU."""

    def __init__(self, p: Params, state, h_site=None, device="cuda", stream=None):
        self.p = p
        # the library updates the state in place: keep a private copy
        self.state = torch.as_tensor(state).to(device=device, dtype=p.dtype).reshape(3, p.nz, p.ny, p.nx).clone()
        self.h_site = None
        if h_site is not None:
            self.h_site = torch.as_tensor(h_site).to(device=device, dtype=p.dtype).reshape(3, p.nz, p.ny, p.nx).clone()
        nbytes = spin_workspace_size(p)
        self.workspace = torch.empty(nbytes // 8 + 32, dtype=torch.float64, device=device)
        self.stream = stream
        self.handle, self.status = spin_lattice_create(p, self.state, self.h_site, self.workspace, stream)

    def step(self, n: int) -> "Lattice":
        spin_step_pulse(self.handle, n)
        return self

    def observables(self):
        M, E, rc = spin_observables(self.handle)
        return M, E

    def samples(self):
        return spin_samples(self.handle)

    @property
    def n(self) -> int:
        return spin_get_step(self.handle)

    def set_step(self, n: int) -> None:
        spin_set_step(self.handle, n)

    def record(self, K: int, nsteps: int) -> None:
        """Checkpoint the trajectory every K steps for the next nsteps steps."""
        nbytes = spin_record_store_size(self.p, K, nsteps)
        self.store = torch.empty(nbytes // 8 + 1, dtype=torch.float64, device=self.state.device)
        self.K = K
        spin_record_begin(self.handle, K, nsteps, self.store)

    def backward(self, dLdM, dLdE: float, field_grad: bool = True, state_grad: bool = False):
        """Gradients of dLdE E + dLdM.M of the current state over the recorded
        run: dict J, D, H and (optionally) h (FP64 (3,nz,ny,nx)) and s0."""
        p = self.p
        ws = torch.empty(spin_backward_workspace_size(p, self.K) // 8 + 32, dtype=torch.float64,
                         device=self.state.device)
        gh = torch.empty((3, p.nz, p.ny, p.nx), dtype=torch.float64, device=self.state.device) if field_grad else None
        gs = torch.empty((3, p.nz, p.ny, p.nx), dtype=p.dtype, device=self.state.device) if state_grad else None
        gJ, gD, gH = spin_backward(self.handle, dLdM, dLdE, ws, gh, gs)
        return {"J": gJ, "D": gD, "H": gH, "h": gh, "s0": gs}

    def close(self) -> None:
        if self.handle is not None:
            spin_lattice_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SpinRunFn(torch.autograd.Function):
    """(E, M) of the final state after nsteps pulse-noise steps from s0, with
    pathwise gradients (noise fixed) w.r.t. J, D, the uniform field H (3) and
    the per-site field h through the library's checkpointed adjoint
    (checkpoint every K steps).  dL/dH = sum_i dL/dh_i, accumulated in FP64."""

    @staticmethod
    def forward(ctx, J, D, H, h_site, s0, p: Params, nsteps: int, K: int):
        import dataclasses
        Hv = tuple(float(v) for v in torch.as_tensor(H, dtype=torch.float64).reshape(3).tolist())
        q = dataclasses.replace(p, J=float(J), D=float(D), H=Hv)
        lat = Lattice(q, s0.detach(), h_site=h_site.detach(), device=s0.device)
        lat.record(K, nsteps)
        lat.step(nsteps)
        M, E = lat.observables()
        ctx.lat = lat
        ctx.h_shape = h_site.shape
        ctx.h_dtype = h_site.dtype
        ctx.H_meta = (torch.as_tensor(H).dtype, torch.as_tensor(H).device, torch.as_tensor(H).shape)
        return (torch.tensor(E, dtype=torch.float64, device=s0.device),
                torch.tensor(M, dtype=torch.float64, device=s0.device))

    @staticmethod
    def backward(ctx, gE, gM):
        g = ctx.lat.backward(gM.detach().cpu().tolist(), float(gE.detach().cpu()), field_grad=True)
        ctx.lat.close()
        dev = gE.device
        h_dtype, h_dev, h_shape = ctx.H_meta
        gH = torch.tensor(g["H"], dtype=torch.float64).to(device=h_dev, dtype=h_dtype).reshape(h_shape)
        return (torch.tensor(g["J"], dtype=torch.float64, device=dev),
                torch.tensor(g["D"], dtype=torch.float64, device=dev),
                gH,
                g["h"].reshape(ctx.h_shape).to(ctx.h_dtype), None, None, None, None)


def _host_doubles(vals):
    vals = [float(v) for v in vals]
    return (ctypes.c_double * len(vals))(*vals)


def _prepare(obj):
    """spin_single_prepare: per-replica noise scales and dampings into the
    object's scratch (once; the run calls are plain asynchronous launches)."""
    lam = None if obj.lam is None else _host_doubles(obj.lam)
    check(B.load().spin_single_prepare(ctypes.byref(obj.p.c()), obj.nrep, _host_doubles(obj.T), lam,
                                       obj.scratch.data_ptr(), _stream_ptr(obj.stream)))


class SingleSpins:
    """nrep independent spins with E = -D s_z^2 - H.s at temperatures T[r]
    and dampings lam[r] (default p.lam), one GPU thread each
    (spin_single_run).  ``state`` is (3, nrep): s_x, s_y, s_z rows."""

    def __init__(self, p: Params, T, state, lam=None, device="cuda", stream=None):
        self.p = p
        self.T = [float(v) for v in T]
        self.nrep = len(self.T)
        self.lam = None if lam is None else [float(v) for v in lam]
        if self.lam is not None and len(self.lam) != self.nrep:
            raise ValueError("lam must have one value per replica")
        self.state = torch.as_tensor(state).to(device=device, dtype=p.dtype).reshape(3, self.nrep).clone()
        self.scratch = torch.empty(2 * self.nrep, dtype=p.dtype, device=device)
        self.first_passage = torch.full((self.nrep,), -1, dtype=torch.int64, device=device)
        self.sz_sum = torch.zeros(self.nrep, dtype=torch.float64, device=device)
        self.sz_count = torch.zeros(self.nrep, dtype=torch.int64, device=device)
        self.n = 0
        self.stream = stream
        _prepare(self)

    def run(self, nsteps: int, stop_on_crossing: bool = False, average: bool = False) -> "SingleSpins":
        check(B.load().spin_single_run(ctypes.byref(self.p.c()), self.nrep,
                                       self.state.data_ptr(), self.scratch.data_ptr(), self.n, int(nsteps),
                                       int(stop_on_crossing), self.first_passage.data_ptr(),
                                       self.sz_sum.data_ptr() if average else None,
                                       self.sz_count.data_ptr() if average else None, _stream_ptr(self.stream)))
        self.n += int(nsteps)
        return self


class EscapeReplicas:
    """Renewal first-passage runs (spin_single_escape): nrep replicas start
    at ``s_init``; every crossing of s_z = 0 ends a trial, whose length in
    steps is summed, and the replica restarts at ``s_init`` at the next
    noise-interval start."""

    def __init__(self, p: Params, T, s_init, lam=None, device="cuda", stream=None):
        self.p = p
        self.T = [float(v) for v in T]
        self.nrep = len(self.T)
        self.lam = None if lam is None else [float(v) for v in lam]
        if self.lam is not None and len(self.lam) != self.nrep:
            raise ValueError("lam must have one value per replica")
        self.s_init = [float(v) for v in s_init]
        init = torch.tensor(self.s_init, dtype=torch.float64).reshape(3, 1).expand(3, self.nrep)
        self.state = init.to(device=device, dtype=p.dtype).contiguous()
        self.scratch = torch.empty(2 * self.nrep, dtype=p.dtype, device=device)
        z = lambda dt: torch.zeros(self.nrep, dtype=dt, device=device)
        self.trial, self.local_step = z(torch.int64), z(torch.int64)
        self.fpt_sum, self.fpt_count, self.fpt_sq = z(torch.int64), z(torch.int64), z(torch.float64)
        self.n = 0
        self.stream = stream
        _prepare(self)

    def run(self, nsteps: int) -> "EscapeReplicas":
        check(B.load().spin_single_escape(ctypes.byref(self.p.c()), self.nrep,
                                          _host_doubles(self.s_init), self.state.data_ptr(),
                                          self.scratch.data_ptr(), self.n, int(nsteps), self.trial.data_ptr(),
                                          self.local_step.data_ptr(), self.fpt_sum.data_ptr(),
                                          self.fpt_sq.data_ptr(), self.fpt_count.data_ptr(),
                                          _stream_ptr(self.stream)))
        self.n += int(nsteps)
        return self

    def mfpt(self, groups=None):
        """Per group of replica indices (default: all replicas) a tuple
        (mean first-passage time, its standard error, finished trials, rate),
        times in time units.  ``rate`` = finished trials / total time inside
        trials, the unfinished trials included and the waits for an interval
        start excluded: for exponentially distributed
        passage times it is the unbiased estimate of 1/MFPT even when the
        run is not much longer than one passage time."""
        torch.cuda.synchronize()
        s = self.fpt_sum.double().cpu()
        q = self.fpt_sq.cpu()
        c = self.fpt_count.double().cpu()
        open_steps = self.local_step.clamp(min=0).double().cpu()
        dt = abs(self.p.dt)
        out = []
        for g in (groups if groups is not None else [list(range(self.nrep))]):
            idx = torch.as_tensor(g, dtype=torch.long)
            n = float(c[idx].sum())
            total = float(s[idx].sum() + open_steps[idx].sum()) * dt
            if n == 0:
                out.append((float("inf"), float("inf"), 0, 0.0))
                continue
            m = float(s[idx].sum()) / n
            var = max(float(q[idx].sum()) / n - m * m, 0.0)
            out.append((m * dt, (var / n) ** 0.5 * dt, int(n), n / total))
        return out if groups is not None else out[0]


def _mc_check(p, state, h_site):
    if not (state.is_cuda and state.dtype == p.dtype and state.is_contiguous()):
        raise ValueError("state must be a contiguous CUDA tensor of the lattice precision")
    if h_site is not None and not (h_site.is_cuda and h_site.dtype == p.dtype and h_site.is_contiguous()):
        raise ValueError("h_site must be a contiguous CUDA tensor of the lattice precision")


def spin_metropolis_sweeps(p: Params, state, nsweeps: int, mc_seed: int, R_trial=None, sweep0: int = 0,
                           h_site=None, accepted=None, stream=None) -> None:
    """Checkerboard Metropolis sweeps on a device state tensor (3, nz, ny, nx)
    of p's precision, in place; ``accepted`` an optional device int64 tensor
    of one element that counts accepted trials."""
    _mc_check(p, state, h_site)
    check(B.load().spin_metropolis_sweeps(ctypes.byref(p.c()), state.data_ptr(),
                                          None if h_site is None else h_site.data_ptr(),
                                          mc_seed & 0xFFFFFFFFFFFFFFFF, -1.0 if R_trial is None else float(R_trial),
                                          int(sweep0), int(nsweeps),
                                          None if accepted is None else accepted.data_ptr(), _stream_ptr(stream)))


def spin_metropolis_color(p: Params, state, sweep: int, color: int, mc_seed: int, R_trial=None, h_site=None,
                          accepted=None, stream=None) -> None:
    """One colour (0: x+y+z even, 1: odd) of checkerboard sweep ``sweep``."""
    _mc_check(p, state, h_site)
    check(B.load().spin_metropolis_color(ctypes.byref(p.c()), state.data_ptr(),
                                         None if h_site is None else h_site.data_ptr(),
                                         mc_seed & 0xFFFFFFFFFFFFFFFF, -1.0 if R_trial is None else float(R_trial),
                                         int(sweep), int(color),
                                         None if accepted is None else accepted.data_ptr(), _stream_ptr(stream)))
