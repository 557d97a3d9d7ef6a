"""Batched replicas through the C-ABI (spin_batch_*): argument marshalling, a
JSON cache of the library's z-chunk autotuning, and per-replica views of the
concatenated state."""
from __future__ import annotations

import ctypes
import json
import os

import numpy as np
import torch

from . import _binding as B
from ._binding import check
from .lattice import Params, _stream_ptr


def _cache_path() -> str:
    base = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(base, "spinpulse", "batch_tuning.json")


def _tune_key(p: Params, L) -> str:
    return f"p{p.precision}-i{p.integrator}-L" + ",".join(str(v) for v in sorted(int(x) for x in L))


def spin_batch_offsets(L) -> np.ndarray:
    n = len(L)
    Lc = (ctypes.c_int32 * n)(*[int(v) for v in L])
    off = (ctypes.c_int64 * (n + 1))()
    check(B.load().spin_batch_offsets(n, Lc, off))
    return np.array(list(off), dtype=np.int64)


def spin_batch_workspace_size(p: Params, L) -> int:
    n = len(L)
    Lc = (ctypes.c_int32 * n)(*[int(v) for v in L])
    out = ctypes.c_size_t()
    check(B.load().spin_batch_workspace_size(ctypes.byref(p.c()), n, Lc, ctypes.byref(out)))
    return int(out.value)


class Batch:
    """nrep cubic periodic replicas of sides L[r] and temperatures T[r].

    ``states``: list of (3, L, L, L) arrays (or one (3, total) array in the
    concatenated layout).  ``chunk_planes``: None = use the cached tuning or let
    the library autotune at create; an int forces the z-chunk length."""

    def __init__(self, p: Params, L, T, states, chunk_planes=None, device="cuda", stream=None, use_cache=True):
        self.p = p
        self.L = [int(v) for v in L]
        self.T = [float(v) for v in T]
        self.nrep = len(self.L)
        self.offsets = spin_batch_offsets(self.L)
        tot = int(self.offsets[-1])
        if isinstance(states, (list, tuple)):
            flat = np.concatenate([np.asarray(s, dtype=np.float32).reshape(3, -1) for s in states], axis=1)
        else:
            flat = np.asarray(states, dtype=np.float32).reshape(3, tot)
        self.state = torch.from_numpy(np.ascontiguousarray(flat)).to(device)
        nbytes = spin_batch_workspace_size(p, self.L)
        self.workspace = torch.empty(nbytes // 8 + 32, dtype=torch.float64, device=device)
        key = _tune_key(p, self.L)
        cache = {}
        if chunk_planes is None and use_cache and os.path.exists(_cache_path()):
            try:
                cache = json.load(open(_cache_path()))
            except Exception:
                cache = {}
        hint = int(chunk_planes) if chunk_planes is not None else int(cache.get(key, 0))
        Lc = (ctypes.c_int32 * self.nrep)(*self.L)
        Tc = (ctypes.c_double * self.nrep)(*self.T)
        h = ctypes.c_void_p()
        check(B.load().spin_batch_create(ctypes.byref(p.c()), self.nrep, Lc, Tc, self.state[0].data_ptr(),
                                         self.state[1].data_ptr(), self.state[2].data_ptr(), hint,
                                         self.workspace.data_ptr(), self.workspace.numel() * 8,
                                         _stream_ptr(stream), ctypes.byref(h)))
        self.handle = h
        cp, ni = ctypes.c_int32(), ctypes.c_int32()
        check(B.load().spin_batch_tuning(h, ctypes.byref(cp), ctypes.byref(ni)))
        self.chunk_planes, self.nitems = cp.value, ni.value
        if chunk_planes is None and use_cache and key not in cache:
            try:
                os.makedirs(os.path.dirname(_cache_path()), exist_ok=True)
                cache[key] = self.chunk_planes
                json.dump(cache, open(_cache_path(), "w"))
            except OSError:
                pass

    def _check(self, rc):
        if rc < 0:
            L = B.load()
            raise B.SpinError(rc, f"{L.spin_strerror(rc).decode()} {L.spin_batch_last_error(self.handle).decode()}")
        return rc

    def step(self, n: int) -> "Batch":
        self._check(B.load().spin_batch_step_pulse(self.handle, int(n)))
        return self

    def observables(self) -> np.ndarray:
        """(nrep, 5): M_x, M_y, M_z, E per spin, non-finite count."""
        out = (ctypes.c_double * (5 * self.nrep))()
        rc = B.load().spin_batch_observables(self.handle, out)
        if rc != B.SPIN_ENONFINITE:
            self._check(rc)
        return np.array(list(out)).reshape(self.nrep, 5)

    def samples(self, max_records: int = B.SPIN_BATCH_SAMPLE_RING) -> np.ndarray:
        """(records, nrep, 5): n, M_x, M_y, M_z, E."""
        out = (ctypes.c_double * (5 * self.nrep * max_records))()
        cnt = ctypes.c_int64()
        self._check(B.load().spin_batch_samples(self.handle, out, max_records, ctypes.byref(cnt)))
        return np.array(out[:5 * self.nrep * cnt.value]).reshape(cnt.value, self.nrep, 5)

    def replica_state(self, r: int) -> torch.Tensor:
        a, b = int(self.offsets[r]), int(self.offsets[r + 1])
        L = self.L[r]
        return self.state[:, a:b].reshape(3, L, L, L)

    def close(self) -> None:
        if getattr(self, "handle", None) is not None:
            B.load().spin_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
