"""Batched replicas through the C-ABI (spin_batch_*): argument marshalling, a
JSON cache of the library's per-size-class tiling choice (tile height and
z-chunk, keyed by side L, precision and integrator), and per-replica views of
the concatenated state."""
from __future__ import annotations

import ctypes
import json
import os

import numpy as np
import torch

from . import _binding as B
from ._binding import check
from .lattice import Params, _stream_ptr

DEFAULT_TILING = -1   # chunk_planes value: every class on the default tiling, no timing


def _cache_path() -> str:
    base = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(base, "spinpulse", "batch_tiling.json")


def _class_key(p: Params, L: int) -> str:
    return f"p{p.precision}-i{p.integrator}-L{int(L)}"


def _load_cache() -> dict:
    try:
        with open(_cache_path()) as f:
            c = json.load(f)
        return c if isinstance(c, dict) else {}
    except (OSError, ValueError):
        return {}


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


def spin_batch_tile_rows(integrator: int) -> list:
    """CTA tile heights the batched step offers for an integrator, tallest first."""
    rows = (ctypes.c_int32 * 8)()
    n = ctypes.c_int32()
    check(B.load().spin_batch_tile_rows(int(integrator), 8, rows, ctypes.byref(n)))
    return list(rows[:n.value])


class Batch:
    """nrep cubic periodic replicas of sides L[r] and temperatures T[r].

    ``states``: list of (3, L, L, L) arrays (or one (3, total) array in the
    concatenated layout).  Tiling (schedule only; the states are bit-identical
    under every choice): ``tiling`` = {L: (tile_rows, chunk)} pins those size
    classes; ``chunk_planes`` = int gives every class that z-chunk on the
    default tile height (``DEFAULT_TILING`` = the library default, untimed);
    otherwise classes found in the JSON cache take the cached choice and the
    library autotunes the rest at create (then cached, when ``use_cache``)."""

    def __init__(self, p: Params, L, T, states, chunk_planes=None, tiling=None, device="cuda", stream=None,
                 use_cache=True):
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
        pinned = {int(k): (int(v[0]), int(v[1])) for k, v in (tiling or {}).items()}
        cache = _load_cache() if (use_cache and chunk_planes is None) else {}
        if chunk_planes is None:
            for l in sorted(set(self.L)):
                hit = cache.get(_class_key(p, l))
                if l not in pinned and isinstance(hit, list) and len(hit) == 2:
                    pinned[l] = (int(hit[0]), int(hit[1]))
        hint = int(chunk_planes) if chunk_planes is not None else DEFAULT_TILING
        Lc = (ctypes.c_int32 * self.nrep)(*self.L)
        Tc = (ctypes.c_double * self.nrep)(*self.T)
        h = ctypes.c_void_p()
        check(B.load().spin_batch_create(ctypes.byref(p.c()), self.nrep, Lc, Tc, self.state[0].data_ptr(),
                                         self.state[1].data_ptr(), self.state[2].data_ptr(), hint,
                                         self.workspace.data_ptr(), self.workspace.numel() * 8,
                                         _stream_ptr(stream), ctypes.byref(h)))
        self.handle = h
        if pinned:
            self.set_tiling(pinned)
        if chunk_planes is None:
            tuned = set(self.L) - set(pinned)
            if tuned:
                self._check(B.load().spin_batch_autotune(self.handle))
                if use_cache:
                    now = self.tiling()
                    cache = _load_cache()
                    for l in tuned:
                        cache[_class_key(p, l)] = list(now[l])
                    try:
                        os.makedirs(os.path.dirname(_cache_path()), exist_ok=True)
                        with open(_cache_path(), "w") as f:
                            json.dump(cache, f, indent=0, sort_keys=True)
                    except OSError:
                        pass
        self._refresh()

    def _refresh(self):
        cp, ni = ctypes.c_int32(), ctypes.c_int32()
        check(B.load().spin_batch_tuning(self.handle, ctypes.byref(cp), ctypes.byref(ni)))
        self.chunk_planes, self.nitems = cp.value, ni.value

    def tiling(self) -> dict:
        """{L: (tile_rows, chunk)} per size class."""
        m = len(set(self.L))
        Ls, rows, ch = (ctypes.c_int32 * m)(), (ctypes.c_int32 * m)(), (ctypes.c_int32 * m)()
        n = ctypes.c_int32()
        self._check(B.load().spin_batch_tiling(self.handle, m, Ls, rows, ch, ctypes.byref(n)))
        return {int(Ls[i]): (int(rows[i]), int(ch[i])) for i in range(n.value)}

    def set_tiling(self, tiling: dict) -> "Batch":
        """Pin {L: (tile_rows, chunk)}; the other classes keep theirs."""
        n = len(tiling)
        ks = list(tiling)
        Ls = (ctypes.c_int32 * n)(*[int(k) for k in ks])
        rows = (ctypes.c_int32 * n)(*[int(tiling[k][0]) for k in ks])
        ch = (ctypes.c_int32 * n)(*[int(tiling[k][1]) for k in ks])
        self._check(B.load().spin_batch_set_tiling(self.handle, n, Ls, rows, ch))
        self._refresh()
        return self

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
