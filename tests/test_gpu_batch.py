"""Batched replicas (spin_batch_*) against the oracle and against single-lattice
handles: replica r of a batch is the lattice with replica index r, so its
state must equal the single-handle run bit for bit (the per-site arithmetic
does not depend on how the work is tiled) and the oracle to the FP32 step
tolerance."""
import numpy as np
import pytest
import torch

import spin_inputs
from gpu_helpers import as_input, gpu_state, orc_params

pytestmark = pytest.mark.gpu

KW = dict(J=1.0, D=0.02, H=(0.0, 0.0, 0.05), lam=0.05, dt=0.1, R=4, seed=4, precision=32)


def _batch(gpu, L, T, seed=7, chunk=None, **over):
    kw = {**KW, **over}
    p = gpu.Params(1, 1, 1, **kw)
    states = [spin_inputs.random_spins(l, l, l, seed=seed + r) for r, l in enumerate(L)]
    return p, states, gpu.Batch(p, L, T, states, chunk_planes=chunk, use_cache=False)


def test_batch_matches_oracle(gpu, orc):
    L = [4, 7, 16, 24, 5, 16]
    T = [0.3, 1.9, 0.8, 1.2, 0.5, 1.6]
    p, states, b = _batch(gpu, L, T)
    b.step(12)
    rec = b.samples()
    assert rec.shape == (3, len(L), 5)
    for r, l in enumerate(L):
        q = gpu.Params(l, l, l, **{**KW, "T": T[r], "replica": r})
        ref, smp = orc.run(orc_params(orc, q), as_input(q, states[r]), 12)
        got = b.replica_state(r).double().cpu().numpy()
        assert np.max(np.abs(got - ref)) < 1e-5, r
        assert np.max(np.abs(rec[:, r, 1:] - smp[:, 1:])) < 5e-6, r
        assert np.array_equal(rec[:, r, 0], smp[:, 0])


@pytest.mark.parametrize("precession,integrator", [(1, 0), (0, 0), (1, 2)])
def test_batch_bitwise_equals_single_lattices(gpu, precession, integrator):
    L = [16, 24, 32, 9]
    T = [0.4, 1.0, 1.7, 0.9]
    p, states, b = _batch(gpu, L, T, precession=precession, integrator=integrator)
    b.step(23)                     # eager, graph replays and a partial interval
    for r, l in enumerate(L):
        q = gpu.Params(l, l, l, **{**KW, "T": T[r], "replica": r, "precession": precession, "integrator": integrator})
        lat = gpu.Lattice(q, torch.from_numpy(states[r]))
        lat.step(23)
        assert torch.equal(lat.state, b.replica_state(r)), r
        M, E = lat.observables()
        ob = b.observables()[r]
        assert np.allclose(ob[:3], M, rtol=0, atol=1e-12) and abs(ob[3] - E) < 1e-12


@pytest.mark.parametrize("integrator", [0, 2])
def test_batch_tiling_does_not_change_results(gpu, integrator):
    """Every tile height the library offers x z-chunks from 3 planes to
    whole-lattice, the same tiling for all classes and a different one per
    class (several launches per step), and the autotuned choice: the states
    after 20 steps (graph replays and a partial interval) are bit-identical."""
    L, T = [32, 24, 16, 24, 9], [1.0, 0.5, 1.5, 0.7, 1.1]
    rows = gpu.spin_batch_tile_rows(integrator)
    assert len(rows) == 3 and rows == sorted(rows, reverse=True)
    _, _, ref = _batch(gpu, L, T, chunk=gpu.batch.DEFAULT_TILING, integrator=integrator)
    ref.step(20)
    for tr in rows:
        for ch in (3, 8, 64):
            _, _, b = _batch(gpu, L, T, chunk=gpu.batch.DEFAULT_TILING, integrator=integrator)
            b.set_tiling({l: (tr, ch) for l in set(L)})
            assert b.tiling() == {l: (tr, ch) for l in (32, 24, 16, 9)}
            b.step(20)
            assert torch.equal(ref.state, b.state), (tr, ch)
            b.close()
    mixed = {32: (rows[0], 5), 24: (rows[1], 16), 16: (rows[2], 8), 9: (rows[1], 64)}
    _, _, m = _batch(gpu, L, T, chunk=gpu.batch.DEFAULT_TILING, integrator=integrator)
    m.set_tiling(mixed)
    m.step(20)
    assert torch.equal(ref.state, m.state)
    _, _, c = _batch(gpu, L, T, chunk=None, integrator=integrator)   # autotuned
    t = c.tiling()
    assert set(t) == {32, 24, 16, 9}
    assert all(r in rows and k in (8, 16, 32, 64) for r, k in t.values())
    c.step(20)
    assert torch.equal(ref.state, c.state)


def test_batch_tiling_rejects_bad_requests(gpu):
    _, _, b = _batch(gpu, [16, 8], [1.0, 1.0], chunk=gpu.batch.DEFAULT_TILING)
    rows = gpu.spin_batch_tile_rows(0)
    with pytest.raises(gpu.SpinError):
        b.set_tiling({12: (rows[0], 8)})        # no replica of side 12
    with pytest.raises(gpu.SpinError):
        b.set_tiling({16: (rows[0] + 1, 8)})    # height not offered
    with pytest.raises(gpu.SpinError):
        b.set_tiling({16: (rows[0], 0)})        # empty chunk
    assert b.tiling() == {16: (rows[0], 32), 8: (rows[0], 32)}


def test_batch_tiling_cache_is_per_size_class(gpu, tmp_path, monkeypatch):
    """The JSON cache holds one entry per (precision, integrator, L); a later
    batch with another mix of sizes reuses the classes it shares."""
    monkeypatch.setenv("XDG_CACHE_HOME", str(tmp_path))
    p = gpu.Params(1, 1, 1, **KW)
    st = lambda L: [spin_inputs.random_spins(l, l, l, seed=3 + r) for r, l in enumerate(L)]
    a = gpu.Batch(p, [16, 24], [1.0, 1.0], st([16, 24]))
    import json
    cache = json.load(open(tmp_path / "spinpulse" / "batch_tiling.json"))
    assert set(cache) == {"p32-i0-L16", "p32-i0-L24"}
    assert {int(k.split("L")[-1]): tuple(v) for k, v in cache.items()} == a.tiling()
    forced = {"p32-i0-L16": [gpu.spin_batch_tile_rows(0)[2], 3]}
    json.dump({**cache, **forced}, open(tmp_path / "spinpulse" / "batch_tiling.json", "w"))
    b = gpu.Batch(p, [16, 32], [1.0, 1.0], st([16, 32]))
    assert b.tiling()[16] == tuple(forced["p32-i0-L16"])
    cache = json.load(open(tmp_path / "spinpulse" / "batch_tiling.json"))
    assert set(cache) == {"p32-i0-L16", "p32-i0-L24", "p32-i0-L32"}


def test_batch_full_size_512_replicas(gpu):
    """The 512-replica workload (L uniform over {16,24,32,48,64}, T uniform in
    [0.2, 2], J=1, D=0.02, H=0, lambda=0.02, RK4 dt=0.2, pulses every 10):
    one noise interval through the autotuned batch, replicas 0, 17, 255 and
    511 bitwise equal to single handles, all spins unit length."""
    w = spin_inputs.WORKLOADS["batch512"]
    L, T = spin_inputs.replica_draws(w["nrep"], w["seed"])
    kw = dict(J=w["J"], D=w["D"], H=w["H"], lam=w["lam"], dt=w["dt"], R=w["R"], seed=w["seed"], precision=32)
    p = gpu.Params(1, 1, 1, **kw)
    states = [spin_inputs.random_spins(int(l), int(l), int(l), seed=1000 + r) for r, l in enumerate(L)]
    b = gpu.Batch(p, L, T, states, use_cache=False)
    b.step(10)
    st = b.state
    assert torch.max(torch.abs((st.double() ** 2).sum(0) - 1.0)).item() < 1e-6
    rec = b.samples()
    assert rec.shape == (1, 512, 5) and np.all(np.isfinite(rec))
    for r in (0, 17, 255, 511):
        l = int(L[r])
        q = gpu.Params(l, l, l, **{**kw, "T": float(T[r]), "replica": r})
        lat = gpu.Lattice(q, torch.from_numpy(states[r]))
        lat.step(10)
        assert torch.equal(lat.state, b.replica_state(r)), r
