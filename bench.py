"""Benchmark of the pulse-noise lattice step (arXiv:1610.04914) on GB300.

One bench step = one noise interval of the 128^3 workload: R = 10 fused RK4
steps delta t = 0.2 of the FP32 state, the noise pulse after step 5, the FP64
sample of M and E after step 10 (J=1, D=0.05 along z, H=(0,0,0.02),
lambda=0.01, T=1.0, random spins seed 2), replayed from the library's CUDA
graph through the C-ABI.  L2 is flushed (256 MiB write) before every timed
step; the 10 steps inside one interval see the L2-resident 50 MB working set,
as a real run does.

Prints one JSON line (see the keys below).  ``--impl reference`` times the
FP64 CPU oracle on the same workload instead (bounded samples per step).
Multi-GPU: independent replicas, one per rank (the path has no exchange).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import spin_inputs  # noqa: E402

WORKLOAD = "lattice128"
T_BENCH = 1.0
FALLBACK_HBM_GBS = 6800.0
SMS, FP32_LANES, MAX_SM_MHZ = 152, 128, 2070.0
# algorithmic FP32 flops of one RK4 spin-step (FMA = 2): 4 x (stencil 23 +
# double cross product and combination 24 + stage update 12) - 6 + renorm 9
RK4_FLOPS_PER_SPIN_STEP = 240.0
# algorithmic FP32 flops of one Butcher-RK5 step of a single spin in a
# uniaxial + transverse field (FMA = 2): 12 non-zero stage couplings x 3 FMA,
# 6 right-hand sides x 29, 5 non-zero weights x 3 FMA, renormalisation 9
RK5_FLOPS_PER_SINGLE_STEP = 285.0
BYTES_PER_SPIN_STEP_FP32 = 24.0
# algorithmic bytes of one backward spin-step of the checkpointed adjoint
# (FP32 state, FP64 field gradient): the recomputed forward step (state read +
# write, 24), the step's input state read by the transposes (12), the adjoint
# state read + write (24), the FP64 dL/dh_i read + write (48)
ADJ_BYTES_PER_SPIN_STEP = 108.0


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def time_plain_steps(torch, lat, R, intervals, stream, flush):
    """Per-launch milliseconds of the plain fused step: CUDA events on the
    launching stream around each run of consecutive plain steps of an
    interval (the pulse step also launches the pulse kernel, the last step the
    reduction), L2 flushed before each interval, and a sleep kernel in front so
    the host has queued the launches and the events bracket back-to-back
    kernels rather than host latency.  Each timed run is one call of an even
    number of steps: a call that ends on an odd step count copies the state
    back into the caller's buffer, which is not part of a step."""
    runs = []
    with torch.cuda.stream(stream):
        for _ in range(intervals):
            flush.zero_()
            torch.cuda._sleep(3_000_000)
            q = 0
            while q < R:
                if (q + 1) % R != 0 and (q + 1) % R != R // 2:
                    j = q
                    while j < R and (j + 1) % R != 0 and (j + 1) % R != R // 2:
                        j += 1
                    even = (j - q) & ~1
                    if even:
                        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        a.record(stream)
                        lat.step(even)
                        b.record(stream)
                        runs.append((a, b, even))
                    if j - q - even:
                        lat.step(j - q - even)
                    q = j
                else:
                    lat.step(1)
                    q += 1
    torch.cuda.synchronize()
    return [a.elapsed_time(b) / n for a, b, n in runs for _ in range(n)]


def whole_job_rate(t_local_s: float, units_local: float):
    """Whole-job throughput of independent replicas, one per rank: units summed
    over ranks divided by the slowest rank's timed duration.  Returns
    (value, t_max, units_total); single process when torch.distributed is
    not initialised."""
    import torch
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
        t = torch.tensor([t_local_s], dtype=torch.float64, device=dev)
        u = torch.tensor([units_local], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        t_max, units = float(t.item()), float(u.item())
    else:
        t_max, units = float(t_local_s), float(units_local)
    return units / t_max, t_max, units


def _measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            if "hbm_gbs" in d:
                return float(d["hbm_gbs"]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples every 20 ms; ``stop`` summarises the
    samples that arrived inside the window marked by ``mark_begin`` /
    ``mark_end`` (the timed region)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []          # (arrival time, line)
        self.t = None
        self.window = (None, None)

    def start(self, wait_s: float = 5.0):
        """Start sampling and wait (up to wait_s) until the first sample has
        arrived, so that the timed region that follows is covered."""
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
            return
        t0 = time.perf_counter()
        while not self.lines and time.perf_counter() - t0 < wait_s and self.proc.poll() is None:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def mark_begin(self):
        self.window = (time.perf_counter(), None)

    def mark_end(self):
        self.window = (self.window[0], time.perf_counter())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        b, e = self.window
        inside = [ln for t, ln in self.lines if b is not None and e is not None and b <= t <= e + 0.05]
        where = "timed region"
        if not inside:
            # a timed region shorter than the sampling period: the samples
            # nearest to it on either side
            where = "nearest to the timed region (none inside it)"
            near = sorted(self.lines, key=lambda q: min(abs(q[0] - (b or 0)), abs(q[0] - (e or 0))))
            inside = [ln for _, ln in near[:2]]
        for ln in inside:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm), "sampled": where}


# the sources k_step_patch's code comes from (the file that instantiates it and
# the headers its device code is in)
PATCH_KERNEL_SOURCES = ("step_patch.cu", "patch_tile.cuh", "patch_common.cuh", "spin_device.cuh", "spin_internal.h")


def _kernel_source_hash():
    h = hashlib.sha256()
    for f in PATCH_KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_1610_04914_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def _ncu_traffic():
    """DRAM bytes per launch of the fused step from the committed ncu summary,
    if it was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "step_rk4_fp32_traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
        if d.get("kernel_source_sha256_16") == _kernel_source_hash():
            return d
    except Exception:
        pass
    return None


def _params(sp, w, rank):
    nx, ny, nz = w["n"]
    return sp.Params(nx, ny, nz, J=w["J"], D=w["D"], H=w["H"], lam=w["lam"], T=T_BENCH, dt=w["dt"], R=w["R"],
                     integrator=sp.RK4, precession=w["precession"], seed=w["noise_seed"], replica=rank,
                     precision=32)


def _cpu_model() -> str:
    """Host CPU model (lscpu, else /proc/cpuinfo), for the CPU-baseline record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def cpu_oracle_rate(w, budget_s=15.0, max_steps=10, threads=False):
    """Spin-steps/s of the FP64 oracle on the full 128^3 workload: steps from
    the start of an interval until the time budget or max_steps is reached (the
    pulse is step 5).  threads=False: the serial build, as it stands;
    threads=True: the same source built with OpenMP over z-planes (identical
    per-site arithmetic) on all host cores."""
    import oracle
    oracle.build()
    nx, ny, nz = w["n"]
    op = oracle.Params(nx, ny, nz, J=w["J"], D=w["D"], H=w["H"], lam=w["lam"], T=T_BENCH, dt=w["dt"], R=w["R"],
                       seed=w["noise_seed"])
    s = spin_inputs.random_spins(nx, ny, nz, seed=w["spin_seed"])
    t0 = time.perf_counter()
    steps = 0
    while steps < max_steps:
        s, _ = oracle.run(op, s, 1, n0=steps, threads=threads)
        steps += 1
        el = time.perf_counter() - t0
        if el + el / steps > budget_s:      # the next step would overrun the budget
            break
    dt = time.perf_counter() - t0
    N = nx * ny * nz
    return N * steps / dt, steps, dt


def _omp_available() -> bool:
    try:
        import oracle
        return oracle.build_omp() is not None
    except Exception:
        return False


def cpu_baseline_record(w, budget_s):
    """The oracle timed on the host: all cores (OpenMP build) as the headline
    figure when the compiler has OpenMP, the serial build beside it."""
    import oracle
    v1, n1, s1 = cpu_oracle_rate(w, budget_s=budget_s)
    rec = {"value": v1, "unit": "spin-steps/s", "cores": 1, "kind": "oracle",
           "sample": f"{n1} FP64 oracle steps (single thread) of the full 128^3 lattice, {s1:.1f} s",
           "cpu_model": _cpu_model(), "host_cores": os.cpu_count()}
    if _omp_available():
        cpu_oracle_rate(w, budget_s=1.0, max_steps=1, threads=True)    # loads the OpenMP build
        vn, nn, sn = cpu_oracle_rate(w, budget_s=budget_s, threads=True)
        rec.update({"value": vn, "cores": oracle.omp_threads(),
                    "sample": f"{nn} FP64 oracle steps of the full 128^3 lattice on {oracle.omp_threads()} "
                              f"OpenMP threads, {sn:.1f} s",
                    "single_core": {"value": v1, "cores": 1,
                                    "sample": f"{n1} steps, single thread, {s1:.1f} s"}})
    return rec


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    import oracle
    w = spin_inputs.WORKLOADS[WORKLOAD]
    threads = _omp_available()
    cores = oracle.omp_threads() if threads else 1
    # bounded samples: the whole run stays within about two minutes
    budget = min(12.0, 120.0 / max(1, args.steps))
    cpu_oracle_rate(w, budget_s=1.0, max_steps=1, threads=threads)   # warm-up: builds/loads the oracle
    vals, secs, nsteps = [], 0.0, 0
    for _ in range(args.steps):
        v, n, dt = cpu_oracle_rate(w, budget_s=budget, max_steps=10, threads=threads)
        vals.append(v)
        secs += dt
        nsteps += n
    N = math.prod(w["n"])
    value = N * nsteps / secs
    how = f"FP64 C oracle, OpenMP over z-planes on {cores} host threads" if threads else "FP64 C oracle, single thread"
    line = {
        "impl": "reference", "metric": "spin-steps/s (128^3 RK4 + pulse noise)", "value": value,
        "unit": "spin-steps/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "128^3 simple-cubic ferromagnet, RK4 dt=0.2, pulse every 10 steps, T=1.0",
                   "impl_note": how},
        "cpu_baseline": {"value": value, "unit": "spin-steps/s", "cores": cores, "kind": "oracle",
                         "sample": f"{nsteps} oracle steps of the full 128^3 lattice over {args.steps} bench steps "
                                   f"({how})",
                         "cpu_model": _cpu_model()},
        "e2e": {"value": value, "unit": "spin-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _e2e_pipelined(torch, lat, R, steps, host_in, stream, barrier):
    """Wall seconds for `steps` noise intervals through the public API with
    host buffers: every interval copies its input state host->device and its
    result state device->host (plus the sample records), the copies on their
    own streams so that they overlap the neighbouring intervals' compute."""
    dev = lat.state.device
    s_in, s_out = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    d_in = [torch.empty_like(lat.state) for _ in range(2)]
    d_out = [torch.empty_like(lat.state) for _ in range(2)]
    host_out = [torch.empty(lat.state.shape, dtype=lat.state.dtype).pin_memory() for _ in range(2)]
    ev = {k: [torch.cuda.Event() for _ in range(2)] for k in ("h2d", "in_free", "out_ready", "out_free")}
    lat.samples()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(steps):
        b = k % 2
        with torch.cuda.stream(s_in):
            if k >= 2:
                s_in.wait_event(ev["in_free"][b])
            d_in[b].copy_(host_in, non_blocking=True)
            ev["h2d"][b].record(s_in)
        with torch.cuda.stream(stream):
            stream.wait_event(ev["h2d"][b])
            lat.state.copy_(d_in[b], non_blocking=True)
            ev["in_free"][b].record(stream)
            lat.step(R)
            if k >= 2:
                stream.wait_event(ev["out_free"][b])
            d_out[b].copy_(lat.state, non_blocking=True)
            ev["out_ready"][b].record(stream)
        with torch.cuda.stream(s_out):
            s_out.wait_event(ev["out_ready"][b])
            host_out[b].copy_(d_out[b], non_blocking=True)
            ev["out_free"][b].record(s_out)
        if (k + 1) % 256 == 0:
            lat.samples()
    lat.samples()
    torch.cuda.synchronize()
    barrier()
    return time.perf_counter() - t0


def adjoint_timing(sp, torch, dev, precision=32, steps=None):
    """fwd+adjoint ms/step on the 64^3 differentiation workload: 500 RK4
    steps with pulses every 10 (recorded, checkpoint every 50), then the
    checkpointed adjoint of E + |M - m*|^2 w.r.t. J, D, H and h_i (FP64
    accumulation).  precision 64 is the plain FP64 comparison arm; steps
    shortens the horizon (accuracy comparison)."""
    w = spin_inputs.WORKLOADS["adjoint64"]
    nx, ny, nz = w["n"]
    p = sp.Params(nx, ny, nz, J=w["J"], D=w["D"], H=w["H"], lam=w["lam"], T=w["T"], dt=w["dt"], R=w["R"],
                  seed=w["noise_seed"], precision=precision)
    s0 = spin_inputs.random_spins(nx, ny, nz, seed=w["spin_seed"])
    hs = spin_inputs.site_fields(nx, ny, nz, w["field_sigma"], seed=w["noise_seed"])
    n, K = (steps or w["steps"]), w["checkpoint"]
    # the whole run twice: the first builds the library's graphs and warms the
    # allocator's cache, the second is timed
    for _ in range(2):
        lat = sp.Lattice(p, torch.from_numpy(s0), h_site=torch.from_numpy(hs), device=dev)
        lat.record(K, n)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lat.step(n)
        M, E = lat.observables()
        t1 = time.perf_counter()
        dLdM = [2.0 * (M[a] - w["m_target"][a]) for a in range(3)]
        g = lat.backward(dLdM, 1.0, field_grad=True)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        gh = g["h"].double().cpu().numpy()
        lat.close()
    return {"workload": f"64^3 FP{precision} RK4, {n} steps, pulse every 10, checkpoint every 50, "
                        "loss E + |M - m*|^2",
            "fwd_ms_per_step": 1e3 * (t1 - t0) / n, "adjoint_ms_per_step": 1e3 * (t2 - t1) / n,
            "fwd_plus_adjoint_ms_per_step": 1e3 * (t2 - t0) / n,
            "grad": {"J": g["J"], "D": g["D"], "H": g["H"]}, "_gh": gh}


def adjoint_vs_fp64(sp, torch, dev, adj32):
    """The FP32 adjoint against the plain FP64 GPU adjoint on the same
    workload: time at the full 500-step horizon, and the FP32 gradients'
    relative error on a 20-step horizon (over 500 steps the pathwise gradient
    grows with the dynamics' chaos, so FP32 and FP64 runs part for physical
    reasons, not through the adjoint)."""
    a64 = adjoint_timing(sp, torch, dev, precision=64)
    s32 = adjoint_timing(sp, torch, dev, precision=32, steps=20)
    s64 = adjoint_timing(sp, torch, dev, precision=64, steps=20)

    def rel(a, b):
        a, b = np.asarray(a, float), np.asarray(b, float)
        return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))

    return {"fp64_fwd_plus_adjoint_ms_per_step": a64["fwd_plus_adjoint_ms_per_step"],
            "fp64_fwd_ms_per_step": a64["fwd_ms_per_step"], "fp64_adjoint_ms_per_step": a64["adjoint_ms_per_step"],
            "fp32_speedup": a64["fwd_plus_adjoint_ms_per_step"] / adj32["fwd_plus_adjoint_ms_per_step"],
            "rel_err_fp32_vs_fp64_20_steps": {"J": rel(s32["grad"]["J"], s64["grad"]["J"]),
                                              "D": rel(s32["grad"]["D"], s64["grad"]["D"]),
                                              "H": rel(s32["grad"]["H"], s64["grad"]["H"]),
                                              "h_i": rel(s32["_gh"], s64["_gh"])}}


def batch_timing(sp, torch, dev, flush, stream, hbm_peak, intervals=3):
    """Throughput of the 512-replica workload (L uniform over {16..64}, T in
    [0.2, 2], RK4 dt=0.2, pulse every 10): whole noise intervals replayed from
    the batch's CUDA graph, L2 flushed before each; the state (~0.5 GB) is
    larger than L2, so the algorithmic-byte fraction is an HBM fraction."""
    w = spin_inputs.WORKLOADS["batch512"]
    L, T = spin_inputs.replica_draws(w["nrep"], w["seed"])
    p = sp.Params(1, 1, 1, J=w["J"], D=w["D"], H=w["H"], lam=w["lam"], dt=w["dt"], R=w["R"], seed=w["seed"],
                  precision=32)
    states = [spin_inputs.random_spins(int(l), int(l), int(l), seed=1000 + r) for r, l in enumerate(L)]
    def run_intervals(b):
        with torch.cuda.stream(stream):
            for _ in range(3):
                b.step(p.R)
            evs = []
            for _ in range(intervals):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                b.step(p.R)
                e1.record(stream)
                evs.append((e0, e1))
        torch.cuda.synchronize()
        return sum(a.elapsed_time(c) for a, c in evs) / 1e3

    with torch.cuda.stream(stream):
        # tiling autotuned per size class at create (fresh, not from a cache)
        b = sp.Batch(p, L, T, states, device=dev, stream=stream, use_cache=False)
    ntot = int(b.offsets[-1])
    tuned = b.tiling()
    items_tuned = b.nitems
    t = run_intervals(b)
    rows = sp.spin_batch_tile_rows(p.integrator)
    with torch.cuda.stream(stream):
        b.set_tiling({l: (rows[0], 32) for l in tuned})
    t_default = run_intervals(b)
    items_default = b.nitems
    rate = ntot * p.R * intervals / t
    b.close()
    out = {"workload": "512 replicas, L in {16,24,32,48,64}, T in [0.2,2], FP32 RK4 dt=0.2, pulse every 10",
           "spins": ntot, "value": rate, "unit": "spin-steps/s", "ms_per_interval": 1e3 * t / intervals,
           "tiling": {str(l): {"tile_rows": r, "chunk": k} for l, (r, k) in sorted(tuned.items())},
           "work_items": items_tuned,
           "default_tiling": {"tile_rows": rows[0], "chunk": 32, "work_items": items_default,
                              "ms_per_interval": 1e3 * t_default / intervals},
           "tuned_speedup_vs_default": t_default / t,
           "hbm_frac_algorithmic": BYTES_PER_SPIN_STEP_FP32 * rate / 1e9 / hbm_peak}
    # comparison arms: the same replicas as separate plain lattices, one
    # interval each, stepped back to back on the stream (FP32: what batching
    # saves; FP64: the plain FP64 GPU step the batched FP32 form replaces)
    for prec in (32, 64):
        lats = []
        with torch.cuda.stream(stream):
            for r, (l, tr) in enumerate(zip(L, T)):
                pr = sp.Params(int(l), int(l), int(l), J=w["J"], D=w["D"], H=w["H"], lam=w["lam"], T=float(tr),
                               dt=w["dt"], R=w["R"], seed=w["seed"], replica=r, precision=prec)
                lt = sp.Lattice(pr, torch.from_numpy(states[r]), device=dev, stream=stream)
                lt.step(pr.R)
                lats.append(lt)
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for lt in lats:
                lt.step(p.R)
            e1.record(stream)
        torch.cuda.synchronize()
        out[f"replica_loop_fp{prec}_ms_per_interval"] = e0.elapsed_time(e1)
        for lt in lats:
            lt.close()
        del lats
    out["batched_speedup_vs_fp64_loop"] = out["replica_loop_fp64_ms_per_interval"] / out["ms_per_interval"]
    out["batched_speedup_vs_fp32_loop"] = out["replica_loop_fp32_ms_per_interval"] / out["ms_per_interval"]
    return out


def single_spin_timing(sp, torch, stream, alu_peak, blocks_per_sm=10, steps32=20000, steps64=2000):
    """Single-spin replica throughput on the escape workload of Sec. III.B
    (renewal first-passage runs, Butcher RK5, delta t = 1/6, Delta t = 1):
    two full waves of 128-thread blocks at 10 resident blocks per SM, FP32
    and FP64, one launch each timed with CUDA events on its stream after a
    warm-up launch; the state (a few MB) is L2-resident and the kernel
    arithmetic-bound, so no flush.  Beside it the C oracle's rate on one
    thread for the same one-spin problem."""
    nrep = 2 * SMS * blocks_per_sm * 128
    out = {"workload": "uniaxial spin in a transverse field, h=1/2, D=1, lambda=0.01, T=0.1, Butcher RK5, "
                       "dt=1/6, pulse every 6 steps, renewal first-passage runs",
           "replicas": nrep, "unit": "replica-steps/s"}
    for prec, steps in ((32, steps32), (64, steps64)):
        with torch.cuda.stream(stream):
            e = _escape_replicas(sp, nrep, prec)   # uploads the noise scales once
            e.stream = stream
            e.run(200)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            e.run(steps)
            b.record(stream)
        torch.cuda.synchronize()
        out[f"fp{prec}"] = nrep * steps / (a.elapsed_time(b) / 1e3)
        out[f"fp{prec}_ms"] = a.elapsed_time(b)
    achieved = out["fp32"] * RK5_FLOPS_PER_SINGLE_STEP / 1e12
    out["roofline"] = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                       "frac": achieved / alu_peak, "flops_per_replica_step": RK5_FLOPS_PER_SINGLE_STEP,
                       "kernel": "k_single_escape<float,PREC=1,6 stages>", "traffic": None,
                       "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz"}
    import oracle
    oracle.build()
    w = ESCAPE
    op = oracle.Params(1, 1, 1, J=0.0, D=w["D"], H=(2 * w["h"] * w["D"], 0.0, 0.0), lam=w["lam"], T=w["T"],
                       dt=w["dt"], R=w["R"], integrator=oracle.RK5_BUTCHER, seed=1)
    s = np.array([w["h"], 0.0, (1 - w["h"] ** 2) ** 0.5]).reshape(3, 1, 1, 1)
    t0 = time.perf_counter()
    n = 200000
    oracle.run(op, s, n)
    out["cpu_oracle"] = {"value": n / (time.perf_counter() - t0), "unit": "replica-steps/s", "cores": 1,
                         "kind": "oracle", "sample": f"{n} FP64 steps of one replica (no stopping)"}
    return out


def noise_model_timing(sp, torch, stream, nrep=2 * SMS * 10 * 128, t_phys=200.0):
    """GPU time per unit of physical time of the three schemes the paper
    compares on the spin in a field (H = 1, lambda = 0.01, T = 1, FP32; Sec.
    III.A): Heun with rectangular noise at delta t = 0.04 (noise drawn every
    step), RK5 with rectangular noise at delta t = 0.25, pulse-noise RK5 at
    delta t = 0.25, Delta t = 10.  One launch each, CUDA events on the stream."""
    schemes = {"heun_rect_dt0.04": (0.04, 1, sp.HEUN, 2), "rk5_rect_dt0.25": (0.25, 1, sp.RK5_BUTCHER, 2),
               "rk5_pulse_dt0.25_Dt10": (0.25, 40, sp.RK5_BUTCHER, 1)}
    out = {"workload": f"spin in a field H=1, lambda=0.01, T=1, FP32, {nrep} replicas",
           "unit": "replica time units per second"}
    for name, (dt, R, integ, noise) in schemes.items():
        p = sp.Params(1, 1, 1, J=0.0, D=0.0, H=(0.0, 0.0, 1.0), lam=0.01, T=1.0, dt=dt, R=R, integrator=integ,
                      precession=1, noise=noise, seed=3, precision=32)
        st = torch.zeros(3, nrep, dtype=torch.float64)
        st[2] = 1.0
        with torch.cuda.stream(stream):
            s = sp.SingleSpins(p, [1.0] * nrep, st, stream=stream)
            n = int(round(t_phys / dt))
            n -= n % R
            s.run(4 * R)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            s.run(n)
            b.record(stream)
        torch.cuda.synchronize()
        out[name] = nrep * n * dt / (a.elapsed_time(b) / 1e3)
    out["pulse_rk5_over_heun"] = out["rk5_pulse_dt0.25_Dt10"] / out["heun_rect_dt0.04"]
    out["rect_rk5_over_heun"] = out["rk5_rect_dt0.25"] / out["heun_rect_dt0.04"]
    return out


def mc_timing(sp, torch, stream, hbm_peak):
    """The paper's speed comparison of Sec. IV on the GPU: checkerboard
    Metropolis, 550 sweeps (the paper's match of t = 2000), against pulse
    noise with precession dropped, delta t = 4, Delta t = 8, 500 steps
    (t = 2000), RK2 midpoint and Butcher RK5; the paper's 64^3 free-boundary
    particle and periodic 128^3 / 256^3 lattices, FP32, T/J = 1, ordered start.
    CUDA events on the stream around each run."""
    out = {"unit": "ms", "sweeps": 550, "pulse_steps": 500}
    for n, bc in ((64, 1), (128, 0), (256, 0)):
        s0 = spin_inputs.aligned_spins(n, n, n)
        pm = sp.Params(n, n, n, J=1.0, T=1.0, bc=bc, precision=32)
        with torch.cuda.stream(stream):
            st = torch.from_numpy(s0).to("cuda", torch.float32).contiguous()
            sp.spin_metropolis_sweeps(pm, st, 10, mc_seed=1, stream=stream)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sp.spin_metropolis_sweeps(pm, st, 550, mc_seed=1, sweep0=10, stream=stream)
            b.record(stream)
        torch.cuda.synchronize()
        mc_ms = a.elapsed_time(b)
        row = {"mc_550_sweeps": mc_ms, "mc_trials_per_s": 550 * n ** 3 / (mc_ms / 1e3),
               "mc_hbm_frac_algorithmic": BYTES_PER_SPIN_STEP_FP32 * 550 * n ** 3 / (mc_ms / 1e3) / 1e9 / hbm_peak}
        for name, integ in (("pulse_rk2_500_steps", sp.RK2_MIDPOINT), ("pulse_rk5_500_steps", sp.RK5_BUTCHER)):
            pp = sp.Params(n, n, n, J=1.0, D=0.0, H=(0.0, 0.0, 0.0), lam=0.01, T=1.0, dt=4.0, R=2,
                           integrator=integ, precession=0, seed=17, precision=32, bc=bc)
            with torch.cuda.stream(stream):
                lat = sp.Lattice(pp, torch.from_numpy(s0), device="cuda:0", stream=stream)
                lat.step(20)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                lat.step(500)
                b.record(stream)
            torch.cuda.synchronize()
            row[name] = a.elapsed_time(b)
            lat.close()
        row["mc_over_pulse_rk2_speed"] = row["pulse_rk2_500_steps"] / mc_ms
        out[f"{n}^3 {'free' if bc else 'periodic'}"] = row
    return out


def time_pulse(torch, lat, R, intervals, stream, flush, plain_ms):
    """Per-launch milliseconds of the noise-pulse kernel: CUDA events around
    the two steps that straddle the pulse (step floor(R/2), which launches the
    fused step and then the pulse kernel, and the plain step after it), minus
    two plain steps.  Starts at the beginning of an interval."""
    h = R // 2
    if h < 1 or h + 1 >= R:
        return None
    pre = h - 1 if (h - 1) % 2 == 0 else h - 2      # an even run of plain steps before the pulse step
    d = []
    with torch.cuda.stream(stream):
        for _ in range(intervals):
            flush.zero_()
            torch.cuda._sleep(3_000_000)
            if pre:
                lat.step(pre)
            if h - 1 - pre:
                lat.step(h - 1 - pre)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            lat.step(2)
            b.record(stream)
            d.append((a, b))
            lat.step(R - h - 1)
    torch.cuda.synchronize()
    return float(np.mean([a.elapsed_time(b) for a, b in d])) - 2 * plain_ms


def kernel_timing_256(sp, torch, dev, flush, stream, hbm_peak):
    """The same fused RK4 step on a 256^3 lattice (201 MB per state copy,
    larger than L2): plain-step launch time and its HBM fraction.  At this
    size the library picks the step with its older planes in tensor memory
    (28-row tiles, no z chunks); the register-ring step (SPIN_TMEM=0) is
    timed beside it."""
    w = dict(spin_inputs.WORKLOADS[WORKLOAD])
    w["n"] = (256, 256, 256)
    p = _params(sp, w, 0)
    s0 = spin_inputs.random_spins(256, 256, 256, seed=w["spin_seed"])
    out = {}
    for label, env in (("tmem", None), ("register_rings", "0")):
        if env is None:
            os.environ.pop("SPIN_TMEM", None)
        else:
            os.environ["SPIN_TMEM"] = env
        try:
            with torch.cuda.stream(stream):
                lat = sp.Lattice(p, torch.from_numpy(s0), device=dev, stream=stream)
                lat.step(p.R)
            out[label] = float(np.mean(time_plain_steps(torch, lat, p.R, 2, stream, flush)))
            lat.close()
        finally:
            os.environ.pop("SPIN_TMEM", None)
    ms = out["tmem"]
    gbs = BYTES_PER_SPIN_STEP_FP32 * p.N / (ms / 1e3) / 1e9
    return {"lattice": "256^3", "kernel": "k_step_patch_tmem<PREC=1> (s and y rings in tensor memory, 28-row tiles)",
            "kernel_ms_per_launch": ms, "achieved_GBps": gbs, "frac": gbs / hbm_peak,
            "spin_steps_per_s": p.N / (ms / 1e3), "register_rings_ms_per_launch": out["register_rings"]}


def fp64_step_timing(sp, torch, dev, flush, stream):
    """The plain FP64 GPU step on the same 128^3 workload (the comparison arm
    for the FP32 path's accuracy/speed trade): plain-step launch time."""
    w = spin_inputs.WORKLOADS[WORKLOAD]
    p = _params(sp, w, 0)
    import dataclasses
    p = dataclasses.replace(p, precision=64)
    s0 = spin_inputs.random_spins(p.nx, p.ny, p.nz, seed=w["spin_seed"])
    with torch.cuda.stream(stream):
        lat = sp.Lattice(p, torch.from_numpy(s0), device=dev, stream=stream)
        lat.step(1)
        flush.zero_()
        torch.cuda._sleep(3_000_000)
        ev = []
        for q in range(3):
            a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            lat.step(1)
            c.record(stream)
            ev.append((a, c))
    torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(c) for a, c in ev]))
    lat.close()
    return {"lattice": "128^3 FP64 RK4 (fused FP64 kernel)", "kernel_ms_per_launch": ms,
            "spin_steps_per_s": p.N / (ms / 1e3)}


def run_ours(args, ws, rank, local):
    import torch

    import paper_1610_04914_gb300 as sp
    from paper_1610_04914_gb300 import build as b

    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    b.build()
    sp.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    w = spin_inputs.WORKLOADS[WORKLOAD]
    p = _params(sp, w, rank)
    N = p.N
    R = p.R
    s0 = spin_inputs.random_spins(p.nx, p.ny, p.nz, seed=w["spin_seed"])
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        lat = sp.Lattice(p, torch.from_numpy(s0), device=dev, stream=stream)
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > L2

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    # warm-up (first interval eager, later ones build and replay the graph)
    for _ in range(max(args.warmup, 3)):
        lat.step(R)
    torch.cuda.synchronize()

    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    clocks.mark_begin()
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            lat.step(R)
            ev[k][1].record(stream)
    torch.cuda.synchronize()
    clocks.mark_end()
    barrier()
    wall = time.perf_counter() - wall0
    step_ms = [a.elapsed_time(bb) for a, bb in ev]
    clk = clocks.stop()
    value, t_dev, _ = whole_job_rate(sum(step_ms) / 1e3, N * R * args.steps)

    # dominant kernel: the fused RK4 step (plain steps), timed with CUDA events
    # on the launching stream around runs of consecutive plain launches
    # (steps 1-4 and 6-9 of each interval: step 5 carries the pulse kernel,
    # step 10 the reduction).  A sleep kernel first lets the host queue the
    # interval, so the events bracket back-to-back kernels, not host latency.
    kern_ms = time_plain_steps(torch, lat, R, max(3, args.steps), stream, flush)
    t_kernel = float(np.mean(kern_ms)) / 1e3
    hbm_peak, peak_src = _measured_peaks()
    achieved_gbs = BYTES_PER_SPIN_STEP_FP32 * N / t_kernel / 1e9
    achieved_tflops = RK4_FLOPS_PER_SPIN_STEP * N / t_kernel / 1e12
    alu_peak = SMS * FP32_LANES * 2 * MAX_SM_MHZ * 1e6 / 1e12
    traffic = _ncu_traffic()
    pulse_ms = time_pulse(torch, lat, R, max(3, args.steps), stream, flush, float(np.mean(kern_ms)))
    pulse = None
    if pulse_ms is not None and pulse_ms > 0:
        pulse_gbs = BYTES_PER_SPIN_STEP_FP32 * N / (pulse_ms / 1e3) / 1e9
        pulse = {"kernel": "k_pulse_f32 (Philox4x64-10 + Box-Muller + rotation, Eq. s_rotation)",
                 "ms_per_launch": pulse_ms, "launches_per_step": 1.0 / R,
                 "algorithmic_bytes_per_launch": BYTES_PER_SPIN_STEP_FP32 * N, "achieved_GBps": pulse_gbs,
                 "frac_hbm": pulse_gbs / hbm_peak,
                 "how": "the pulse step and the next plain step by CUDA events, minus two plain steps",
                 "bound": "64-bit integer multiplies of the counter-based generator (20 per site)"}

    # end to end through the public API with host buffers
    host_in = torch.from_numpy(s0.astype(np.float32)).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    e2e_t = []
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lat.state.copy_(host_in, non_blocking=True)
            lat.step(R)
            host_out.copy_(lat.state, non_blocking=True)
            smp = lat.samples()          # synchronises the stream; reads the sample record
            stream.synchronize()
            e2e_t.append(time.perf_counter() - t0)
    e2e_serial, _, _ = whole_job_rate(sum(e2e_t), N * R * args.steps)
    h2d = host_in.numel() * host_in.element_size()
    d2h = host_out.numel() * host_out.element_size() + 5 * 8

    # the same, pipelined: each interval's input arrives host->device on a copy
    # stream into a device staging buffer while the previous interval
    # computes, and each interval's result state is snapshotted on the device
    # and read back device->host on a third stream while the next computes;
    # the sample records are read every 256 intervals and at the end
    e2e_secs = _e2e_pipelined(torch, lat, R, args.steps, host_in, stream, barrier)
    e2e_value, _, _ = whole_job_rate(e2e_secs, N * R * args.steps)

    adj = adjoint_timing(sp, torch, dev) if rank == 0 and not args.no_extra else None
    if adj is not None:
        adj.pop("_gh")
        adj["vs_fp64"] = adjoint_vs_fp64(sp, torch, dev, adj)
        n_adj = int(np.prod(spin_inputs.WORKLOADS["adjoint64"]["n"]))
        hbm_pk, pk_src = _measured_peaks()
        ach = ADJ_BYTES_PER_SPIN_STEP * n_adj / (adj["adjoint_ms_per_step"] * 1e-3) / 1e9
        adj["roofline"] = {"bound": "hbm", "achieved": ach, "peak": hbm_pk, "unit": "GB/s", "frac": ach / hbm_pk,
                           "bytes_per_spin_step": ADJ_BYTES_PER_SPIN_STEP, "traffic": None,
                           "peak_source": f"{pk_src} HBM copy bandwidth",
                           "note": "whole backward pass per step (recompute + transposes) by wall clock"}
    bat = batch_timing(sp, torch, dev, flush, stream, hbm_peak) if rank == 0 and not args.no_extra else None
    k256 = kernel_timing_256(sp, torch, dev, flush, stream, hbm_peak) if rank == 0 and not args.no_extra else None
    f64 = fp64_step_timing(sp, torch, dev, flush, stream) if rank == 0 and not args.no_extra else None
    single = single_spin_timing(sp, torch, stream, alu_peak) if rank == 0 and not args.no_extra else None
    noise_models = noise_model_timing(sp, torch, stream) if rank == 0 and not args.no_extra else None
    mc = mc_timing(sp, torch, stream, hbm_peak) if rank == 0 and not args.no_extra else None

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_record(w, budget_s=float(os.environ.get("SPIN_CPU_BUDGET_S", "12")))

    if rank == 0:
        frac_hbm = achieved_gbs / hbm_peak
        frac_alu = achieved_tflops / alu_peak
        roof_hbm = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": frac_hbm,
                    "traffic": (traffic["dram_bytes_per_launch"] if traffic else None),
                    "peak_source": f"{peak_src} HBM copy bandwidth",
                    "kernel": "k_step_patch<4,PREC=1,HSITE=0,PULSE=0> (fused RK4 step, plain steps)",
                    "kernel_ms_per_launch": t_kernel * 1e3,
                    "algorithmic_bytes_per_launch": BYTES_PER_SPIN_STEP_FP32 * N}
        roof_alu = {"bound": "alu", "achieved": achieved_tflops, "peak": alu_peak, "unit": "TFLOP/s",
                    "frac": frac_alu, "flops_per_spin_step": RK4_FLOPS_PER_SPIN_STEP,
                    "traffic": roof_hbm["traffic"], "kernel": roof_hbm["kernel"],
                    "kernel_ms_per_launch": t_kernel * 1e3,
                    "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz"}
        # the roof the kernel sits closest to (arithmetic intensity 10 flop/B
        # against a ridge of 11.8 flop/B: the HBM roof is the lower one)
        roof = roof_hbm if frac_hbm >= frac_alu else roof_alu
        line = {
            "metric": "spin-steps/s (128^3 RK4 + pulse noise)", "value": value, "unit": "spin-steps/s",
            "n_gpus": ws, "steps": args.steps, "warmup": max(args.warmup, 3),
            "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "128^3 simple-cubic ferromagnet, FP32 state, RK4 dt=0.2, pulse every 10 steps "
                                   "(one bench step = one noise interval: 10 steps + pulse + FP64 sample), "
                                   "J=1, D=0.05, H=(0,0,0.02), lambda=0.01, T=1.0",
                       "l2": "flushed (256 MiB write) before every timed step",
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
            "roofline": roof,
            "roofline_hbm": roof_hbm,
            "roofline_alu": roof_alu,
            "pulse": pulse,
            "e2e": {"value": e2e_value, "unit": "spin-steps/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h,
                    "mode": "copies on their own streams, overlapped with the neighbouring intervals' compute",
                    "serial_value": e2e_serial},
            "gpu_launches": args.steps * (R + 3),   # R steps + pulse + 2 reduction kernels per interval
            "clocks": clk,
            "adjoint": adj,
            "batched": bat,
            "roofline_256": k256,
            "fp64_step": f64,
            "single_spin": single,
            "noise_models": noise_models,
            "metropolis_vs_pulse": mc,
            "wall_s_timed_region": wall,
            "cpu_baseline": cpu,
            # the metric's third part, repeated last so that a reader of the
            # line's tail sees it: 64^3 FP32 forward + checkpointed adjoint
            "fwd_plus_adjoint_ms_per_step": adj["fwd_plus_adjoint_ms_per_step"] if adj else None,
        }
        print(json.dumps(line), flush=True)
    lat.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


ESCAPE = dict(D=1.0, h=0.5, lam=0.01, T=0.1, dt=1.0 / 6.0, R=6)


def _escape_replicas(sp, nrep, precision):
    """Renewal first-passage replicas of the escape workload (Sec. III.B)."""
    w = ESCAPE
    p = sp.Params(1, 1, 1, J=0.0, D=w["D"], H=(2 * w["h"] * w["D"], 0.0, 0.0), lam=w["lam"], T=w["T"], dt=w["dt"],
                  R=w["R"], integrator=sp.RK5_BUTCHER, precession=1, seed=1, precision=precision)
    return sp.EscapeReplicas(p, [w["T"]] * nrep, (w["h"], 0.0, (1 - w["h"] ** 2) ** 0.5))


def run_profile_case(args):
    """A small fixed case for ncu: the benchmark's physics on an L^3 FP32
    lattice, advanced by single eager steps (step 5 of each interval carries
    the pulse); --profile-integrator rk5 runs Butcher RK5 instead of RK4."""
    import torch

    import paper_1610_04914_gb300 as sp
    from paper_1610_04914_gb300 import build as b
    b.build()
    sp.load()
    w = dict(spin_inputs.WORKLOADS[WORKLOAD])
    L = args.profile_lattice
    w["n"] = (L, L, L)
    p = _params(sp, w, 0)
    if args.profile_integrator == "rk5":
        import dataclasses
        p = dataclasses.replace(p, integrator=sp.RK5_BUTCHER)
    s0 = spin_inputs.random_spins(L, L, L, seed=w["spin_seed"])
    lat = sp.Lattice(p, torch.from_numpy(s0), device="cuda:0")
    for _ in range(args.profile_steps):
        lat.step(1)
    torch.cuda.synchronize()
    M, E = lat.observables()
    print(json.dumps({"profile_lattice": L, "steps": args.profile_steps, "M": M, "E": E}))
    lat.close()
    return 0


def run_profile_mc(args):
    """A small fixed case for ncu: checkerboard Metropolis on an L^3 periodic
    FP32 ferromagnet at T/J = 1 from random spins, --profile-steps sweeps."""
    import torch

    import paper_1610_04914_gb300 as sp
    from paper_1610_04914_gb300 import build as b
    b.build()
    sp.load()
    L = args.profile_mc
    p = sp.Params(L, L, L, J=1.0, T=1.0, precision=32)
    st = torch.from_numpy(spin_inputs.random_spins(L, L, L, seed=1)).to("cuda", torch.float32).contiguous()
    acc = torch.zeros(1, dtype=torch.int64, device="cuda")
    sp.spin_metropolis_sweeps(p, st, args.profile_steps, mc_seed=1, accepted=acc)
    torch.cuda.synchronize()
    print(json.dumps({"profile_mc": L, "sweeps": args.profile_steps,
                      "acceptance": int(acc.item()) / (args.profile_steps * L ** 3)}))
    return 0


def run_profile_adjoint(args):
    """A fixed case for ncu launch lists: the 64^3 differentiation workload
    (FP32 RK4, pulse every 10, h_i, checkpoint every 50), --profile-steps
    recorded forward steps, then the checkpointed adjoint; prints the
    wall-clock split."""
    import torch

    import paper_1610_04914_gb300 as sp
    from paper_1610_04914_gb300 import build as b
    b.build()
    sp.load()
    w = spin_inputs.WORKLOADS["adjoint64"]
    nx, ny, nz = w["n"]
    p = sp.Params(nx, ny, nz, J=w["J"], D=w["D"], H=w["H"], lam=w["lam"], T=w["T"], dt=w["dt"], R=w["R"],
                  seed=w["noise_seed"], precision=32)
    lat = sp.Lattice(p, torch.from_numpy(spin_inputs.random_spins(nx, ny, nz, seed=w["spin_seed"])),
                     h_site=torch.from_numpy(spin_inputs.site_fields(nx, ny, nz, w["field_sigma"],
                                                                     seed=w["noise_seed"])))
    n = args.profile_steps
    lat.record(w["checkpoint"], n)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lat.step(n)
    M, E = lat.observables()
    t1 = time.perf_counter()
    g = lat.backward([2.0 * (M[a] - w["m_target"][a]) for a in range(3)], 1.0, field_grad=True)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    print(json.dumps({"profile_adjoint": n, "fwd_ms_per_step": 1e3 * (t1 - t0) / n,
                      "adjoint_ms_per_step": 1e3 * (t2 - t1) / n, "gJ": g["J"]}))
    lat.close()
    return 0


def run_profile_single(args):
    """A small fixed case for ncu: the escape workload of Sec. III.B (h = 1/2,
    D = 1, lambda = 0.01, T = 0.1, Butcher RK5, delta t = 1/6, Delta t = 1,
    FP32), nrep replicas, one warm-up launch of 100 steps then one launch of
    --profile-steps steps."""
    import torch

    import paper_1610_04914_gb300 as sp
    from paper_1610_04914_gb300 import build as b
    b.build()
    sp.load()
    nrep = args.profile_single
    e = _escape_replicas(sp, nrep, 32)
    e.run(100)
    e.run(args.profile_steps)
    torch.cuda.synchronize()
    print(json.dumps({"profile_single": nrep, "steps": args.profile_steps, "passages": int(e.fpt_count.sum())}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=150)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the adjoint, batched and 256^3 side measurements")
    ap.add_argument("--profile-lattice", type=int, default=0,
                    help="profiling driver: L^3 FP32 RK4 lattice, --profile-steps single steps, no timing")
    ap.add_argument("--profile-steps", type=int, default=4)
    ap.add_argument("--profile-integrator", default="rk4", choices=["rk4", "rk5"],
                    help="integrator of --profile-lattice")
    ap.add_argument("--profile-adjoint", action="store_true",
                    help="profiling driver: 64^3 adjoint workload with --profile-steps steps")
    ap.add_argument("--profile-mc", type=int, default=0,
                    help="profiling driver: checkerboard Metropolis on an L^3 lattice, --profile-steps sweeps")
    ap.add_argument("--profile-single", type=int, default=0,
                    help="profiling driver: escape workload with this many single-spin replicas, no timing")
    args = ap.parse_args()
    ws, rank, local = _dist()
    if args.profile_lattice:
        return run_profile_case(args)
    if args.profile_single:
        return run_profile_single(args)
    if args.profile_mc:
        return run_profile_mc(args)
    if args.profile_adjoint:
        return run_profile_adjoint(args)
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    return run_ours(args, ws, rank, local)


if __name__ == "__main__":
    sys.exit(main())
