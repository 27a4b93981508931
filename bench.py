"""Throughput of the QVA hot path on GB300: amplitude-layer updates per second for one
objective + adjoint-gradient solve of QAOA weighted max-cut, n = 28 qubits (2^28 complex64
amplitudes), G(28, 1/2) with U[0,1] weights, p = 8 layers.

One step = qvs_gradient on that instance: forward evolution through 8 layers (phase + hypercube
mixer), the objective <psi|Q|psi> and the adjoint sweep giving all 16 gradient entries.
Units: 2^28 * 8 amplitude-layer updates per step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the fp64 CPU oracle (the only reference: the paper ships no code) on a
bounded sample of the same workload family. Under torchrun (N > 1) every rank runs an independent
replica (the path does not shard across ranks); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

N_QUBITS = 28
P_LAYERS = 8
METRIC = "amplitude-layer updates/s (fwd+adjoint grad) n=28 QAOA; % of HBM peak"
UNIT = "amp-layer/s"
WORKLOAD = "QAOA weighted max-cut, n=28 (2^28 complex64 amplitudes), G(28,1/2) U[0,1] weights, p=8, objective + adjoint gradient"


# DRAM traffic of the dominant kernel per amplitude: ncu dram__bytes_read.sum +
# dram__bytes_write.sum of one capture at n = 25, averaged over the launch mix of the n = 28, p = 8
# solve, with the sha256 of the kernel sources it was taken on. Reported only while the sources
# still hash to that value (null otherwise: the capture no longer describes the built kernel).
TRAFFIC = {"hc_pass_R1_c64": {"bytes_per_amp": 32.0,
                              "sources_sha256": "7c1a236ef3537adea55cb14b82f65ae2f027be52b49a9734c8997ab13b9cd97a"}}
TRAFFIC_SOURCES = ["hc_kernels.cuh", "hc_pass.cuh", "hc_staged.cuh", "hypercube.cu", "hc_pass_th_a.cu",
                   "hc_pass_th_b.cu", "hc_pass_th_c.cu", "hc_pass_th_d.cu"]
GOLDEN = os.path.join(ROOT, "tests", "golden")


def kernel_sources_sha256() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_2110_03963_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _traffic_per_launch(kernel: str, amplitudes: int):
    """ncu DRAM bytes per launch of `kernel` at the benchmark size, or None when the capture no
    longer describes the built kernels."""
    t = TRAFFIC.get(kernel)
    if t is None or t["sources_sha256"] != kernel_sources_sha256():
        return None
    return t["bytes_per_amp"] * amplitudes


def _stored_oracle(name: str):
    """Stored fp64 oracle values of a benchmark instance (written by the oracle-only script beside
    the test fixtures), or None."""
    path = os.path.join(GOLDEN, f"oracle_{name}.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        return json.load(f)


def _rel(a, b):
    return abs(a - b) / max(abs(b), 1e-30)


def _grad_err(dg, dt, rdg, rdt):
    g = np.concatenate([np.asarray(dg), np.asarray(dt)])
    r = np.concatenate([np.asarray(rdg), np.asarray(rdt)])
    return float(np.max(np.abs(g - r)) / max(np.max(np.abs(r)), 1e-30))


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while the timed region runs."""

    FIELDS = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
             "clocks_event_reasons.sw_power_cap"

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.first = 0

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_first(self, timeout: float = 3.0):
        """Wait (at most `timeout` s) for the first sample, so that nvidia-smi's start-up lies
        before the timed region."""
        t_end = time.time() + timeout
        while self.proc is not None and not self.lines and time.time() < t_end:
            time.sleep(0.02)

    def mark(self):
        """The timed region starts: the summary uses the samples from here on (all of them when
        none arrives before stop)."""
        self.first = len(self.lines)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in (self.lines[self.first:] if len(self.lines) > self.first else self.lines):
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


def qubo_scale_bits(c, h, J) -> int:
    """F of the fixed-point rule of qvs_set_quality_qubo (reported in the config only)."""
    n = len(h)
    S = abs(c) + sum(abs(x) for x in h) + sum(abs(J[u][v]) for u in range(n) for v in range(u + 1, n))
    F = 40
    while F > -30 and S * 2.0 ** F + 1024.0 > 2.0 ** 30:
        F -= 1
    return F


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def replica_aggregate(local_ms: float, units_per_rank: float, world: int, allreduce_max=None):
    """Whole-job figures of `world` independent replicas (the path does not shard): the step time
    is the maximum over ranks (allreduce_max reduces one float across ranks), and the throughput
    counts every rank's units. Returns (ms, units per second)."""
    ms = float(allreduce_max(local_ms)) if world > 1 else float(local_ms)
    return ms, units_per_rank * world / (ms * 1e-3)


# ------------------------------------------------------------------ CPU oracle sample

def oracle_sample(seconds_target: float = 15.0):
    """Time the fp64 numpy oracle (as it stands) on the same workload family: weighted max-cut on
    G(n, 1/2), p = 8, objective + adjoint gradient, at the largest n (starting from 16) whose
    solve stays near the time target. Returns (amp-layer/s, description)."""
    import oracle as orc
    best = None
    for n in range(16, N_QUBITS + 1):
        inst = wl.wmaxcut(n, P_LAYERS)
        G = inst.graph
        prob = orc.maxcut_problem(n, G.eu, G.ev, G.w, q_dtype=np.float32)
        t0 = time.perf_counter()
        orc.gradient(prob, inst.gammas, inst.ts)
        dt = time.perf_counter() - t0
        best = (n, dt)
        if dt * 2.2 > seconds_target:
            break
    n, dt = best
    rate = (1 << n) * P_LAYERS / dt
    desc = (f"oracle (numpy fp64, single thread) objective + adjoint gradient of weighted max-cut on G({n},1/2), "
            f"p={P_LAYERS}: {dt:.2f} s per solve of 2^{n} amplitudes")
    return rate, desc, n


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the baseline record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def _host_numa(ptr: int, nbytes: int, gpu_index: int):
    """Where a host buffer's pages live relative to the GPU: {"buffer_pages": {"N0": pages, ...},
    "gpu_node": node}, the pages summed over the mappings (/proc/self/maps, numa_maps) that overlap
    the buffer, the node from the GPU's PCI device in sysfs; None for a part that cannot be read (a
    diagnostic of the upload rate only)."""
    out = {"buffer_pages": None, "gpu_node": None}
    try:
        starts = set()
        with open("/proc/self/maps") as f:
            for ln in f:
                lo, hi = (int(x, 16) for x in ln.split()[0].split("-"))
                if lo < ptr + nbytes and hi > ptr:
                    starts.add(lo)
        pages = {}
        with open("/proc/self/numa_maps") as f:
            for ln in f:
                parts = ln.split()
                if parts and int(parts[0], 16) in starts:
                    for x in parts[2:]:
                        k, _, v = x.partition("=")
                        if k.startswith("N") and k[1:].isdigit():
                            pages[k] = pages.get(k, 0) + int(v)
        out["buffer_pages"] = pages or None
    except Exception:   # a diagnostic: never let it stop the bench
        pass
    try:
        bus = subprocess.run(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=pci.bus_id", "--format=csv,noheader"],
                             capture_output=True, text=True, timeout=20).stdout.strip().lower()
        dom, rest = bus.split(":", 1)
        with open(f"/sys/bus/pci/devices/{dom[-4:]}:{rest}/numa_node") as f:
            out["gpu_node"] = int(f.read().strip())
    except Exception:
        pass
    return out


def _oracle_solve_worker(args):
    """One oracle objective + adjoint-gradient solve (run in a spawned worker process)."""
    n, instance = args
    import oracle as orc
    inst = wl.wmaxcut(n, P_LAYERS, instance=instance)
    G = inst.graph
    prob = orc.maxcut_problem(n, G.eu, G.ev, G.w, q_dtype=np.float32)
    t0 = time.perf_counter()
    orc.gradient(prob, inst.gammas, inst.ts)
    return time.perf_counter() - t0


class OracleCores:
    """The oracle on every host core at once: a pool of spawned single-threaded workers (spawn, so
    no worker inherits a CUDA context), each solving its own instance of the workload family.
    Throughput = workers x 2^n x p amplitude-layers / wall time of the whole round."""

    def __init__(self, cores=None):
        import multiprocessing as mp
        self.cores = int(cores or os.cpu_count() or 1)
        for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[var] = "1"
        self.pool = mp.get_context("spawn").Pool(self.cores)

    def close(self):
        self.pool.close()
        self.pool.join()

    def pick_n(self, seconds_target: float) -> int:
        """Largest n (16..22) whose parallel round is predicted to stay within the target, from
        one timed n = 16 round (time doubles per qubit)."""
        t16 = max(self.round(16)[0], 1e-3)
        n = 16
        while n < 22 and t16 * 2.0 ** (n + 1 - 16) <= seconds_target:
            n += 1
        return n

    def round(self, n: int, base: int = 0):
        t0 = time.perf_counter()
        per = self.pool.map(_oracle_solve_worker, [(n, base + i) for i in range(self.cores)])
        wall = time.perf_counter() - t0
        rate = self.cores * (1 << n) * P_LAYERS / wall
        return wall, rate, per


def oracle_all_cores(seconds_target: float = 15.0):
    pool = OracleCores()
    try:
        n = pool.pick_n(seconds_target)
        wall, rate, per = pool.round(n, base=1000)
    finally:
        pool.close()
    desc = (f"oracle (numpy fp64) on {pool.cores} worker processes, one single-threaded objective + adjoint "
            f"gradient of weighted max-cut on G({n},1/2), p={P_LAYERS} each: {wall:.2f} s wall for "
            f"{pool.cores} solves of 2^{n} amplitudes (per solve {min(per):.2f}-{max(per):.2f} s)")
    return rate, desc, n, pool.cores


def run_reference(args):
    """The oracle (the reference arm: the paper ships no code) on all host cores; each step is one
    round of per-core solves of the same workload family at a bounded size."""
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    t_all = time.perf_counter()
    pool = OracleCores()
    try:
        target = max(2.0, 120.0 / max(1, args.warmup + args.steps))
        n_used = pool.pick_n(target)
        vals, walls = [], []
        for i in range(args.warmup + args.steps):
            wall, rate, _ = pool.round(n_used, base=100 * i)
            if i >= args.warmup:
                vals.append(rate)
                walls.append(wall)
    finally:
        pool.close()
    value = float(np.median(vals))
    desc = (f"oracle (numpy fp64) on {pool.cores} worker processes, each step one single-threaded objective + "
            f"adjoint gradient per worker of weighted max-cut on G({n_used},1/2), p={P_LAYERS}; host CPU: "
            f"{cpu_model()}")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": float(np.median(walls)) * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_n_qubits": n_used, "solves_per_step": pool.cores},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": time.perf_counter() - t_all,
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ the other hot-path configurations

def _time_steps(torch, stream, fn, steps, warmup):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def _kernel_summary(qvs, h, peak, nsteps):
    stats = qvs.qvs_kernel_stats(h)
    if not stats:
        return None, {}
    total = sum(s["ms"] for s in stats) or 1.0
    top = max(stats, key=lambda s: s["ms"])
    gbps = top["bytes"] / (top["ms"] * 1e-3) / 1e9
    roof = {"bound": "hbm", "kernel": top["name"], "achieved": gbps, "peak": peak, "unit": "GB/s",
            "frac": gbps / peak, "peak_source": "measured" if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else "fallback"}
    ker = {s["name"]: {"launches_per_step": s["launches"] / nsteps, "avg_ms": s["ms"] / s["launches"],
                       "share": s["ms"] / total} for s in stats}
    return roof, ker


def run_extras(qvs, torch, stream, peak, steps, warmup, only=None, qwoa_n=26, qwoa_p=6, qaoaz_n=24, qaoaz_p=4,
               batch_count=4096, headline=None):
    # the batched lines tune their schedule afresh (a schedule cache in the user's home directory
    # from an earlier run on another GPU or build would otherwise be reused)
    import tempfile
    os.environ.setdefault("QVS_TUNE_CACHE", os.path.join(tempfile.mkdtemp(prefix="qvs_tune_"), "batch_tune.json"))
    """Objective + adjoint-gradient throughput of the QWOA circulant (N=2^26, p=6), QAOAz CSR
    (n=24, weight 12, p=4) and batched QAOA (4096 instances) workloads."""
    out = {}
    if only in (None, "c128"):
        out.update(_extra_config1(qvs, torch, stream, steps, warmup))
        out.update(_extra_c128_n28(qvs, torch, stream, peak, steps, warmup, headline))
    if only is None:
        out.update(_extra_inpass(qvs, torch, stream, peak, steps, warmup))
        out.update(_extra_exqaoa(qvs, torch, stream, peak, steps, warmup))
    if only in (None, "qwoa"):
        out.update(_extra_qwoa(qvs, torch, stream, peak, steps, warmup, qwoa_n, qwoa_p))
    if only in (None, "parity"):
        out.update(_extra_parity(qvs, torch, stream, peak, steps, warmup, qaoaz_n if only == "parity" else 24,
                                 qaoaz_p if only == "parity" else 4))
    if only in (None, "qaoaz"):
        out.update(_extra_qaoaz(qvs, torch, stream, peak, steps, warmup, qaoaz_n, qaoaz_p))
    if only in (None, "batch"):
        out.update(_extra_batch(qvs, torch, stream, peak, steps, warmup, batch_count, plain=only is None))
    return out


def _extra_config1(qvs, torch, stream, steps, warmup):
    """QAOA max-cut, n = 10, random 3-regular graph, integer qualities, p = 2, complex128, forward
    objective only: latency of one evolve + expectation call (host arrays in, E out)."""
    inst = wl.maxcut10()
    G = inst.graph
    n, p = 10, 2
    q = torch.empty(1 << n, dtype=torch.int32, device="cuda")
    qvs.qvs_quality_maxcut(n, G.eu, G.ev, None, q, qvs.QVS_I32, stream)
    sim = qvs.Simulator(1 << n, qvs.QVS_C128, stream)
    sim.set_quality(q).set_mixer(qvs.QVS_MIX_HYPERCUBE, qvs.hypercube_desc(n))
    reps = 2000
    for _ in range(50):
        E = sim.evolve(inst.gammas, inst.ts)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        E = sim.evolve(inst.gammas, inst.ts)
    us = (time.perf_counter() - t0) / reps * 1e6
    launches = sim.launches()
    sim.close()
    ref = _stored_oracle("maxcut3_n10_p2")
    units = float(1 << n) * p
    return {"qaoa_maxcut3_n10_p2_c128_forward": {
        "value": units / (us * 1e-6), "unit": UNIT, "us_per_solve": us, "launches_per_solve": launches,
        "timing": "host wall clock per qvs_evolve + qvs_expectation call (synchronous), mean of %d" % reps,
        "objective": E, "rel_err_E_vs_oracle": _rel(E, ref["f"]) if ref else None}}


def _extra_c128_n28(qvs, torch, stream, peak, steps, warmup, headline):
    """The plain complex128 path on the benchmark instance (the fp64-accuracy GPU solve), timed
    beside the complex64 line, and the complex64 result's errors against it and against the stored
    fp64 oracle objective."""
    n, p = N_QUBITS, P_LAYERS
    inst = wl.wmaxcut(n, p)
    G = inst.graph
    q = torch.empty(1 << n, dtype=torch.float32, device="cuda")
    qvs.qvs_quality_maxcut(n, G.eu, G.ev, G.w, q, qvs.QVS_F32, stream)
    sim = qvs.Simulator(1 << n, qvs.QVS_C128, stream)
    sim.set_quality(q).set_mixer(qvs.QVS_MIX_HYPERCUBE, qvs.hypercube_desc(n))
    del q
    gs, ts = np.asarray(inst.gammas), np.asarray(inst.ts)
    ms = _time_steps(torch, stream, lambda: sim.gradient(gs, ts), max(3, steps // 3), max(1, warmup // 2))
    E, dg, dt = sim.gradient(gs, ts)
    sim.set_option(qvs.QVS_OPT_PROFILE, 1)
    sim.gradient(gs, ts)
    roof, ker = _kernel_summary(qvs, sim.h, peak, 1)
    sim.close()
    torch.cuda.empty_cache()
    ref = _stored_oracle(f"wmaxcut_n{n}_p{p}")
    units = float(1 << n) * p
    entry = {"value": units / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "dtype": "c128",
             "objective": E, "roofline": roof, "kernels": ker,
             "rel_err_E_vs_oracle": _rel(E, ref["f"]) if ref else None}
    if headline is not None:
        E64, dg64, dt64 = headline
        entry["c64_headline_errors"] = {
            "rel_err_E_vs_c128": _rel(E64, E), "max_rel_grad_err_vs_c128": _grad_err(dg64, dt64, dg, dt),
            "rel_err_E_vs_oracle": _rel(E64, ref["f"]) if ref else None}
    return {f"qaoa_wmaxcut_n{n}_p{p}_c128": entry}


def _extra_inpass(qvs, torch, stream, peak, steps, warmup, n=N_QUBITS, p=P_LAYERS):
    """The benchmark instance with its max-cut cost given as a quadratic form: the phase passes
    evaluate q in the pass (no quality vector in HBM); e2e uploads the form each step."""
    inst = wl.wmaxcut(n, p)
    G = inst.graph
    c, h, J = qvs.qvs_qubo_from_maxcut(n, G.eu, G.ev, G.w)
    sim = qvs.Simulator(1 << n, qvs.QVS_C64, stream)
    sim.set_quality_qubo(n, c, h, J).set_mixer(qvs.QVS_MIX_HYPERCUBE, qvs.hypercube_desc(n))
    gs, ts = np.asarray(inst.gammas), np.asarray(inst.ts)
    ms = _time_steps(torch, stream, lambda: sim.gradient(gs, ts), steps, warmup)
    sim.set_option(qvs.QVS_OPT_PROFILE, 1)
    for _ in range(2):
        sim.gradient(gs, ts)
    roof, ker = _kernel_summary(qvs, sim.h, peak, 2)
    sim.set_option(qvs.QVS_OPT_PROFILE, 0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps = max(3, steps // 2)
    for _ in range(e2e_steps):
        sim.set_quality_qubo(n, c, h, J)
        sim.gradient(gs, ts)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    sim.close()
    units = float(1 << n) * p
    return {f"qaoa_wmaxcut_n{n}_p{p}_quality_in_pass": {
        "value": units / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
        "quality": "quadratic form, fixed point 2^-%d, evaluated in the phase passes" % qubo_scale_bits(c, h, J),
        "e2e": {"value": units / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 8 * (1 + n + n * n) + 16 * p,
                "d2h_bytes_per_step": 8 * (1 + 2 * p)},
        "roofline": roof, "kernels": ker}}


def _extra_exqaoa(qvs, torch, stream, peak, steps, warmup, n=N_QUBITS, p=P_LAYERS):
    """ex-QAOA (Sec. 2.3.2) on the benchmark graph: one gamma per edge term 1/2 w_e Z_u Z_v (Example 2's
    form), gammas uniform on [0, pi]; objective + gradient of all p * (1 + |E|) parameters."""
    inst = wl.wmaxcut(n, p)
    G = inst.graph
    q = torch.empty(1 << n, dtype=torch.float32, device="cuda")
    qvs.qvs_quality_maxcut(n, G.eu, G.ev, G.w, q, qvs.QVS_F32, stream)
    sim = qvs.Simulator(1 << n, qvs.QVS_C64, stream)
    sim.set_quality(q).set_mixer(qvs.QVS_MIX_HYPERCUBE, qvs.hypercube_desc(n))
    sim.set_phase_terms(G.eu, G.ev, [0.5 * w for w in G.w])
    Gm = wl.rng_for(190).uniform(0.0, math.pi, size=(p, len(G.eu)))
    ts = np.asarray(inst.ts)
    ms = _time_steps(torch, stream, lambda: sim.gradient_ex(Gm, ts), steps, warmup)
    sim.set_option(qvs.QVS_OPT_PROFILE, 1)
    for _ in range(2):
        sim.gradient_ex(Gm, ts)
    roof, ker = _kernel_summary(qvs, sim.h, peak, 2)
    sim.close()
    del q
    torch.cuda.empty_cache()
    units = float(1 << n) * p
    return {f"exqaoa_wmaxcut_n{n}_p{p}_{len(G.eu)}terms": {
        "value": units / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
        "parameters": p * (1 + len(G.eu)), "roofline": roof, "kernels": ker}}


def _extra_qwoa(qvs, torch, stream, peak, steps, warmup, n, p):
    out = {}
    inst = wl.qwoa(n, p)
    q = torch.empty(1 << n, dtype=torch.float32, device="cuda")
    qvs.qvs_quality_subset(n, inst.weights, q, qvs.QVS_F32, stream)
    sim = qvs.Simulator(1 << n, qvs.QVS_C64, stream)
    sim.set_quality(q).set_mixer(qvs.QVS_MIX_CIRCULANT, qvs.circulant_desc(inst.offsets))
    ms = _time_steps(torch, stream, lambda: sim.gradient(inst.gammas, inst.ts), steps, warmup)
    sim.set_option(qvs.QVS_OPT_PROFILE, 1)
    for _ in range(2):
        sim.gradient(inst.gammas, inst.ts)
    roof, ker = _kernel_summary(qvs, sim.h, peak, 2)
    units = float(1 << n) * p
    out[f"qwoa_circulant_n{n}_p{p}"] = {"value": units / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
                                        "launches_per_step": sim.launches(), "roofline": roof, "kernels": ker}
    sim.close()
    return out


def _extra_parity(qvs, torch, stream, peak, steps, warmup, n, p, A=2):
    """QAOAz with the paper's parity-ring mixer (Sec. 2.4.1) on the full 2^n register: portfolio
    qualities of every basis state, parity initial state with constraint value A."""
    out = {}
    dim = 1 << n
    port = wl.portfolio(n // 2, wl.rng_for(99, n))
    states = torch.arange(dim, dtype=torch.int64, device="cuda")
    q = torch.empty(dim, dtype=torch.float32, device="cuda")
    qvs.qvs_quality_portfolio(n, states, port.returns, port.cov, port.omega, q, qvs.QVS_F32, stream)
    del states
    psi0 = torch.empty(dim, dtype=torch.complex64, device="cuda")
    qvs.qvs_state_parity(n, A, psi0, stream)
    sim = qvs.Simulator(dim, qvs.QVS_C64, stream)
    sim.set_quality(q).set_mixer(qvs.QVS_MIX_PARITY, qvs.parity_desc(n)).set_initial_state(psi0)
    gs, ts = wl.thetas(p, wl.rng_for(100, 0))
    ms = _time_steps(torch, stream, lambda: sim.gradient(gs, ts), steps, warmup)
    sim.set_option(qvs.QVS_OPT_PROFILE, 1)
    for _ in range(2):
        sim.gradient(gs, ts)
    roof, ker = _kernel_summary(qvs, sim.h, peak, 2)
    units = float(dim) * p
    out[f"qaoaz_parity_n{n}_A{A}_p{p}"] = {"value": units / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
                                          "launches_per_step": sim.launches(), "roofline": roof, "kernels": ker}
    sim.close()
    return out


def _extra_qaoaz(qvs, torch, stream, peak, steps, warmup, n, p):
    out = {}
    # QAOAz XY ring on the Hamming-weight-n/2 subspace of n qubits
    inst = wl.qaoaz(n, n // 2, p)
    states, rowptr, colind = qvs.qvs_xy_ring_csr(n, n // 2)
    dim = states.shape[0]
    st = torch.from_numpy(states).cuda()
    q = torch.empty(dim, dtype=torch.float32, device="cuda")
    qvs.qvs_quality_portfolio(n, st, inst.port.returns, inst.port.cov, inst.port.omega, q, qvs.QVS_F32, stream)
    sim = qvs.Simulator(dim, qvs.QVS_C64, stream)
    sim.set_quality(q).set_mixer(qvs.QVS_MIX_CSR, qvs.csr_desc(rowptr, colind, None, 2.0))
    ms = _time_steps(torch, stream, lambda: sim.gradient(inst.gammas, inst.ts), max(2, steps // 2), 2)
    sim.set_option(qvs.QVS_OPT_PROFILE, 1)
    sim.gradient(inst.gammas, inst.ts)
    roof, ker = _kernel_summary(qvs, sim.h, peak, 1)
    units = float(dim) * p
    out[f"qaoaz_csr_n{n}_k{n // 2}_p{p}"] = {"value": units / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
                                             "launches_per_step": sim.launches(), "roofline": roof, "kernels": ker,
                                             "nnz": int(colind.shape[0])}
    E_csr = sim.gradient(inst.gammas, inst.ts)[0]
    sim.close()
    # the same ring without the stored matrix: neighbour ranks generated from each row's state bits
    sim = qvs.Simulator(dim, qvs.QVS_C64, stream)
    sim.set_quality(q).set_mixer(qvs.QVS_MIX_XY_RING, qvs.xy_ring_desc(n, n // 2))
    ms = _time_steps(torch, stream, lambda: sim.gradient(inst.gammas, inst.ts), max(2, steps // 2), 2)
    sim.set_option(qvs.QVS_OPT_PROFILE, 1)
    E_xy = sim.gradient(inst.gammas, inst.ts)[0]
    roof, ker = _kernel_summary(qvs, sim.h, peak, 1)
    out[f"qaoaz_xy_ring_matrix_free_n{n}_k{n // 2}_p{p}"] = {
        "value": units / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "launches_per_step": sim.launches(),
        "roofline": roof, "kernels": ker, "rel_diff_E_vs_csr": abs(E_xy - E_csr) / abs(E_csr),
        "note": "QVS_MIX_XY_RING: the config's XY ring applied without the CSR arrays"}
    sim.close()
    return out


def _batch_roofline(torch, info, ms, peak):
    """HBM and FP32-FMA rooflines of one batched solve from the library's cost model."""
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    mhz = 2070.0
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    fma_peak = props.multi_processor_count * 128 * mhz * 1e6    # FP32 lanes x clock
    gbs = info["bytes_per_solve"] / (ms * 1e-3) / 1e9
    fmas = info["fma_per_solve"] / (ms * 1e-3)
    return {"hbm": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                    "bytes_per_solve": info["bytes_per_solve"]},
            "alu": {"bound": "alu", "achieved": fmas / 1e12, "peak": fma_peak / 1e12, "unit": "TFMA/s",
                    "frac": fmas / fma_peak, "fma_per_solve": info["fma_per_solve"],
                    "peak_note": f"{props.multi_processor_count} SMs x 128 FP32 lanes x {mhz:.0f} MHz"}}


def _extra_shared(qvs, torch, stream, peak, steps, n=20, count=1024):
    """Many parameter sets of ONE instance (weighted max-cut on G(20,1/2)), depths 2..8: one shared
    2^n quality vector against per-set copies of it."""
    inst = wl.wmaxcut(n, 8, instance=7)
    G = inst.graph
    q = torch.empty(1 << n, dtype=torch.float32, device="cuda")
    qvs.qvs_quality_maxcut(n, G.eu, G.ev, G.w, q, qvs.QVS_F32, stream)
    rng = wl.rng_for(250, count)
    ps = rng.integers(2, 9, size=count)
    th = [wl.thetas(int(p), wl.rng_for(251, k)) for k, p in enumerate(ps)]
    gl, tl = [t[0] for t in th], [t[1] for t in th]
    units = float(1 << n) * float(ps.sum())
    res = {}
    for mode in ("shared", "copies"):
        b = qvs.Batch([n] * count, ps, stream)
        if mode == "shared":
            b.set_quality_shared(q)
        else:
            b.set_quality(q.repeat(count))
        ms = _time_steps(torch, stream, lambda: b.gradient(gl, tl), max(3, steps // 2), 2)
        res[mode] = {"value": units / (ms * 1e-3), "ms_per_step": ms,
                     "roofline": _batch_roofline(torch, b.info(), ms, peak)}
        b.close()
        torch.cuda.empty_cache()
    return {f"parameter_sets_{count}_of_one_wmaxcut_n{n}": {
        "value": res["shared"]["value"], "unit": UNIT, "ms_per_step": res["shared"]["ms_per_step"],
        "roofline": res["shared"]["roofline"], "per_set_quality_copies": res["copies"],
        "note": f"{count} parameter sets, p uniform in 2..8, one persistent launch; q read by all sets"}}


def _extra_batch(qvs, torch, stream, peak, steps, warmup, count, plain=True):
    out = {}
    # batched QAOA: n in 12..20, p in 2..8, 3-regular graphs
    spec = wl.batch_spec(count=count)
    insts = [wl.maxcut3(int(n), int(p), instance=2 * 100000 + i) for i, (n, p) in enumerate(zip(spec.ns, spec.ps))]
    sizes = [1 << int(n) for n in spec.ns]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    q = torch.empty(int(offs[-1]), dtype=torch.float32, device="cuda")
    for k, inst in enumerate(insts):
        qvs.qvs_quality_maxcut(inst.graph.n, inst.graph.eu, inst.graph.ev, None, q[int(offs[k]):int(offs[k + 1])],
                               qvs.QVS_F32, stream)
    b = qvs.Batch(spec.ns, spec.ps, stream).set_quality(q)
    gl, tl = [i.gammas for i in insts], [i.ts for i in insts]
    ms = _time_steps(torch, stream, lambda: b.gradient(gl, tl), max(3, steps // 2), 2)
    units = float(sum(s * int(p) for s, p in zip(sizes, spec.ps)))
    info = b.info()
    entry = {"value": units / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
             "instances_per_s": len(insts) / (ms * 1e-3), "launches_per_step": 1, "autotune": info,
             "roofline": _batch_roofline(torch, info, ms, peak)}
    # the device optimiser: one BFGS per instance, all advanced together (gtol 1e-3, <= 30 iterations)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, _, f, it, ev, stop = b.optimise(gl, tl, gtol=1e-3, max_iter=30)
    opt_s = time.perf_counter() - t0
    E0, _, _ = b.gradient(gl, tl)
    entry["optimise"] = {
        "instances_per_s": len(insts) / opt_s, "s_per_batch": opt_s, "gtol": 1e-3, "max_iter": 30,
        "evaluations_max": int(ev.max()), "evaluations_mean": float(ev.mean()),
        "stop_counts": {str(k): int((stop == k).sum()) for k in (0, 1, 2)},
        "mean_relative_decrease": float(np.mean((E0 - f) / np.abs(E0))),
        "note": "wall time of qvs_batch_optimise: one batched objective + gradient launch and one BFGS step "
                "kernel per iteration (CUDA graph), all instances at once"}
    b.close()
    out[f"batched_qaoa_{count}"] = entry
    out.update(_extra_shared(qvs, torch, stream, peak, steps))
    if not plain:
        return out
    # the plain per-instance path over the same instances, timed once
    sims = []
    t0 = time.perf_counter()
    for k, inst in enumerate(insts):
        sim = qvs.Simulator(sizes[k], qvs.QVS_C64, stream)
        sim.set_quality(q[int(offs[k]):int(offs[k + 1])]).set_mixer(qvs.QVS_MIX_HYPERCUBE, qvs.hypercube_desc(inst.graph.n))
        sims.append(sim)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k, inst in enumerate(insts):
        sims[k].gradient(inst.gammas, inst.ts)
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - t0
    for sim in sims:
        sim.close()
    entry["plain_per_instance"] = {"value": units / plain_s, "unit": UNIT, "s_per_batch": plain_s,
                                   "note": "looped single-instance qvs_gradient calls, complex64"}
    entry["speedup_vs_plain"] = plain_s / (ms * 1e-3)
    # the plain complex128 path (fp64-accuracy state) over the same instances, one handle reused per size
    sims = {}
    for k, inst in enumerate(insts):
        n = inst.graph.n
        if n not in sims:
            sims[n] = qvs.Simulator(sizes[k], qvs.QVS_C128, stream)
            sims[n].set_mixer(qvs.QVS_MIX_HYPERCUBE, qvs.hypercube_desc(n))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k, inst in enumerate(insts):
        sim = sims[inst.graph.n]
        sim.set_quality(q[int(offs[k]):int(offs[k + 1])])
        sim.gradient(inst.gammas, inst.ts)
    torch.cuda.synchronize()
    plain128_s = time.perf_counter() - t0
    for sim in sims.values():
        sim.close()
    entry["plain_per_instance_c128"] = {"value": units / plain128_s, "unit": UNIT, "s_per_batch": plain128_s,
                                        "note": "looped single-instance qvs_gradient calls, complex128 (quality "
                                                "copied into the handle before each call)"}
    entry["speedup_vs_plain_c128"] = plain128_s / (ms * 1e-3)
    return out


# ------------------------------------------------------------------ GPU arm

def run_ours(args):
    import torch
    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    from paper_2110_03963_gb300 import _build
    if rank == 0 or world == 1:
        _build.build()
    if world > 1:
        torch.distributed.barrier()
    import paper_2110_03963_gb300 as qvs

    n, p = args.qubits, args.layers
    dim = 1 << n
    inst = wl.wmaxcut(n, p, instance=rank)
    G = inst.graph
    stream = torch.cuda.current_stream()
    sim = qvs.Simulator(dim, qvs.QVS_C64, stream)
    qubo = args.quality == "qubo"
    if qubo:
        # the max-cut cost as a quadratic form: the phase passes evaluate q themselves
        qc, qh, qJ = qvs.qvs_qubo_from_maxcut(n, G.eu, G.ev, G.w)
        sim.set_quality_qubo(n, qc, qh, qJ)
        sim_qubo_F = qubo_scale_bits(qc, qh, qJ)
    else:
        q = torch.empty(dim, dtype=torch.float32, device="cuda")
        qvs.qvs_quality_maxcut(n, G.eu, G.ev, G.w, q, qvs.QVS_F32, stream)
        sim.set_quality(q)
    sim.set_mixer(qvs.QVS_MIX_HYPERCUBE, qvs.hypercube_desc(n))
    if args.ckpt is not None:
        sim.set_option(qvs.QVS_OPT_CKPT_LAYERS, args.ckpt)
    sim.set_option(qvs.QVS_OPT_STAGED, args.staged)
    gs, ts = np.asarray(inst.gammas), np.asarray(inst.ts)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---- device-resident timing (the clock sampler starts before the warm-up, so that its
    # start-up does not fall into the timed steps)
    sampler = ClockSampler(dev)
    sampler.start()
    sampler.wait_first()
    for _ in range(args.warmup):
        sim.gradient(gs, ts)
    launches_per_step = sim.launches()
    barrier()
    sampler.mark()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    results = []
    for _ in range(args.steps):
        results.append(sim.gradient(gs, ts))
    ev1.record(stream)
    barrier()
    clocks = sampler.stop()
    def allreduce_max(x):
        t = torch.tensor([x], device="cuda", dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t.item())

    units = float(dim) * p
    ms, value = replica_aggregate(ev0.elapsed_time(ev1) / args.steps, units, world, allreduce_max)

    # ---- per-kernel event timing (separate, profiled steps)
    sim.set_option(qvs.QVS_OPT_PROFILE, 1)
    for _ in range(max(2, min(args.steps, 5))):
        sim.gradient(gs, ts)
    stats = qvs.qvs_kernel_stats(sim.h)
    sim.set_option(qvs.QVS_OPT_PROFILE, 0)
    total_ms = sum(s["ms"] for s in stats) or 1.0
    top = max(stats, key=lambda s: s["ms"])
    peak, peak_kind = _peaks()
    achieved = top["bytes"] / (top["ms"] * 1e-3) / 1e9
    kernels = {s["name"]: {"launches": s["launches"], "avg_ms": s["ms"] / s["launches"],
                           "share": s["ms"] / total_ms,
                           "GBps": s["bytes"] / (s["ms"] * 1e-3) / 1e9 if s["ms"] > 0 else None}
               for s in stats}
    step_bytes = sum(s["bytes"] for s in stats) / max(2, min(args.steps, 5))

    # ---- end to end through the C ABI with host buffers
    numa = None
    if qubo:
        def set_inputs():                     # H2D of the step's quadratic form (host arrays)
            sim.set_quality_qubo(n, qc, qh, qJ)
        h2d_quality = 8 * (1 + n + n * n)
    else:
        q_host = torch.empty(dim, dtype=torch.float32, pin_memory=True)
        q_host.copy_(q.cpu())
        numa = _host_numa(q_host.data_ptr(), 4 * dim, dev)
        del q
        torch.cuda.empty_cache()

        def set_inputs():                     # H2D of the step's quality vector (pinned host)
            sim.set_quality(q_host.numpy())
        h2d_quality = 4 * dim
    for _ in range(2):
        set_inputs()
        sim.gradient(gs, ts)
    barrier()
    t0 = time.perf_counter()
    e2e_steps = max(3, args.steps // 2)
    t_up = t_solve = 0.0
    for _ in range(e2e_steps):
        ta = time.perf_counter()
        set_inputs()
        torch.cuda.synchronize()              # separates the upload from the solve in the split below
        tb = time.perf_counter()
        E, dg, dt = sim.gradient(gs, ts)      # returns E and 2p gradient entries to the host
        t_up += tb - ta
        t_solve += time.perf_counter() - tb
    barrier()
    e2e_ms, e2e_value = replica_aggregate((time.perf_counter() - t0) / e2e_steps * 1e3, units, world, allreduce_max)

    extras = None
    if rank == 0 and world == 1 and not args.no_extras and (n, p) == (N_QUBITS, P_LAYERS):
        sim.close()
        torch.cuda.empty_cache()
        extras = run_extras(qvs, torch, stream, peak, args.steps, args.warmup,
                            headline=(results[-1][0], results[-1][1], results[-1][2]))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate_all, desc_all, _, cores = oracle_all_cores(seconds_target=15.0)
        rate1, desc1, _ = oracle_sample(seconds_target=15.0)
        cpu = {"value": rate_all, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc_all,
               "cpu_model": cpu_model(),
               "single_thread": {"value": rate1, "unit": UNIT, "cores": 1, "sample": desc1}}

    if rank == 0:
        E0 = results[-1][0]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64 (fp32 complex; fp64 phase turns, reductions)",
            "data": "synthetic",
            "config": {"workload": WORKLOAD if (n, p) == (N_QUBITS, P_LAYERS) else
                       f"QAOA weighted max-cut, n={n}, G({n},1/2) U[0,1] weights, p={p}, objective + adjoint gradient",
                       "n_qubits": n, "p": p, "amplitudes": dim,
                       "parallelism": "replicas" if world > 1 else "single",
                       "quality": ("quadratic form evaluated in the phase passes (fixed point 2^-%d)"
                                   % sim_qubo_F if qubo else "fp32 vector in HBM"),
                       "l2": "inputs larger than L2 (2 GiB state%s)" % ("" if qubo else ", 1 GiB q"),
                       "ckpt_layers": args.ckpt if args.ckpt is not None else "ceil(sqrt(p))",
                       "staged_passes": bool(args.staged)},
            "roofline": {"bound": "hbm", "kernel": top["name"], "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_kind,
                         "traffic": _traffic_per_launch(top["name"], dim) if (n, p) == (N_QUBITS, P_LAYERS)
                         else None,
                         "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum at n=25, "
                                           "scaled by amplitudes"},
            "step_roofline": {"algorithmic_bytes_per_step": step_bytes,
                              "GBps": step_bytes / (ms * 1e-3) / 1e9,
                              "frac": step_bytes / (ms * 1e-3) / 1e9 / peak},
            "kernels": kernels,
            "gpu_launches": launches_per_step * args.steps,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d_quality + 16 * p,
                    "d2h_bytes_per_step": 8 * (1 + 2 * p),
                    "upload_ms_per_step": t_up / e2e_steps * 1e3, "solve_ms_per_step": t_solve / e2e_steps * 1e3,
                    "host_numa": numa},
            "clocks": clocks,
            "objective": E0,
        }
        if cpu:
            line["cpu_baseline"] = cpu
        if extras:
            line["extras"] = extras
        print(json.dumps(line), flush=True)
    if extras is None:
        sim.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_workload(args):
    """One diagnostic line for a non-benchmark workload (QWOA, QAOAz or batched)."""
    import torch
    torch.cuda.set_device(0)
    from paper_2110_03963_gb300 import _build
    _build.build()
    import paper_2110_03963_gb300 as qvs
    stream = torch.cuda.current_stream()
    peak, _ = _peaks()
    n = args.qubits if args.qubits != N_QUBITS else {"qwoa": 26, "qaoaz": 24, "parity": 24, "batch": 0,
                                                     "c128": 28}[args.workload]
    p = args.layers if args.layers != P_LAYERS else {"qwoa": 6, "qaoaz": 4, "parity": 4, "batch": 0,
                                                     "c128": 8}[args.workload]
    res = run_extras(qvs, torch, stream, peak, args.steps, args.warmup, only=args.workload, qwoa_n=n, qwoa_p=p,
                     qaoaz_n=n, qaoaz_p=p, batch_count=args.count)
    for name, entry in res.items():
        print(json.dumps({"workload": name, **entry}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ckpt", type=int, default=None, help="checkpoint interval in layers (0 = ceil(sqrt(p)))")
    ap.add_argument("--quality", default="vector", choices=["vector", "qubo"],
                    help="vector: q generated once into HBM and read by the phase passes; qubo: the max-cut "
                         "cost as a quadratic form evaluated inside the phase passes")
    ap.add_argument("--staged", type=int, default=1, choices=[0, 1],
                    help="1: two-vector hypercube passes as TMA-staged persistent kernels; 0: one CTA per tile")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the QWOA, QAOAz and batched lines")
    ap.add_argument("--workload", default="qaoa", choices=["qaoa", "qwoa", "qaoaz", "parity", "batch", "c128"],
                    help="qaoa = the benchmark line; the others print one diagnostic line for that workload "
                         "(sizes from --qubits/--layers/--count)")
    ap.add_argument("--count", type=int, default=4096, help="instances for --workload batch")
    ap.add_argument("--qubits", type=int, default=N_QUBITS, help="state size 2^qubits (28 is the benchmark)")
    ap.add_argument("--layers", type=int, default=P_LAYERS, help="depth p (8 is the benchmark)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "qaoa":
        return run_workload(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
