"""Write the stored fp64 oracle values that the large-size GPU parity tests compare against.

At the sizes the benchmark runs (QWOA on N = 2^24 .. 2^27, the QAOAz XY ring on C(20,10) and
C(24,12), QAOA max-cut at n = 28) the numpy oracle needs minutes to hours per solve, far longer
than a GPU test should hold a GPU. This script runs the oracle once, here on the CPU, and stores
per case: the objective f, the adjoint gradient (dgamma, dt) where the case asks for it, and a
seeded sample of final-state amplitudes. Every stored number comes from `oracle/` alone; the
inputs are the seeded instances of `workloads/` that the GPU tests rebuild bit for bit (the GPU
generates the same fp32 qualities, which the oracle promotes exactly to fp64).

    python tests/golden/make_oracle_values.py CASE [CASE ...]     (or: all)

Each case writes tests/golden/oracle_<case>.json.
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle as orc  # noqa: E402
import workloads as wl  # noqa: E402

SAMPLE = 4096          # final-state amplitudes stored per case
SAMPLE_SEED = 301      # workloads.rng_for(SAMPLE_SEED, case number) draws the sampled indices


def _qwoa(log2n: int, p: int):
    inst = wl.qwoa(log2n, p)
    prob = orc.qwoa_problem(log2n, inst.weights, inst.offsets, q_dtype=np.float32)
    desc = (f"QWOA circulant mixer (Sec. 2.4.2, Sec. 3), N=2^{log2n}, offsets 2^m (m=0..{log2n - 1}), "
            f"quality = subset sums of workloads.qwoa({log2n}, {p}).weights rounded to fp32, p={p}, "
            f"uniform initial state")
    return prob, inst.gammas, inst.ts, desc


def _csr(n: int, k: int, p: int):
    inst = wl.qaoaz(n, k, p)
    port = inst.port
    prob = orc.qaoaz_problem(n, k, port.returns, port.cov, port.omega, q_dtype=np.float32)
    desc = (f"QAOAz XY-ring mixer (Sec. 2.4.1) on the Hamming-weight-{k} subspace of {n} qubits "
            f"(C({n},{k}) = {prob.dim} states in increasing order), portfolio quality of "
            f"workloads.qaoaz({n}, {k}, {p}) rounded to fp32, p={p}, uniform initial state on the subspace")
    return prob, inst.gammas, inst.ts, desc


def _wmaxcut(n: int, p: int):
    inst = wl.wmaxcut(n, p)
    G = inst.graph
    prob = orc.maxcut_problem(n, G.eu, G.ev, G.w, q_dtype=np.float32)
    desc = (f"QAOA weighted max-cut (Sec. 6.1 cost, hypercube mixer Sec. 2.3.1), n={n}, graph "
            f"workloads.wmaxcut({n}, {p}) (G({n},1/2), U[0,1] weights), quality rounded to fp32, p={p}")
    return prob, inst.gammas, inst.ts, desc


def _maxcut10():
    inst = wl.maxcut10()
    G = inst.graph
    prob = orc.maxcut_problem(10, G.eu, G.ev)
    desc = ("QAOA max-cut (Sec. 6.1 cost, integer uncut-edge counts), n=10, random 3-regular graph "
            "workloads.maxcut10(), hypercube mixer (Sec. 2.3.1), p=2, complex128")
    return prob, inst.gammas, inst.ts, desc


# case name -> (case number, builder, with gradient)
CASES = {
    "maxcut3_n10_p2": (8, _maxcut10, True),
    "batch_optimise_64": (9, None, None),
    "benchmark_n12_d1_3": (10, None, None),
    "qwoa_n24_p3": (1, lambda: _qwoa(24, 3), True),
    "qwoa_n25_p2": (2, lambda: _qwoa(25, 2), True),
    "qwoa_n26_p6": (3, lambda: _qwoa(26, 6), True),
    "qwoa_n27_p2": (4, lambda: _qwoa(27, 2), True),
    "csr_n20_k10_p2": (5, lambda: _csr(20, 10, 2), True),
    "csr_n24_k12_p4": (6, lambda: _csr(24, 12, 4), True),
    "wmaxcut_n28_p8": (7, lambda: _wmaxcut(28, 8), False),
}


def optimise_instances(count: int = 64):
    """(n, p, instance) of the sampled optimisation instances: 3-regular max-cut (the batched
    workload's family) with n in 12..15 and p in 1..3, sizes the oracle optimises in seconds."""
    rng = wl.rng_for(SAMPLE_SEED, 100)
    ns = rng.integers(12, 16, size=count)
    ps = rng.integers(1, 4, size=count)
    return [(int(n), int(p), 5000 + i) for i, (n, p) in enumerate(zip(ns, ps))]


def run_optimise_case(name: str = "batch_optimise_64") -> str:
    """The oracle's BFGS (gtol 1e-8) from each instance's seeded start point (workloads.maxcut3)."""
    t0 = time.time()
    rows = []
    for n, p, inst_id in optimise_instances():
        inst = wl.maxcut3(n, p, instance=inst_id)
        G = inst.graph
        prob = orc.maxcut_problem(n, G.eu, G.ev)
        gs, ts, f, it, ev, stop = orc.optimise(prob, inst.gammas, inst.ts, gtol=1e-8, max_iter=500)
        rows.append({"n": n, "p": p, "instance": inst_id, "f0": orc.objective(prob, inst.gammas, inst.ts),
                     "f": float(f), "gammas": [float(x) for x in gs], "ts": [float(x) for x in ts],
                     "iterations": int(it), "evaluations": int(ev), "stop": int(stop)})
    out = {"what": "BFGS (Sec. 4) of 64 QAOA max-cut instances on random 3-regular graphs "
                   "(workloads.maxcut3(n, p, instance)), integer qualities, from the seeded start points, "
                   "gtol 1e-8, max_iter 500",
           "written_by": "tests/golden/make_oracle_values.py (calls only oracle/ on workloads/ inputs)",
           "instances": rows, "oracle_seconds": round(time.time() - t0, 1)}
    path = os.path.join(HERE, f"oracle_{name}.json")
    lines = [f"{json.dumps(k)}: {json.dumps(v, separators=(',', ':'))}" for k, v in out.items() if k != "instances"]
    body = ",\n".join(json.dumps(r, separators=(",", ":")) for r in rows)
    with open(path, "w") as fh:
        fh.write("{\n" + ",\n".join(lines) + ',\n"instances": [\n' + body + "\n]\n}\n")
    return path


def benchmark_inputs():
    """Instance and start values of the depth-sweep case: 3-regular max-cut on 12 qubits, depths
    1..3, 6 repeats; first-depth starts uniform on [0, pi], later new layers uniform on [0, pi]."""
    inst = wl.maxcut3(12, 1, instance=7000)
    rng = wl.rng_for(SAMPLE_SEED, 200)
    repeats, d_min, d_max = 6, 1, 3
    init = rng.uniform(0.0, np.pi, size=repeats * 2 * d_min + repeats * 2 * (d_max - d_min))
    return inst.graph, d_min, d_max, repeats, init


def run_benchmark_case(name: str = "benchmark_n12_d1_3") -> str:
    t0 = time.time()
    G, d_min, d_max, repeats, init = benchmark_inputs()
    prob = orc.maxcut_problem(G.n, G.eu, G.ev)
    f, best = orc.benchmark(prob, d_min, d_max, repeats, init, gtol=1e-8, max_iter=500)
    out = {"what": "depth sweep with persisted parameters (Sec. 5 benchmark, param_persist): 3-regular max-cut "
                   "workloads.maxcut3(12, 1, instance=7000).graph, integer qualities, D = 1..3, 6 repeats, "
                   "oracle BFGS gtol 1e-8, start values from workloads.rng_for(301, 200)",
           "written_by": "tests/golden/make_oracle_values.py (calls only oracle/ on workloads/ inputs)",
           "init": [float(x) for x in init], "f": [[float(x) for x in row] for row in f],
           "best": [[[float(x) for x in g], [float(x) for x in t]] for g, t in best],
           "oracle_seconds": round(time.time() - t0, 1)}
    path = os.path.join(HERE, f"oracle_{name}.json")
    lines = [f"{json.dumps(k)}: {json.dumps(v, separators=(',', ':'))}" for k, v in out.items()]
    with open(path, "w") as fh:
        fh.write("{\n" + ",\n".join(lines) + "\n}\n")
    return path


def run_case(name: str) -> str:
    if name == "batch_optimise_64":
        return run_optimise_case(name)
    if name == "benchmark_n12_d1_3":
        return run_benchmark_case(name)
    number, build, with_grad = CASES[name]
    t0 = time.time()
    prob, gammas, ts, desc = build()
    t_build = time.time() - t0
    psi = orc.evolve(prob, gammas, ts)
    f_evolve = orc.expectation(psi, prob.q)
    idx = np.sort(wl.rng_for(SAMPLE_SEED, number).choice(prob.dim, size=min(SAMPLE, prob.dim), replace=False))
    samp = psi[idx]
    norm = float(np.linalg.norm(psi))
    del psi
    out = {
        "what": desc,
        "written_by": "tests/golden/make_oracle_values.py (calls only oracle/ on workloads/ inputs)",
        "gammas": [float(x) for x in gammas],
        "ts": [float(x) for x in ts],
        "f": f_evolve,
        "norm": norm,
        "sample_seed": [SAMPLE_SEED, number],
        "sample_index": [int(i) for i in idx],
        "sample_re": [float(x) for x in samp.real],
        "sample_im": [float(x) for x in samp.imag],
    }
    if with_grad:
        f, dg, dt = orc.gradient(prob, gammas, ts)
        out["f_gradient_pass"] = float(f)
        out["dgamma"] = [float(x) for x in dg]
        out["dt"] = [float(x) for x in dt]
    out["oracle_seconds"] = {"build": round(t_build, 1), "total": round(time.time() - t0, 1)}
    path = os.path.join(HERE, f"oracle_{name}.json")
    write_json(path, out)
    return path


def write_json(path: str, out: dict):
    """One line per key; sampled amplitudes rounded to 10 significant digits (the tests compare
    complex64 results at 1e-4 of the amplitude scale), scalars kept in full."""
    out = dict(out)
    for key in ("sample_re", "sample_im"):
        out[key] = [float(f"{x:.10g}") for x in out[key]]
    lines = [f"{json.dumps(k)}: {json.dumps(v, separators=(',', ':'))}" for k, v in out.items()]
    with open(path, "w") as fh:
        fh.write("{\n" + ",\n".join(lines) + "\n}\n")


def main(argv):
    names = list(CASES) if argv == ["all"] else argv
    for nm in names:
        if nm not in CASES:
            raise SystemExit(f"unknown case {nm}; choose from {sorted(CASES)}")
    for nm in names:
        t0 = time.time()
        path = run_case(nm)
        print(f"{nm}: {time.time() - t0:.0f} s -> {path}", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
