"""The stored oracle values under tests/golden still belong to the seeded inputs and to the oracle
(CPU). The small case is recomputed in full; every other case is checked for the parameters,
sampled indices and start values that the GPU tests rebuild from workloads/ (the large cases take
the oracle minutes to hours, so their values are not recomputed here)."""
import importlib.util
import json
import math
import os

import numpy as np
import pytest

import oracle as orc
import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def writer():
    spec = importlib.util.spec_from_file_location("make_oracle_values", os.path.join(GOLDEN, "make_oracle_values.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _load(name):
    path = os.path.join(GOLDEN, f"oracle_{name}.json")
    if not os.path.exists(path):
        pytest.skip(f"stored oracle values {name} not generated")
    with open(path) as f:
        return json.load(f)


def test_small_case_recomputes(writer):
    ref = _load("maxcut3_n10_p2")
    number, build, _ = writer.CASES["maxcut3_n10_p2"]
    prob, gammas, ts, _ = build()
    assert list(gammas) == ref["gammas"] and list(ts) == ref["ts"]
    psi = orc.evolve(prob, gammas, ts)
    assert abs(orc.expectation(psi, prob.q) - ref["f"]) <= 1e-13 * abs(ref["f"])
    f, dg, dt = orc.gradient(prob, gammas, ts)
    assert np.max(np.abs(np.concatenate([dg, dt]) - np.array(ref["dgamma"] + ref["dt"]))) < 1e-12
    idx = np.array(ref["sample_index"])
    got = psi[idx]
    want = np.array(ref["sample_re"]) + 1j * np.array(ref["sample_im"])
    assert np.max(np.abs(got - want)) <= 1e-9 * np.max(np.abs(want))   # stored to 10 digits


@pytest.mark.parametrize("name", ["qwoa_n24_p3", "qwoa_n25_p2", "qwoa_n26_p6", "qwoa_n27_p2", "csr_n20_k10_p2",
                                  "wmaxcut_n28_p8"])
def test_large_case_inputs_are_the_seeded_ones(writer, name):
    ref = _load(name)
    number, _, with_grad = writer.CASES[name]
    kind, *sizes = name.split("_")
    if kind == "qwoa":
        log2n, p = int(sizes[0][1:]), int(sizes[1][1:])
        inst, dim = wl.qwoa(log2n, p), 1 << log2n
    elif kind == "csr":
        n, k, p = int(sizes[0][1:]), int(sizes[1][1:]), int(sizes[2][1:])
        inst, dim = wl.qaoaz(n, k, p), math.comb(n, k)
    else:
        n, p = int(sizes[0][1:]), int(sizes[1][1:])
        inst, dim = wl.wmaxcut(n, p), 1 << n
    assert list(inst.gammas) == ref["gammas"] and list(inst.ts) == ref["ts"]
    assert ref["sample_seed"] == [writer.SAMPLE_SEED, number]
    idx = np.sort(wl.rng_for(writer.SAMPLE_SEED, number).choice(dim, size=min(writer.SAMPLE, dim), replace=False))
    assert idx.tolist() == ref["sample_index"]
    assert abs(ref["norm"] - 1.0) < 1e-12
    assert ("dgamma" in ref) == bool(with_grad)


def test_optimise_case_instances_and_a_recomputed_sample(writer):
    ref = _load("batch_optimise_64")
    rows = ref["instances"]
    assert [(r["n"], r["p"], r["instance"]) for r in rows] == writer.optimise_instances()
    for r in rows[:3]:
        inst = wl.maxcut3(r["n"], r["p"], instance=r["instance"])
        prob = orc.maxcut_problem(r["n"], inst.graph.eu, inst.graph.ev)
        gs, ts, f, it, ev, stop = orc.optimise(prob, inst.gammas, inst.ts, gtol=1e-8, max_iter=500)
        assert (it, ev, stop) == (r["iterations"], r["evaluations"], r["stop"])
        assert abs(f - r["f"]) <= 1e-12 * max(1.0, abs(r["f"]))


def test_depth_sweep_case_start_values(writer):
    ref = _load("benchmark_n12_d1_3")
    _, d_min, d_max, repeats, init = writer.benchmark_inputs()
    assert list(init) == ref["init"]
    assert len(ref["f"]) == d_max - d_min + 1 and all(len(row) == repeats for row in ref["f"])
