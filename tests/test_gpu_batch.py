"""GPU parity of the batched persistent solve (one launch, many instances) against the
single-instance path and the fp64 oracle."""
import numpy as np
import pytest

import oracle as orc
import workloads as wl
from tests.gpu_util import TOL_E, TOL_G, lib, rel_err_E, rel_err_grad

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qvs():
    return lib()


def _build_batch(qvs, ns, ps, seed):
    import torch
    insts = [wl.maxcut3(int(n), int(p), instance=seed * 100000 + i) for i, (n, p) in enumerate(zip(ns, ps))]
    tot = int(sum(1 << int(n) for n in ns))
    q = torch.empty(tot, dtype=torch.float32, device="cuda")
    off = 0
    for inst in insts:
        n = inst.graph.n
        qvs.qvs_quality_maxcut(n, inst.graph.eu, inst.graph.ev, None, q[off:off + (1 << n)], qvs.QVS_F32)
        off += 1 << n
    b = qvs.Batch(ns, ps).set_quality(q)
    return b, insts, q


def test_batch_small_mixed_vs_single_and_oracle(qvs):
    ns = [12, 13, 16, 12, 20, 21, 14, 17, 12, 15]
    ps = [1, 3, 2, 5, 2, 2, 4, 1, 8, 3]
    b, insts, q = _build_batch(qvs, ns, ps, seed=1)
    E, dg, dt = b.gradient([i.gammas for i in insts], [i.ts for i in insts])
    for k, inst in enumerate(insts):
        n = inst.graph.n
        prob = orc.maxcut_problem(n, inst.graph.eu, inst.graph.ev)
        if n <= 17:
            f, rdg, rdt = orc.gradient(prob, inst.gammas, inst.ts)
            assert rel_err_E(E[k], f) < TOL_E, k
            assert rel_err_grad(dg[k], dt[k], rdg, rdt) < TOL_G, k
        sim = qvs.Simulator(1 << n, qvs.QVS_C64)
        off = int(sum(1 << int(x) for x in ns[:k]))
        sim.set_quality(q[off:off + (1 << n)]).set_mixer(qvs.QVS_MIX_HYPERCUBE, qvs.hypercube_desc(n))
        Es, dgs, dts = sim.gradient(inst.gammas, inst.ts)
        assert rel_err_E(E[k], Es) < TOL_E, k
        assert rel_err_grad(dg[k], dt[k], dgs, dts) < TOL_G, k
        sim.close()
    # graph replay with new parameters
    rng = wl.rng_for(120, 0)
    th = [wl.thetas(p, rng) for p in ps]
    E2, dg2, dt2 = b.gradient([t[0] for t in th], [t[1] for t in th])
    for k in [0, 3, 8]:
        inst = insts[k]
        prob = orc.maxcut_problem(inst.graph.n, inst.graph.eu, inst.graph.ev)
        f, rdg, rdt = orc.gradient(prob, th[k][0], th[k][1])
        assert rel_err_E(E2[k], f) < TOL_E
        assert rel_err_grad(dg2[k], dt2[k], rdg, rdt) < TOL_G
    assert b.info()["ctas_per_sm"] in (1, 2)
    b.close()


def test_batch_4096_sampled_vs_oracle(qvs):
    """The batched workload (4096 instances, n in 12..20, p in 2..8): a random subset against the
    oracle, and the whole batch against the single-instance path on a larger subset."""
    spec = wl.batch_spec()
    b, insts, q = _build_batch(qvs, spec.ns, spec.ps, seed=2)
    E, dg, dt = b.gradient([i.gammas for i in insts], [i.ts for i in insts])
    rng = wl.rng_for(121, 0)
    small = [k for k in range(len(insts)) if insts[k].graph.n <= 16]
    for k in rng.choice(small, size=24, replace=False):
        inst = insts[k]
        prob = orc.maxcut_problem(inst.graph.n, inst.graph.eu, inst.graph.ev)
        f, rdg, rdt = orc.gradient(prob, inst.gammas, inst.ts)
        assert rel_err_E(E[k], f) < TOL_E, k
        assert rel_err_grad(dg[k], dt[k], rdg, rdt) < TOL_G, k
    offs = np.concatenate([[0], np.cumsum([1 << int(n) for n in spec.ns])])
    for k in rng.choice(len(insts), size=64, replace=False):
        inst = insts[k]
        n = inst.graph.n
        sim = qvs.Simulator(1 << n, qvs.QVS_C64)
        sim.set_quality(q[int(offs[k]):int(offs[k + 1])]).set_mixer(qvs.QVS_MIX_HYPERCUBE, qvs.hypercube_desc(n))
        Es, dgs, dts = sim.gradient(inst.gammas, inst.ts)
        assert rel_err_E(E[k], Es) < TOL_E, k
        assert rel_err_grad(dg[k], dt[k], dgs, dts) < TOL_G, k
        sim.close()
    b.close()


@pytest.mark.parametrize("ctas,policy", [(1, 0), (2, 0), (1, 1), (2, 1)])
def test_batch_every_schedule_vs_oracle(qvs, ctas, policy):
    """Every schedule the autotuner can pick (1 or 2 CTAs per SM; forward states stored every
    ceil(sqrt(p)) layers with uncompute between, or at every pass boundary) gives the oracle's
    objective and gradient."""
    ns = [12, 14, 16, 13, 18, 12, 15]
    ps = [3, 5, 2, 8, 4, 1, 6]
    b, insts, _ = _build_batch(qvs, ns, ps, seed=3)
    b.set_schedule(ctas, policy)
    E, dg, dt = b.gradient([i.gammas for i in insts], [i.ts for i in insts])
    info = b.info()
    assert info["ctas_per_sm"] == ctas and info["ckpt_policy"] == policy and not info["from_cache"]
    for k, inst in enumerate(insts):
        prob = orc.maxcut_problem(inst.graph.n, inst.graph.eu, inst.graph.ev)
        f, rdg, rdt = orc.gradient(prob, inst.gammas, inst.ts)
        assert rel_err_E(E[k], f) < TOL_E, k
        assert rel_err_grad(dg[k], dt[k], rdg, rdt) < TOL_G, k
    b.close()


def test_batch_autotuner_and_schedule_cache(qvs, tmp_path, monkeypatch):
    """The first batch of a mix times the candidates and records its choice in the cache file; a
    second batch of the same (n, p) mix takes the choice from the cache without timing; a batch of
    another mix is tuned afresh."""
    import json
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("QVS_TUNE_CACHE", str(cache))
    ns, ps = [13, 16, 12, 15], [2, 3, 4, 2]
    b1, insts, _ = _build_batch(qvs, ns, ps, seed=4)
    b1.gradient([i.gammas for i in insts], [i.ts for i in insts])
    i1 = b1.info()
    assert not i1["from_cache"] and i1["ctas_per_sm"] in (1, 2) and i1["ckpt_policy"] in (0, 1)
    assert sum(t > 0 for t in i1["trial_ms_all"]) >= 2
    entries = json.loads(cache.read_text())["batch_schedules"]
    assert len(entries) == 1
    assert entries[0]["ctas_per_sm"] == i1["ctas_per_sm"] and entries[0]["ckpt_policy"] == i1["ckpt_policy"]
    # the same multiset of (n, p) in another order
    b2, insts2, _ = _build_batch(qvs, ns[::-1], ps[::-1], seed=5)
    E2, _, _ = b2.gradient([i.gammas for i in insts2], [i.ts for i in insts2])
    i2 = b2.info()
    assert i2["from_cache"] and (i2["ctas_per_sm"], i2["ckpt_policy"]) == (i1["ctas_per_sm"], i1["ckpt_policy"])
    assert i2["trial_ms_all"] == [0.0, 0.0, 0.0, 0.0]
    prob = orc.maxcut_problem(insts2[0].graph.n, insts2[0].graph.eu, insts2[0].graph.ev)
    assert rel_err_E(E2[0], orc.objective(prob, insts2[0].gammas, insts2[0].ts)) < TOL_E
    b3, insts3, _ = _build_batch(qvs, [12, 12], [1, 2], seed=6)
    b3.gradient([i.gammas for i in insts3], [i.ts for i in insts3])
    assert not b3.info()["from_cache"]
    assert len(json.loads(cache.read_text())["batch_schedules"]) == 2
    for b in (b1, b2, b3):
        b.close()
