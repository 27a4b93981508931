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
