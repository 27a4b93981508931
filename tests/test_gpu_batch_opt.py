"""GPU checks of the batched device optimiser (qvs_batch_optimise: one BFGS per instance, Sec. 4)
against the fp64 oracle's BFGS, and of batches of parameter sets sharing one quality vector."""
import json
import os

import numpy as np
import pytest

import oracle as orc
import workloads as wl
from tests.gpu_util import TOL_E, TOL_G, lib, rel_err_E, rel_err_grad

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def qvs():
    return lib()


def _batch_q(qvs, insts, torch):
    sizes = [1 << i.graph.n for i in insts]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    q = torch.empty(int(offs[-1]), dtype=torch.float32, device="cuda")
    for k, inst in enumerate(insts):
        qvs.qvs_quality_maxcut(inst.graph.n, inst.graph.eu, inst.graph.ev, None,
                               q[int(offs[k]):int(offs[k + 1])], qvs.QVS_F32)
    return q


def _interleave(dg, dt):
    g = np.empty(2 * len(dg))
    g[0::2], g[1::2] = dg, dt
    return g


def test_batch_optimise_follows_the_host_bfgs_on_the_same_objective():
    """The device BFGS step kernel against the host BFGS (qvs_bfgs_minimize, whose iterates equal the
    oracle's BFGS on test functions) when both see the same objective: the host loop evaluates each
    instance through a one-instance batch, the same batched kernel the device optimiser calls. The
    two runs take the same iterations and evaluations and end at the same point (fp64 rounding of
    the step arithmetic aside)."""
    import torch
    qvs = lib()
    insts = [wl.maxcut3(12 + (k % 4), 1 + (k % 3), instance=6100 + k) for k in range(8)]
    b = qvs.Batch([i.graph.n for i in insts], [i.p for i in insts]).set_quality(_batch_q(qvs, insts, torch))
    gl, tl, f, it, ev, stop = b.optimise([i.gammas for i in insts], [i.ts for i in insts], gtol=1e-4, max_iter=60)
    same = 0
    for k, inst in enumerate(insts):
        b1 = qvs.Batch([inst.graph.n], [inst.p]).set_quality(_batch_q(qvs, [inst], torch))

        def fg(th):
            E, dg, dt = b1.gradient([th[0::2]], [th[1::2]])
            return E[0], _interleave(dg[0], dt[0])
        x, fh, ith, evh, stoph = qvs.qvs_bfgs_minimize(fg, _interleave(inst.gammas, inst.ts), gtol=1e-4, max_iter=60)
        b1.close()
        if (ith, evh, stoph) == (it[k], ev[k], stop[k]) and abs(fh - f[k]) <= 1e-12 * abs(fh):
            assert np.max(np.abs(x - _interleave(gl[k], tl[k]))) < 1e-9
            same += 1
    assert same >= 7, same
    b.close()


def test_batch_optimise_vs_oracle_bfgs():
    """64 instances (n 12..15, p 1..3) optimised at once on the device, against the fp64 oracle's BFGS
    from the same start points. A non-convex BFGS run may settle in another local optimum when the
    complex64 objective moves an Armijo decision, so: every device result is a stationary point of
    the fp64 objective to the resolution of the complex64 one (max|grad| <= 1e-2: a line search that can
    no longer lower the complex64 objective stops there), where the fp64 objective equals the returned one to 1e-5
    and is no higher than at the start; at least 56 of the 64 are the oracle's own optimum (1e-5);
    and the returned parameters reproduce the returned objective exactly on the device."""
    import torch
    qvs = lib()
    path = os.path.join(GOLDEN, "oracle_batch_optimise_64.json")
    if not os.path.exists(path):
        pytest.skip("stored oracle optimisation not generated")
    ref = json.load(open(path))["instances"]
    insts = [wl.maxcut3(r["n"], r["p"], instance=r["instance"]) for r in ref]
    b = qvs.Batch([r["n"] for r in ref], [r["p"] for r in ref]).set_quality(_batch_q(qvs, insts, torch))
    gl, tl, f, it, ev, stop = b.optimise([i.gammas for i in insts], [i.ts for i in insts], gtol=1e-4, max_iter=500)
    errs = np.array([rel_err_E(f[k], r["f"]) for k, r in enumerate(ref)])
    assert np.sum(errs < 1e-5) >= 56, (np.sort(errs)[-8:], stop)
    for k, r in enumerate(ref):
        G = insts[k].graph
        prob = orc.maxcut_problem(G.n, G.eu, G.ev)
        fo, dgo, dto = orc.gradient(prob, gl[k], tl[k])
        assert rel_err_E(fo, f[k]) < 1e-5
        assert max(np.max(np.abs(dgo)), np.max(np.abs(dto))) <= 1e-2, (k, dgo, dto, stop[k])
        assert fo <= r["f0"] + 1e-9
    E, _, _ = b.gradient(gl, tl)
    assert np.array_equal(E, f)
    b.close()


def test_batch_optimise_stop_reasons_and_iteration_cap():
    """max_iter = 0 evaluates the start point only (stop 1 unless already stationary); a small cap
    stops instances with reason 1 at an improved point."""
    import torch
    qvs = lib()
    insts = [wl.maxcut3(12 + (k % 3), 1 + (k % 2), instance=6000 + k) for k in range(8)]
    b = qvs.Batch([i.graph.n for i in insts], [i.p for i in insts]).set_quality(_batch_q(qvs, insts, torch))
    g0, t0 = [i.gammas for i in insts], [i.ts for i in insts]
    E0, _, _ = b.gradient(g0, t0)
    gl, tl, f, it, ev, stop = b.optimise(g0, t0, gtol=1e-12, max_iter=0)
    assert np.all(stop == 1) and np.all(it == 0) and np.all(ev == 1)
    assert np.array_equal(f, E0)
    assert all(np.array_equal(a, c) for a, c in zip(gl, g0))
    gl, tl, f, it, ev, stop = b.optimise(g0, t0, gtol=1e-12, max_iter=2)
    assert np.all(it <= 2) and np.all((stop == 1) | (stop == 2) | (stop == 0))
    assert np.all(f <= E0)
    b.close()


def test_shared_quality_parameter_sets_vs_oracle():
    """B parameter sets of ONE instance (one 2^n quality vector read by all): each result equals the
    oracle's, and the batch equals the same batch with per-instance copies of q bit for bit."""
    import torch
    qvs = lib()
    n, B = 15, 24
    G = wl.gnp_graph(n, 0.5, wl.rng_for(240, n))
    q = torch.empty(1 << n, dtype=torch.float32, device="cuda")
    qvs.qvs_quality_maxcut(n, G.eu, G.ev, G.w, q, qvs.QVS_F32)
    ps = [1 + (k % 4) for k in range(B)]
    thetas = [wl.thetas(p, wl.rng_for(241, k)) for k, p in enumerate(ps)]
    b = qvs.Batch([n] * B, ps).set_quality_shared(q)
    E, dg, dt = b.gradient([t[0] for t in thetas], [t[1] for t in thetas])
    prob = orc.maxcut_problem(n, G.eu, G.ev, G.w, q_dtype=np.float32)
    for k in range(0, B, 5):
        f, rdg, rdt = orc.gradient(prob, thetas[k][0], thetas[k][1])
        assert rel_err_E(E[k], f) < TOL_E
        assert rel_err_grad(dg[k], dt[k], rdg, rdt) < TOL_G
    b2 = qvs.Batch([n] * B, ps).set_quality(q.repeat(B))
    E2, dg2, dt2 = b2.gradient([t[0] for t in thetas], [t[1] for t in thetas])
    assert np.array_equal(E, E2)
    assert all(np.array_equal(x, y) for x, y in zip(dg, dg2))
    # switching the same handle back to per-instance qualities
    b.set_quality(q.repeat(B))
    E3, _, _ = b.gradient([t[0] for t in thetas], [t[1] for t in thetas])
    assert np.array_equal(E3, E2)
    with pytest.raises(qvs.QvsError):
        qvs.Batch([n, n + 1], [1, 1]).set_quality_shared(q)
    b.close()
    b2.close()


def test_benchmark_depth_sweep_persistence_and_oracle():
    """qvs_benchmark (the depth sweep with persisted parameters): its outputs equal a replay of the
    same rules on the batch API (one shared-quality batch per depth, start points persisted from the
    best repeat) bit for bit; every depth's reported best is the minimum over its repeats and a
    stationary point of the fp64 objective with that value; at depth 1, where all repeats of both
    reach the global optimum, it equals the oracle's benchmark (1e-5)."""
    import torch
    qvs = lib()
    path = os.path.join(GOLDEN, "oracle_benchmark_n12_d1_3.json")
    if not os.path.exists(path):
        pytest.skip("stored oracle depth sweep not generated")
    ref = json.load(open(path))
    inst = wl.maxcut3(12, 1, instance=7000)
    G = inst.graph
    q = torch.empty(1 << 12, dtype=torch.float32, device="cuda")
    qvs.qvs_quality_maxcut(12, G.eu, G.ev, None, q, qvs.QVS_F32)
    init = np.array(ref["init"])
    repeats = 6
    f, best = qvs.qvs_benchmark(12, q, 1, 3, repeats, init, gtol=1e-4, max_iter=500)
    # replay on the batch API
    pos, prev = 0, None
    for D in range(1, 4):
        if D == 1:
            g0 = [init[2 * r:2 * r + 1] for r in range(repeats)]
            t0 = [init[2 * r + 1:2 * r + 2] for r in range(repeats)]
            pos = 2 * repeats
        else:
            g0 = [np.append(prev[0], init[pos + 2 * r]) for r in range(repeats)]
            t0 = [np.append(prev[1], init[pos + 2 * r + 1]) for r in range(repeats)]
            pos += 2 * repeats
        b = qvs.Batch([12] * repeats, [D] * repeats).set_quality_shared(q)
        gl, tl, fr, _, _, _ = b.optimise(g0, t0, gtol=1e-4, max_iter=500)
        b.close()
        assert np.array_equal(fr, f[D - 1])
        kb = int(np.argmin(fr))
        prev = (gl[kb], tl[kb])
        assert np.array_equal(best[D - 1][0], gl[kb]) and np.array_equal(best[D - 1][1], tl[kb])
    prob = orc.maxcut_problem(12, G.eu, G.ev)
    for D, (g, t) in enumerate(best, start=1):
        fo, dgo, dto = orc.gradient(prob, g, t)
        assert rel_err_E(fo, f[D - 1].min()) < 1e-5
        assert max(np.max(np.abs(dgo)), np.max(np.abs(dto))) <= 1e-2
    rf = np.array(ref["f"])
    assert np.all(np.abs(f[0] - rf[0]) <= 1e-5 * np.abs(rf[0]))
