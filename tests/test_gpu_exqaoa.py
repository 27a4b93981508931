"""GPU parity of ex-QAOA (Sec. 2.3.2) on the hypercube path through the C ABI: per-term phases in
the phase passes and per-term gradients from the stored g(x) moments, against the fp64 oracle."""
import math

import numpy as np
import pytest

import oracle as orc
import workloads as wl
from tests.gpu_util import TOL_E, TOL_G, infidelity, lib, rel_err_E

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qvs():
    return lib()


def _torch():
    import torch
    assert torch.cuda.is_available()
    return torch


def _rel_grad(dG, dt, rG, rt):
    g = np.concatenate([np.ravel(dG), dt])
    r = np.concatenate([np.ravel(rG), rt])
    return float(np.max(np.abs(g - r)) / max(np.max(np.abs(r)), 1e-30))


def _sim(qvs, n, G):
    """hypercube simulator with the weighted max-cut vector of graph G"""
    torch = _torch()
    q = torch.empty(1 << n, dtype=torch.float32, device="cuda")
    qvs.qvs_quality_maxcut(n, G.eu, G.ev, G.w, q, qvs.QVS_F32)
    sim = qvs.Simulator(1 << n, qvs.QVS_C64)
    sim.set_quality(q)
    sim.set_mixer(qvs.QVS_MIX_HYPERCUBE, qvs.hypercube_desc(n))
    return sim


def _random_terms(n, seed, n_single, n_pair):
    rng = wl.rng_for(170, seed)
    tu, tv, c = [], [], []
    for _ in range(n_single):
        tu.append(int(rng.integers(0, n))), tv.append(-1), c.append(float(rng.standard_normal()))
    for _ in range(n_pair):
        u, v = rng.choice(n, size=2, replace=False)
        tu.append(int(u)), tv.append(int(v)), c.append(float(rng.standard_normal()))
    return tu, tv, c


FRAME_TS = {"plain": [0.3, 0.6, 0.2], "flips": [1.3, 1.9, 0.4]}


@pytest.mark.parametrize("n", [13, 16, 21])
@pytest.mark.parametrize("pattern", sorted(FRAME_TS))
def test_exqaoa_random_terms_vs_oracle(qvs, n, pattern):
    G = wl.gnp_graph(n, 0.5, wl.rng_for(171, n))
    tu, tv, c = _random_terms(n, n, 4, 12)
    sim = _sim(qvs, n, G).set_phase_terms(tu, tv, c)
    p = 3
    Gm = wl.rng_for(172, n).uniform(0, math.pi, size=(p, len(c)))
    ts = np.array(FRAME_TS[pattern])
    prob = orc.maxcut_problem(n, G.eu, G.ev, G.w, q_dtype=np.float32)
    terms = orc.exqaoa_term_diags(n, tu, tv, c)
    E = sim.evolve_ex(Gm, ts)
    ref_psi = orc.exqaoa_evolve(prob, terms, Gm, ts)
    assert rel_err_E(E, orc.expectation(ref_psi, prob.q)) < TOL_E
    assert infidelity(sim.state(), ref_psi) < 1e-6
    E2, dG, dt = sim.gradient_ex(Gm, ts)
    f, rG, rt = orc.exqaoa_gradient(prob, terms, Gm, ts)
    assert rel_err_E(E2, f) < TOL_E
    assert _rel_grad(dG, dt, rG, rt) < TOL_G


def test_exqaoa_example2_edge_terms(qvs):
    """Example 2's form: one parameter per edge term 1/2 Z_u Z_v of the max-cut cost, p = 2."""
    n, p = 14, 2
    G = wl.gnp_graph(n, 0.5, wl.rng_for(173, n))
    tu, tv, c = list(G.eu), list(G.ev), [0.5 * w for w in G.w]
    sim = _sim(qvs, n, G).set_phase_terms(tu, tv, c)
    Gm = wl.rng_for(174).uniform(0, math.pi, size=(p, len(c)))
    ts = np.array([0.8, 2.2])
    prob = orc.maxcut_problem(n, G.eu, G.ev, G.w, q_dtype=np.float32)
    terms = orc.exqaoa_term_diags(n, tu, tv, c)
    E2, dG, dt = sim.gradient_ex(Gm, ts)
    f, rG, rt = orc.exqaoa_gradient(prob, terms, Gm, ts)
    assert rel_err_E(E2, f) < TOL_E
    assert _rel_grad(dG, dt, rG, rt) < TOL_G


def test_exqaoa_equal_gammas_match_qaoa_path(qvs):
    """Edge terms 1/2 Z_u Z_v with gamma_{k,e} = gamma_k: the max-cut cost minus its constant, so the
    objective and dt equal the plain QAOA path's, and each layer's term derivatives sum to its
    dgamma (n = 20, g = 3 passes)."""
    n, p = 20, 3
    G = wl.gnp_graph(n, 0.5, wl.rng_for(175, n))
    sim = _sim(qvs, n, G)
    gs, ts = wl.thetas(p, wl.rng_for(176))
    E0, dg0, dt0 = sim.gradient(gs, ts)
    sim.set_phase_terms(list(G.eu), list(G.ev), [0.5 * w for w in G.w])
    Gm = np.repeat(np.asarray(gs)[:, None], len(G.eu), axis=1)
    E1, dG, dt1 = sim.gradient_ex(Gm, ts)
    assert rel_err_E(E1, E0) < TOL_E
    assert np.max(np.abs(dt1 - dt0)) / np.max(np.abs(dt0)) < TOL_G
    assert np.max(np.abs(dG.sum(axis=1) - dg0)) / np.max(np.abs(dg0)) < TOL_G


def test_exqaoa_argument_errors(qvs):
    G = wl.gnp_graph(13, 0.5, wl.rng_for(177))
    sim = _sim(qvs, 13, G)
    with pytest.raises(qvs.QvsError):
        sim.gradient_ex(np.zeros((1, 1)), [0.1])            # no terms
    with pytest.raises(qvs.QvsError):
        sim.set_phase_terms([0], [0], [1.0])                 # Z_u Z_u
    with pytest.raises(qvs.QvsError):
        sim.set_phase_terms([13], [-1], [1.0])               # qubit out of range
    small = qvs.Simulator(1 << 10, qvs.QVS_C64)
    torch = _torch()
    q = torch.zeros(1 << 10, dtype=torch.float32, device="cuda")
    small.set_quality(q).set_mixer(qvs.QVS_MIX_HYPERCUBE, qvs.hypercube_desc(10)).set_phase_terms([0], [-1], [1.0])
    with pytest.raises(qvs.QvsError):
        small.gradient_ex(np.zeros((1, 1)), [0.1])           # n <= 12: one-CTA path has no ex-QAOA


def test_exqaoa_full24(qvs):
    """n=24 G(24,1/2) with 1/2 Z_u Z_v edge terms, p=2.

    Equal gammas per layer reproduce the plain QAOA path (objective, dt, summed term derivatives).
    Random gammas: Richardson central differences of sampled per-term derivatives and of dt
    through the same device path. The objective carries fp32 rounding of ~1e-7 relative (a few
    1e-6 absolute here), so a difference quotient over 2h = 2e-2 is noisy at ~1e-3 of the
    gradient scale; the bound is 1e-2 of it."""
    n, p = 24, 2
    G = wl.gnp_graph(n, 0.5, wl.rng_for(178, n))
    sim = _sim(qvs, n, G)
    gs, ts = np.array([0.9, 2.1]), np.array([0.45, 1.7])
    E0, dg0, dt0 = sim.gradient(gs, ts)
    sim.set_phase_terms(list(G.eu), list(G.ev), [0.5 * w for w in G.w])
    E1, dG1, dt1 = sim.gradient_ex(np.repeat(gs[:, None], len(G.eu), axis=1), ts)
    assert rel_err_E(E1, E0) < TOL_E
    assert np.max(np.abs(dt1 - dt0)) / np.max(np.abs(dt0)) < TOL_G
    assert np.max(np.abs(dG1.sum(axis=1) - dg0)) / np.max(np.abs(dg0)) < TOL_G

    Gm = wl.rng_for(179).uniform(0, math.pi, size=(p, len(G.eu)))
    E, dG, dt = sim.gradient_ex(Gm, ts)
    assert rel_err_E(sim.evolve_ex(Gm, ts), E) < TOL_E
    scale = max(np.max(np.abs(dG)), np.max(np.abs(dt)))

    def rich(fun, h=2e-2):
        d = lambda hh: (fun(hh) - fun(-hh)) / (2 * hh)
        return (4 * d(h / 2) - d(h)) / 3

    rng = wl.rng_for(180)
    for k, j in [(0, int(rng.integers(len(G.eu)))), (1, int(rng.integers(len(G.eu)))), (1, 0)]:
        def fg(hh, k=k, j=j):
            Gx = Gm.copy()
            Gx[k, j] += hh
            return sim.evolve_ex(Gx, ts)
        assert abs(rich(fg) - dG[k, j]) / scale < 1e-2
    for k in range(p):
        def ft(hh, k=k):
            tx = ts.copy()
            tx[k] += hh
            return sim.evolve_ex(Gm, tx)
        assert abs(rich(ft) - dt[k]) / scale < 1e-2
