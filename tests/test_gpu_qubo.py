"""GPU parity of quadratic (QUBO) qualities: the fixed-point generator bit for bit against the
oracle, the hypercube passes that evaluate q themselves against the same passes reading the
generated vector (identical results) and against the fp64 oracle, and the other mixers, which
materialise the vector."""
import math

import numpy as np
import pytest

import oracle as orc
import workloads as wl
from tests.gpu_util import TOL_E, TOL_E_C128, TOL_G, infidelity, lib, rel_err_E, rel_err_grad

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qvs():
    return lib()


def _torch():
    import torch
    assert torch.cuda.is_available()
    return torch


def _random_qubo(n, seed, scale=1.0):
    rng = wl.rng_for(140, seed)
    c = scale * rng.standard_normal()
    h = scale * rng.standard_normal(n)
    J = scale * rng.standard_normal((n, n))   # the lower triangle and diagonal must be ignored
    return c, h, J


def _wmaxcut_qubo(qvs, n, seed):
    G = wl.gnp_graph(n, 0.5, wl.rng_for(141, seed))
    return qvs.qvs_qubo_from_maxcut(n, G.eu, G.ev, G.w)


# ------------------------------------------------------------------ generator: bit-exact

@pytest.mark.parametrize("n,kind", [(1, "rand"), (8, "rand"), (13, "rand"), (20, "rand"), (16, "int"), (18, "wmc"),
                                    (12, "tiny"), (10, "huge")])
def test_quality_qubo_bit_exact(qvs, n, kind):
    torch = _torch()
    if kind == "int":
        G = wl.regular3_graph(n, wl.rng_for(142, n))
        c, h, J = qvs.qvs_qubo_from_maxcut(n, G.eu, G.ev)
    elif kind == "wmc":
        c, h, J = _wmaxcut_qubo(qvs, n, n)
    else:
        c, h, J = _random_qubo(n, n, {"rand": 1.0, "tiny": 1e-9, "huge": 1e7}[kind])
    ref = orc.qubo_quality_fixed(n, c, h, J)
    q32 = torch.empty(1 << n, dtype=torch.float32, device="cuda")
    q64 = torch.empty(1 << n, dtype=torch.float64, device="cuda")
    qvs.qvs_quality_qubo(n, c, h, J, q32, qvs.QVS_F32)
    qvs.qvs_quality_qubo(n, c, h, J, q64, qvs.QVS_F64)
    assert np.array_equal(q64.cpu().numpy(), ref)
    assert np.array_equal(q32.cpu().numpy(), ref.astype(np.float32))
    if kind == "int":
        assert np.array_equal(ref, orc.maxcut_quality(n, G.eu, G.ev))


def test_quality_qubo_full_size_sampled(qvs):
    """n=28 weighted G(28,1/2) max-cut form: sampled entries against the oracle's fixed-point
    definition evaluated on those basis states only."""
    torch = _torch()
    n = 28
    G = wl.wmaxcut(n, 8).graph
    c, h, J = qvs.qvs_qubo_from_maxcut(n, G.eu, G.ev, G.w)
    q = torch.empty(1 << n, dtype=torch.float32, device="cuda")
    qvs.qvs_quality_qubo(n, c, h, J, q, qvs.QVS_F32)
    idx = np.concatenate([np.arange(64), wl.rng_for(143, 0).integers(0, 1 << n, 4096), [(1 << n) - 1]])
    got = q[torch.from_numpy(idx).cuda()].cpu().numpy()
    F, ci, hi, Ji = orc.qubo_fixed_point(n, c, h, J)
    x = orc.qubit_bits(n, idx).astype(np.int64)
    qi = np.full(idx.shape[0], ci, dtype=np.int64)
    for u in range(n):
        qi += hi[u] * x[u]
        for v in range(u + 1, n):
            qi += Ji[u][v] * x[u] * x[v]
    ref = (qi.astype(np.float64) * 2.0 ** (-F)).astype(np.float32)
    assert np.array_equal(got, ref)
    # within the fixed-point rounding of the exact weighted cut values
    xb = orc.qubit_bits(n, idx)
    cut = np.zeros(idx.shape[0])
    for e in range(len(G.eu)):
        cut += np.where(xb[G.eu[e]] == xb[G.ev[e]], G.w[e], 0.0)
    assert np.max(np.abs(got - cut)) < 1e-4


# ------------------------------------------------------------------ hypercube passes: q computed in the pass

FRAME_TS = {
    "plain": [0.3, 0.5, 0.2, 0.6],
    "all_flip": [1.3, 1.9, 1.6, 1.45],
    "alternate": [0.4, 1.7, 2.9, 1.2],
}


def _sims(qvs, n, c, h, J, precision=None):
    """(simulator with the quadratic form, simulator with the generated vector)"""
    torch = _torch()
    precision = qvs.QVS_C64 if precision is None else precision
    dim = 1 << n
    a = qvs.Simulator(dim, precision)
    a.set_quality_qubo(n, c, h, J)
    a.set_mixer(qvs.QVS_MIX_HYPERCUBE, qvs.hypercube_desc(n))
    dt = torch.float32 if precision == qvs.QVS_C64 else torch.float64
    q = torch.empty(dim, dtype=dt, device="cuda")
    qvs.qvs_quality_qubo(n, c, h, J, q, qvs.QVS_F32 if precision == qvs.QVS_C64 else qvs.QVS_F64)
    b = qvs.Simulator(dim, precision)
    b.set_quality(q)
    b.set_mixer(qvs.QVS_MIX_HYPERCUBE, qvs.hypercube_desc(n))
    return a, b, q


@pytest.mark.parametrize("n", [13, 16, 20, 23])
@pytest.mark.parametrize("pattern", sorted(FRAME_TS))
def test_hypercube_qubo_in_pass_equals_vector(qvs, n, pattern):
    """Same fp32 q values, same pass arithmetic: objective, gradient and state identical to the
    passes that read the generated vector (g = 2 for n <= 20, g = 3 above; both frames)."""
    c, h, J = _wmaxcut_qubo(qvs, n, n) if n % 2 else _random_qubo(n, n)
    a, b, _ = _sims(qvs, n, c, h, J)
    ts = np.array(FRAME_TS[pattern])
    gs = np.array([0.7, 2.3, 1.1, 0.2])
    Ea, dga, dta = a.gradient(gs, ts)
    Eb, dgb, dtb = b.gradient(gs, ts)
    assert Ea == Eb
    assert np.array_equal(dga, dgb) and np.array_equal(dta, dtb)
    assert a.evolve(gs, ts) == b.evolve(gs, ts)
    assert np.array_equal(a.state(), b.state())


@pytest.mark.parametrize("n,p", [(13, 3), (17, 4), (21, 2)])
def test_hypercube_qubo_vs_oracle(qvs, n, p):
    c, h, J = _random_qubo(n, 100 + n)
    a, _, _ = _sims(qvs, n, c, h, J)
    prob = orc.Problem(q=orc.qubo_quality_fixed(n, c, h, J), mixer="hypercube", n=n)
    gs, ts = wl.thetas(p, wl.rng_for(144, n))
    E = a.evolve(gs, ts)
    ref_psi = orc.evolve(prob, gs, ts)
    assert rel_err_E(E, orc.expectation(ref_psi, prob.q)) < TOL_E
    assert infidelity(a.state(), ref_psi) < 1e-6
    E2, dg, dt = a.gradient(gs, ts)
    f, rdg, rdt = orc.gradient(prob, gs, ts)
    assert rel_err_E(E2, f) < TOL_E
    assert rel_err_grad(dg, dt, rdg, rdt) < TOL_G


def test_hypercube_qubo_c128_vs_oracle(qvs):
    n, p = 14, 3
    c, h, J = _random_qubo(n, 150)
    a, _, _ = _sims(qvs, n, c, h, J, qvs.QVS_C128)
    prob = orc.Problem(q=orc.qubo_quality_fixed(n, c, h, J), mixer="hypercube", n=n)
    gs, ts = np.array([0.4, 1.2, 2.2]), np.array([1.3, 0.2, 2.0])
    E2, dg, dt = a.gradient(gs, ts)
    f, rdg, rdt = orc.gradient(prob, gs, ts)
    assert rel_err_E(E2, f) < TOL_E_C128
    assert rel_err_grad(dg, dt, rdg, rdt) < 1e-10
    a.evolve(gs, ts)
    assert np.max(np.abs(a.state() - orc.evolve(prob, gs, ts))) < 1e-12


def test_hypercube_qubo_small_register_materialised(qvs):
    """n <= 12 runs the one-CTA kernel, which reads the materialised vector."""
    n, p = 10, 3
    c, h, J = _random_qubo(n, 151)
    a, b, _ = _sims(qvs, n, c, h, J)
    prob = orc.Problem(q=orc.qubo_quality_fixed(n, c, h, J), mixer="hypercube", n=n)
    gs, ts = wl.thetas(p, wl.rng_for(145, 0))
    E2, dg, dt = a.gradient(gs, ts)
    f, rdg, rdt = orc.gradient(prob, gs, ts)
    assert rel_err_E(E2, f) < TOL_E
    assert rel_err_grad(dg, dt, rdg, rdt) < TOL_G
    Eb, dgb, dtb = b.gradient(gs, ts)
    assert E2 == Eb and np.array_equal(dg, dgb) and np.array_equal(dt, dtb)


def test_quality_switch_back_to_vector(qvs):
    """A vector set after a quadratic form replaces it (and the other way round)."""
    torch = _torch()
    n = 14
    c, h, J = _random_qubo(n, 152)
    a, b, q = _sims(qvs, n, c, h, J)
    gs, ts = np.array([0.5, 1.0]), np.array([0.3, 1.4])
    E_form = a.evolve(gs, ts)
    q2 = torch.empty_like(q)
    qvs.qvs_quality_qubo(n, 2 * c, 2 * h, 2 * J, q2, qvs.QVS_F32)
    a.set_quality(q2)
    b.set_quality_qubo(n, 2 * c, 2 * h, 2 * J)
    assert a.evolve(gs, ts) == b.evolve(gs, ts)
    a.set_quality_qubo(n, c, h, J)
    assert a.evolve(gs, ts) == E_form


def test_set_quality_qubo_rejects_bad_arguments(qvs):
    sim = qvs.Simulator(1 << 13, qvs.QVS_C64)
    with pytest.raises(qvs.QvsError):
        sim.set_quality_qubo(12, 0.0, np.zeros(12), np.zeros((12, 12)))
    h = np.zeros(13)
    h[3] = np.nan
    with pytest.raises(qvs.QvsError):
        sim.set_quality_qubo(13, 0.0, h, np.zeros((13, 13)))


# ------------------------------------------------------------------ other mixers: materialised vector

def test_circulant_with_qubo_quality(qvs):
    n, p = 17, 2
    c, h, J = _random_qubo(n, 153)
    sim = qvs.Simulator(1 << n, qvs.QVS_C64)
    sim.set_quality_qubo(n, c, h, J)
    offsets = wl.circulant_offsets_pow2(n)
    sim.set_mixer(qvs.QVS_MIX_CIRCULANT, qvs.circulant_desc(offsets))
    lam = orc.circulant_eigenvalues(orc.circulant_first_row_from_offsets(1 << n, offsets))
    prob = orc.Problem(q=orc.qubo_quality_fixed(n, c, h, J), mixer="circulant", lam=lam)
    gs, ts = wl.thetas(p, wl.rng_for(146, 0))
    E2, dg, dt = sim.gradient(gs, ts)
    f, rdg, rdt = orc.gradient(prob, gs, ts)
    assert rel_err_E(E2, f) < TOL_E
    assert rel_err_grad(dg, dt, rdg, rdt) < TOL_G


def test_parity_mixer_with_qubo_quality(qvs):
    """The portfolio cost expanded into a quadratic form drives the parity-ring mixer."""
    torch = _torch()
    n, A, p = 12, 2, 2
    port = wl.portfolio(n // 2, wl.rng_for(147, n))
    om = port.omega
    h = np.zeros(n)
    J = np.zeros((n, n))
    for a_ in range(n // 2):
        la, sa = 2 * a_, 2 * a_ + 1
        h[la] += om * port.cov[a_][a_] - (1 - om) * port.returns[a_]
        h[sa] += om * port.cov[a_][a_] + (1 - om) * port.returns[a_]
        J[la, sa] += -2 * om * port.cov[a_][a_]
        for b_ in range(a_ + 1, n // 2):
            lb, sb = 2 * b_, 2 * b_ + 1
            k = 2 * om * port.cov[a_][b_]
            J[la, lb] += k
            J[sa, sb] += k
            J[la, sb] -= k
            J[sa, lb] -= k
    sim = qvs.Simulator(1 << n, qvs.QVS_C64)
    sim.set_quality_qubo(n, 0.0, h, J)
    sim.set_mixer(qvs.QVS_MIX_PARITY, qvs.parity_desc(n))
    psi0 = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    qvs.qvs_state_parity(n, A, psi0)
    torch.cuda.synchronize()
    sim.set_initial_state(psi0)
    qf = orc.qubo_quality_fixed(n, 0.0, h, J)
    assert np.max(np.abs(qf - orc.portfolio_quality(n, np.arange(1 << n), port.returns, port.cov, om))) < 1e-6
    prob = orc.qaoaz_parity_problem(n, A, port.returns, port.cov, om)
    prob.q = qf
    gs, ts = wl.thetas(p, wl.rng_for(148, 0))
    E2, dg, dt = sim.gradient(gs, ts)
    f, rdg, rdt = orc.gradient(prob, gs, ts)
    assert rel_err_E(E2, f) < TOL_E
    assert rel_err_grad(dg, dt, rdg, rdt) < TOL_G


# ------------------------------------------------------------------ full size

def test_full28_qubo_in_pass_equals_vector(qvs):
    """n=28 weighted G(28,1/2), p=8 (g = 3, 17 passes): the in-pass quality gives the same
    objective and gradient as the generated vector, bit for bit."""
    n = 28
    inst = wl.wmaxcut(n, 8)
    c, h, J = qvs.qvs_qubo_from_maxcut(n, inst.graph.eu, inst.graph.ev, inst.graph.w)
    a, b, q = _sims(qvs, n, c, h, J)
    Ea, dga, dta = a.gradient(inst.gammas, inst.ts)
    a.close()
    Eb, dgb, dtb = b.gradient(inst.gammas, inst.ts)
    b.close()
    assert Ea == Eb and np.array_equal(dga, dgb) and np.array_equal(dta, dtb)
