"""Pins of the fp64 oracle against things other than itself (CPU only).

Each test is chosen so that a plausible mistake in the oracle (a dropped term, a wrong sign, a
wrong bit order, a transposed operand, a swapped parameter order) makes at least one fail.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg

import oracle as orc
import workloads as wl
from tests import closed_forms as cf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _dense_pauli(n, ops):
    """Dense 2^n matrix of a Pauli string {qubit: 'X'|'Y'|'Z'} (qubit u = bit n-1-u, so qubit 0 is
    the leftmost Kronecker factor)."""
    P = {"I": np.eye(2), "X": np.array([[0, 1], [1, 0]]), "Y": np.array([[0, -1j], [1j, 0]]),
         "Z": np.diag([1.0, -1.0])}
    m = np.array([[1.0 + 0j]])
    for u in range(n):
        m = np.kron(m, P[ops.get(u, "I")])
    return m


# ------------------------------------------------------------------ P1/P2: the paper's Example 1

def _ex1():
    with open(os.path.join(GOLDEN, "ex1_maxcut_cl4.json")) as f:
        return json.load(f)


def test_p1_example1_objective_matches_printed_value():
    g = _ex1()
    e = np.array(g["edges"])
    prob = orc.maxcut_problem(g["n"], e[:, 0], e[:, 1])
    th = g["theta_interleaved"]
    f = orc.objective(prob, th[0::2], th[1::2])
    assert abs(f - g["f_printed"]) <= g["f_tolerance"], f


def test_p1_example1_rejects_other_conventions():
    """Blocked parameter order or the literal X^{tensor n} mixer do not reproduce 2.30."""
    g = _ex1()
    e = np.array(g["edges"])
    prob = orc.maxcut_problem(g["n"], e[:, 0], e[:, 1])
    th = g["theta_interleaved"]
    f_blocked = orc.objective(prob, th[:2], th[2:])
    assert abs(f_blocked - g["f_printed"]) > 0.5
    # phase with the opposite sign moves f as well
    f_neg = orc.objective(prob, [-x for x in th[0::2]], th[1::2])
    assert abs(f_neg - g["f_printed"]) > 0.5


def test_p2_example1_optimal_quality_and_bit_order():
    g = _ex1()
    e = np.array(g["edges"])
    q = orc.maxcut_quality(g["n"], e[:, 0], e[:, 1])
    assert q[g["optimal_index"]] == g["optimal_quality"]
    bits = [int(b) for b in np.binary_repr(g["optimal_index"], width=g["n"])]
    assert bits == g["optimal_bits"]
    # the optimum and its complement are the only zero-quality states
    assert set(np.nonzero(q == 0)[0].tolist()) == {g["optimal_index"], (1 << g["n"]) - 1 - g["optimal_index"]}
    assert q.max() == len(g["edges"])


# ------------------------------------------------------------------ P3: p=1 closed form

@pytest.mark.parametrize("n,weighted,seed", [(8, False, 0), (10, False, 1), (9, True, 2), (11, True, 3)])
def test_p3_p1_closed_form(n, weighted, seed):
    rng = wl.rng_for(99, seed)
    if weighted:
        G = wl.gnp_graph(n, 0.5, rng, weighted=True)
    else:
        G = wl.regular3_graph(n, rng)
    prob = orc.maxcut_problem(n, G.eu, G.ev, G.w)
    for gamma, t in [(0.37, 0.81), (2.9, 1.3), (1.1, 2.7)]:
        f = orc.objective(prob, [gamma], [t])
        ref = cf.p1_maxcut_expectation(n, G.eu, G.ev, G.w, gamma, t)
        assert abs(f - ref) < 1e-12 * max(1.0, abs(ref)), (f, ref)


def test_p3_p1_amplitudes_explicit_sum():
    n = 9
    G = wl.gnp_graph(n, 0.5, wl.rng_for(98, 0), weighted=True)
    prob = orc.maxcut_problem(n, G.eu, G.ev, G.w)
    psi = orc.evolve(prob, [0.7], [0.4])
    for i in [0, 5, 77, 300, 511]:
        a = cf.p1_hypercube_amplitude(n, prob.q, 0.7, 0.4, i)
        assert abs(psi[i] - a) < 1e-13


# ------------------------------------------------------------------ P4: dense matrix exponentials

def test_p4_hypercube_vs_expm():
    n = 6
    W = sum(_dense_pauli(n, {u: "X"}) for u in range(n))
    rng = np.random.default_rng(4)
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    for t in [0.3, 1.7, -2.2]:
        ref = scipy.linalg.expm(-1j * t * W) @ psi
        assert np.max(np.abs(orc.mix_hypercube(psi, n, t) - ref)) < 1e-12
        assert np.max(np.abs(orc.apply_hypercube_W(psi, n) - W @ psi)) < 1e-12


def test_p4_circulant_vs_expm():
    N = 64
    row = orc.circulant_first_row_from_offsets(N, [1, 2, 4, 8, 16, 32])
    C = np.array([[row[(k - j) % N] for k in range(N)] for j in range(N)])
    lam = orc.circulant_eigenvalues(row)
    rng = np.random.default_rng(5)
    psi = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    for t in [0.25, 1.9]:
        ref = scipy.linalg.expm(-1j * t * C) @ psi
        assert np.max(np.abs(orc.mix_circulant(psi, lam, t) - ref)) < 1e-11
    assert np.max(np.abs(orc.apply_circulant_W(psi, lam) - C @ psi)) < 1e-11
    # a weighted symmetric first row (one weight per offset, as the library's offset weights)
    roww = np.zeros(N)
    for s_, w_ in zip([1, 3, 10, 32], [0.4, 1.7, 0.9, 2.5]):
        roww[s_] = roww[(N - s_) % N] = w_
    Cw = np.array([[roww[(k - j) % N] for k in range(N)] for j in range(N)])
    lamw = orc.circulant_eigenvalues(roww)
    assert np.max(np.abs(orc.mix_circulant(psi, lamw, 0.8) - scipy.linalg.expm(-0.8j * Cw) @ psi)) < 1e-11


@pytest.mark.parametrize("n,k", [(6, 3), (8, 4), (7, 2)])
def test_p4_xy_ring_vs_expm(n, k):
    H = np.zeros((1 << n, 1 << n), dtype=complex)
    for a in range(n):
        b = (a + 1) % n
        H += _dense_pauli(n, {a: "X", b: "X"}) + _dense_pauli(n, {a: "Y", b: "Y"})
    states = orc.subspace_states(n, k)
    Hs = H[np.ix_(states, states)]
    # the Hamming-weight subspace is invariant: nothing leaks out of it
    other = np.setdiff1d(np.arange(1 << n), states)
    assert np.max(np.abs(H[np.ix_(other, states)])) == 0
    rng = np.random.default_rng(6)
    psi = rng.standard_normal(states.shape[0]) + 1j * rng.standard_normal(states.shape[0])
    assert np.max(np.abs(orc.xy_ring_apply(psi, n, states) - Hs @ psi)) < 1e-12
    for t in [0.2, 1.3]:
        ref = scipy.linalg.expm(-1j * t * Hs) @ psi
        assert np.max(np.abs(orc.mix_xy_ring(psi, n, states, t) - ref)) < 1e-11


def test_dense_mixer_vs_independent_forms():
    """The dense symmetric mixer (eigendecomposition) against methods it shares nothing with: the
    XY-ring Taylor series on a Hamming-weight subspace, the 2x2 Givens closed form, and unitarity
    plus exact reversal on a random matrix with a nonzero diagonal."""
    n, k = 6, 3
    states = orc.subspace_states(n, k)
    dim = states.shape[0]
    W = np.zeros((dim, dim))
    for c in range(dim):
        e = np.zeros(dim)
        e[c] = 1.0
        W[:, c] = orc.xy_ring_apply(e, n, states).real
    rng = np.random.default_rng(14)
    psi = rng.standard_normal(dim) + 1j * rng.standard_normal(dim)
    for t in [0.3, 1.7]:
        assert np.max(np.abs(orc.mix_dense(psi, W, t) - orc.mix_xy_ring(psi, n, states, t))) < 1e-11
    G = np.array([[0.0, 2.0], [2.0, 0.0]])
    v = np.array([0.6, 0.8j])
    for t in [0.4, 2.2]:
        assert np.max(np.abs(orc.mix_dense(v, G, t) - cf.givens_xy(t) @ v)) < 1e-14
    A = rng.standard_normal((40, 40))
    A = A + A.T + np.diag(rng.standard_normal(40) * 3)
    x = rng.standard_normal(40) + 1j * rng.standard_normal(40)
    y = orc.mix_dense(x, A, 0.9)
    assert abs(np.linalg.norm(y) - np.linalg.norm(x)) < 1e-12
    assert np.max(np.abs(orc.mix_dense(y, A, -0.9) - x)) < 1e-12


def test_p4_full_ansatz_vs_dense_qaoa():
    """Whole p=3 ansatz against dense exponentials of W and diag(q) (n=7)."""
    n = 7
    G = wl.gnp_graph(n, 0.5, wl.rng_for(97, 0), weighted=True)
    prob = orc.maxcut_problem(n, G.eu, G.ev, G.w)
    W = sum(_dense_pauli(n, {u: "X"}) for u in range(n))
    Q = np.diag(prob.q)
    psi = np.full(1 << n, 1 / math.sqrt(1 << n), dtype=complex)
    gs, ts = [0.3, 1.2, 2.2], [0.9, 0.4, 2.8]
    for g, t in zip(gs, ts):
        psi = scipy.linalg.expm(-1j * t * W) @ (scipy.linalg.expm(-1j * g * Q) @ psi)
    assert np.max(np.abs(orc.evolve(prob, gs, ts) - psi)) < 1e-12


# ------------------------------------------------------------------ P5/P7: circulant closed forms

def test_p5_complete_graph_mixer():
    N = 256
    row = np.ones(N)
    row[0] = 0.0
    lam = orc.circulant_eigenvalues(row)
    assert lam[0] == pytest.approx(N - 1)
    assert np.max(np.abs(lam[1:] + 1.0)) < 1e-9
    rng = np.random.default_rng(7)
    psi = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    for t in [0.1, 0.77, 3.0]:
        assert np.max(np.abs(orc.mix_circulant(psi, lam, t) - cf.complete_graph_mix(psi, t))) < 1e-11


@pytest.mark.parametrize("log2n", [4, 9, 12])
def test_p7_circulant_eigenvalues(log2n):
    N = 1 << log2n
    row = orc.circulant_first_row_from_offsets(N, wl.circulant_offsets_pow2(log2n))
    lam = orc.circulant_eigenvalues(row)
    assert np.max(np.abs(lam - cf.pow2_circulant_eigs(log2n))) < 1e-10
    # library FFT of the first row gives the same spectrum
    assert np.max(np.abs(lam - np.fft.fft(row).real)) < 1e-9
    # the QWOA problem builder takes the same spectrum and the subset-sum qualities
    w = wl.item_weights(log2n, wl.rng_for(95, log2n))
    prob = orc.qwoa_problem(log2n, w, wl.circulant_offsets_pow2(log2n))
    assert np.max(np.abs(prob.lam - cf.pow2_circulant_eigs(log2n))) < 1e-10
    assert np.array_equal(prob.q, orc.subset_quality(log2n, w))
    # degree: every vertex has 2*(log2n-1) + 1 neighbours
    assert lam[0] == pytest.approx(2 * (log2n - 1) + 1)


# ------------------------------------------------------------------ P8: XY pair rotation

def test_p8_xy_pair_is_givens():
    """On n=2 the 'ring' has the pair (0,1) twice, so W = 2 (XX + YY); check exp on |01>,|10>."""
    n = 2
    states = orc.subspace_states(n, 1)       # [1, 2] = |01>, |10>
    psi = np.array([0.6, 0.8j])
    for t in [0.3, 1.1]:
        ref = cf.givens_xy(2 * t) @ psi
        assert np.max(np.abs(orc.mix_xy_ring(psi, n, states, t) - ref)) < 1e-12


# ------------------------------------------------------------------ P9: invariants

def _qaoa_small(n=8, seed=0):
    G = wl.gnp_graph(n, 0.5, wl.rng_for(96, seed), weighted=True)
    return orc.maxcut_problem(n, G.eu, G.ev, G.w)


def test_p9_norm_and_reversibility():
    for prob in [_qaoa_small(),
                 orc.qwoa_problem(8, wl.item_weights(8, wl.rng_for(95, 0)), wl.circulant_offsets_pow2(8)),
                 orc.qaoaz_problem(8, 4, *(lambda P: (P.returns, P.cov, P.omega))(wl.portfolio(4, wl.rng_for(94, 0))))]:
        gs, ts = [0.4, 2.1, 1.3], [0.7, 0.2, 2.9]
        psi = orc.evolve(prob, gs, ts)
        assert abs(np.vdot(psi, psi).real - 1.0) < 1e-13
        # un-evolve: apply the inverse layers in reverse order
        back = psi
        for g, t in zip(gs[::-1], ts[::-1]):
            back = prob.mix(back, -t)
            back = orc.phase(back, prob.q, -g)
        assert np.max(np.abs(back - prob.initial_state())) < 1e-12
        f = orc.expectation(psi, prob.q)
        assert prob.q.min() - 1e-12 <= f <= prob.q.max() + 1e-12


def test_p9_periodicities_and_symmetry():
    n = 8
    G = wl.regular3_graph(n, wl.rng_for(93, 0))
    prob = orc.maxcut_problem(n, G.eu, G.ev)       # integer q
    gs, ts = [0.4, 2.1], [0.7, 1.9]
    f = orc.objective(prob, gs, ts)
    assert orc.objective(prob, [gs[0] + 2 * math.pi, gs[1]], ts) == pytest.approx(f, abs=1e-12)
    assert orc.objective(prob, gs, [ts[0] + math.pi, ts[1]]) == pytest.approx(f, abs=1e-12)
    # real initial state and real q: E(-gamma, -t) = E(gamma, t)
    assert orc.objective(prob, [-x for x in gs], [-x for x in ts]) == pytest.approx(f, abs=1e-12)
    # relabelling the vertices does not change E
    perm = wl.rng_for(93, 1).permutation(n)
    prob2 = orc.maxcut_problem(n, perm[G.eu], perm[G.ev])
    assert orc.objective(prob2, gs, ts) == pytest.approx(f, abs=1e-12)
    # complete graph: E is periodic in t with period 2 pi / N
    N = 64
    row = np.ones(N)
    row[0] = 0
    pc = orc.Problem(q=prob.q[:N], mixer="circulant", lam=orc.circulant_eigenvalues(row))
    fc = orc.objective(pc, [0.5], [0.3])
    assert orc.objective(pc, [0.5], [0.3 + 2 * math.pi / N]) == pytest.approx(fc, abs=1e-11)


# ------------------------------------------------------------------ QAOAz parity-ring mixer (Sec. 2.4.1)

def _xy_dense(n, pairs):
    B = np.zeros((1 << n, 1 << n), dtype=complex)
    for u, v in pairs:
        B += _dense_pauli(n, {u: "X", v: "X"}) + _dense_pauli(n, {u: "Y", v: "Y"})
    return B


@pytest.mark.parametrize("n", [6, 8])
def test_parity_mixer_vs_dense_factors(n):
    """Each factor against the dense exponential of its Pauli sum, the whole U_parity against the
    product in the printed order, and the order itself (the factors do not commute)."""
    rounds = orc.parity_ring_rounds(n)
    for pairs in rounds:   # pairs of one factor are disjoint; the two rings share no qubit
        qs = [q for pr in pairs for q in pr]
        assert len(qs) == len(set(qs))
    rng = np.random.default_rng(15)
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    Bs = [_xy_dense(n, pairs) for pairs in rounds]
    for t in [0.35, 1.9]:
        U = np.eye(1 << n)
        for B, pairs in zip(Bs, rounds):
            assert np.max(np.abs(orc.xy_pairs_apply(psi, n, pairs) - B @ psi)) < 1e-12
            E = scipy.linalg.expm(-1j * t * B)
            assert np.max(np.abs(orc.xy_pairs_exp(psi, n, pairs, t) - E @ psi)) < 1e-12
            U = E @ U
        assert np.max(np.abs(orc.mix_parity(psi, n, t) - U @ psi)) < 1e-12
        Urev = np.eye(1 << n)
        for B in reversed(Bs):
            Urev = scipy.linalg.expm(-1j * t * B) @ Urev
        assert np.max(np.abs(Urev @ psi - U @ psi)) > 1e-3


def test_parity_mixer_ring_geometry_and_two_site_ring():
    """Rings of 3 close through B_last, rings of 4 through B_even (n=6, 8); a ring of 2 gets its
    one edge twice (B_odd and the closing pair of B_even), i.e. a Givens rotation by 2t twice."""
    r6 = orc.parity_ring_rounds(6)
    assert r6 == [[(0, 2), (1, 3)], [(2, 4), (3, 5)], [(4, 0), (5, 1)]]
    r8 = orc.parity_ring_rounds(8)
    assert sorted(r8[1]) == sorted([(2, 4), (6, 0), (3, 5), (7, 1)]) and r8[2] == []
    psi = np.zeros(16, dtype=complex)
    psi[0b0001] = 0.6            # qubit 3 set (ring of qubits 1, 3)
    psi[0b1000] = 0.8j           # qubit 0 set (ring of qubits 0, 2)
    for t in [0.2, 0.9]:
        out = orc.mix_parity(psi, 4, t)
        G = cf.givens_xy(2 * t)  # exp(-it(XX+YY)) applied twice = rotation by 4t on |01>,|10>
        ref = np.zeros(16, dtype=complex)
        ref[[0b0100, 0b0001]] = G @ np.array([0.0, 0.6])      # qubits (1, 3): |10> <-> |01>
        ref[[0b1000, 0b0010]] = G @ np.array([0.8j, 0.0])     # qubits (0, 2)
        assert np.max(np.abs(out - ref)) < 1e-14


def test_parity_state_and_conservation():
    """The parity state is normalised and supported on weight(odd qubits) - weight(even qubits) = A;
    the mixer conserves each ring's Hamming weight (Sec. 2.4.1: amplitude stays in the subspace)."""
    n = 8
    odd_mask = sum(1 << (n - 1 - q) for q in range(1, n, 2))
    even_mask = sum(1 << (n - 1 - q) for q in range(0, n, 2))
    idx = np.arange(1 << n)
    w_odd = np.array([bin(i & odd_mask).count("1") for i in idx])
    w_even = np.array([bin(i & even_mask).count("1") for i in idx])
    for A in [0, 1, 2, 4]:
        s = orc.parity_state(n, A)
        assert abs(np.vdot(s, s) - 1.0) < 1e-14
        assert np.all(np.abs(s[(w_odd - w_even) != A]) == 0)
        # the first A assets are |01>: qubit 2a = 0, qubit 2a+1 = 1
        for a in range(A):
            sup = idx[np.abs(s) > 0]
            assert np.all(((sup >> (n - 1 - 2 * a)) & 1) == 0) and np.all(((sup >> (n - 2 - 2 * a)) & 1) == 1)
    # the QAOAz parity problem starts from the parity state of its constraint value
    P = wl.portfolio(n // 2, wl.rng_for(94, 1))
    for A in [1, 3]:
        s0 = orc.qaoaz_parity_problem(n, A, P.returns, P.cov, P.omega).initial_state()
        assert abs(np.vdot(s0, s0) - 1.0) < 1e-14 and np.all(np.abs(s0[(w_odd - w_even) != A]) == 0)
    rng = np.random.default_rng(16)
    psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    out = orc.mix_parity(psi, n, 1.1)
    for wo in range(5):
        for we in range(5):
            sel = (w_odd == wo) & (w_even == we)
            assert abs(np.sum(np.abs(out[sel]) ** 2) - np.sum(np.abs(psi[sel]) ** 2)) < 1e-10


# ------------------------------------------------------------------ P10: gradients

@pytest.mark.parametrize("kind", ["hypercube", "circulant", "xy_ring", "dense", "parity"])
def test_p10_adjoint_vs_richardson_fd(kind):
    if kind == "hypercube":
        prob = _qaoa_small(7, 1)
    elif kind == "parity":
        P = wl.portfolio(4, wl.rng_for(94, 0))
        prob = orc.qaoaz_parity_problem(8, 2, P.returns, P.cov, P.omega)
    elif kind == "dense":
        rng = np.random.default_rng(93)
        A = rng.standard_normal((30, 30))
        A = 0.5 * (A + A.T) + np.diag(rng.standard_normal(30))
        prob = orc.Problem(q=rng.uniform(0, 3, 30), mixer="dense", W=A)
    elif kind == "circulant":
        prob = orc.qwoa_problem(7, wl.item_weights(7, wl.rng_for(92, 0)), wl.circulant_offsets_pow2(7))
    else:
        P = wl.portfolio(4, wl.rng_for(91, 0))
        prob = orc.qaoaz_problem(8, 4, P.returns, P.cov, P.omega)
    gs, ts = [0.4, 2.1, 1.3], [0.7, 0.2, 2.9]
    f, dg, dt = orc.gradient(prob, gs, ts)
    assert f == pytest.approx(orc.objective(prob, gs, ts), abs=1e-13)
    fdg, fdt = orc.central_fd(prob, gs, ts, h=1e-3)
    scale = max(np.max(np.abs(dg)), np.max(np.abs(dt)))
    assert np.max(np.abs(dg - fdg)) < 1e-8 * scale
    assert np.max(np.abs(dt - fdt)) < 1e-8 * scale


def test_p10_adjoint_vs_closed_form_derivative():
    n = 9
    G = wl.gnp_graph(n, 0.5, wl.rng_for(90, 0), weighted=True)
    prob = orc.maxcut_problem(n, G.eu, G.ev, G.w)
    f, dg, dt = orc.gradient(prob, [1.3], [0.6])
    cg, ct = cf.p1_maxcut_gradient(n, G.eu, G.ev, G.w, 1.3, 0.6)
    assert dg[0] == pytest.approx(cg, rel=1e-7, abs=1e-9)
    assert dt[0] == pytest.approx(ct, rel=1e-7, abs=1e-9)


# ------------------------------------------------------------------ qualities

def test_quality_subset_and_portfolio_small_cases():
    # subset: qubit b selects item b (qubit 0 = most significant bit)
    q = orc.subset_quality(3, [1.0, 10.0, 100.0])
    assert q.tolist() == [0, 100, 10, 110, 1, 101, 11, 111]
    # portfolio: one asset: |10> long (z=+1), |01> short (z=-1)
    states = np.array([0, 1, 2, 3])
    q = orc.portfolio_quality(2, states, [2.0], [[3.0]], 0.25)
    # z = [0, -1, +1, 0]: omega*3*z^2 - 0.75*2*z
    assert np.allclose(q, [0.0, 0.75 + 1.5, 0.75 - 1.5, 0.0])


def test_portfolio_two_assets_hand_computed():
    """Two assets, every position pair written out by hand (cross-covariance terms included)."""
    cov = [[2.0, 0.5], [0.5, 3.0]]
    r = [1.0, -2.0]
    om = 0.25
    # qubits (0 long, 1 short) for asset 0 and (2 long, 3 short) for asset 1, qubit 0 = MSB
    cases = {(1, 0, 1, 0): (1, 1), (1, 0, 0, 1): (1, -1), (0, 1, 0, 0): (-1, 0), (1, 1, 0, 1): (0, -1)}
    for bits, (z0, z1) in cases.items():
        idx = int("".join(map(str, bits)), 2)
        q = orc.portfolio_quality(4, np.array([idx]), r, cov, om)[0]
        expect = om * (2.0 * z0 * z0 + 0.5 * z0 * z1 + 0.5 * z1 * z0 + 3.0 * z1 * z1) - (1 - om) * (1.0 * z0 - 2.0 * z1)
        assert q == pytest.approx(expect, abs=1e-15)


def test_subspace_count():
    assert orc.subspace_states(10, 5).shape[0] == math.comb(10, 5)
    assert orc.subspace_states(24, 12).shape[0] == 2704156
    # the QAOAz problem lives on the weight-k states
    P = wl.portfolio(4, wl.rng_for(91, 0))
    st = orc.qaoaz_problem(8, 3, P.returns, P.cov, P.omega).states
    assert st.shape[0] == math.comb(8, 3) and all(bin(int(x)).count("1") == 3 for x in st)


# ------------------------------------------------------------------ quadratic (QUBO) qualities

def _maxcut_as_qubo(n, eu, ev, w):
    """[x_u == x_v] = 1 - x_u - x_v + 2 x_u x_v: the textbook identity, written in the test."""
    c, h, J = 0.0, np.zeros(n), np.zeros((n, n))
    for e in range(len(eu)):
        u, v = sorted((int(eu[e]), int(ev[e])))
        we = 1.0 if w is None else float(w[e])
        c += we
        h[u] -= we
        h[v] -= we
        J[u, v] += 2 * we
    return c, h, J


def test_qubo_reduces_to_maxcut_subset_and_portfolio():
    """Special cases with independent definitions: max-cut (edge sums, pinned by Example 1 above),
    subset sums (J = 0) and the portfolio cost (z_a = x_2a - x_2a+1 expanded by hand)."""
    G = wl.regular3_graph(10, wl.rng_for(120))
    c, h, J = _maxcut_as_qubo(10, G.eu, G.ev, None)
    assert np.array_equal(orc.qubo_quality(10, c, h, J), orc.maxcut_quality(10, G.eu, G.ev))
    Gw = wl.gnp_graph(9, 0.5, wl.rng_for(121))
    c, h, J = _maxcut_as_qubo(9, Gw.eu, Gw.ev, Gw.w)
    assert np.max(np.abs(orc.qubo_quality(9, c, h, J) - orc.maxcut_quality(9, Gw.eu, Gw.ev, Gw.w))) < 1e-12
    w = [0.5, -1.25, 3.0, 7.5, 0.125]
    assert np.array_equal(orc.qubo_quality(5, 0.0, w, np.zeros((5, 5))), orc.subset_quality(5, w))
    # portfolio, 3 assets: z_a^2 = x_l + x_s - 2 x_l x_s, z_a z_b = x_la x_lb - x_la x_sb - x_sa x_lb + x_sa x_sb
    port = wl.portfolio(3, wl.rng_for(122))
    om, M = port.omega, 3
    h = np.zeros(6)
    J = np.zeros((6, 6))
    for a in range(M):
        la, sa = 2 * a, 2 * a + 1
        h[la] += om * port.cov[a][a] - (1 - om) * port.returns[a]
        h[sa] += om * port.cov[a][a] + (1 - om) * port.returns[a]
        J[la, sa] += -2 * om * port.cov[a][a]
        for b in range(a + 1, M):
            lb, sb = 2 * b, 2 * b + 1
            k = 2 * om * port.cov[a][b]
            J[la, lb] += k
            J[sa, sb] += k
            J[la, sb] -= k
            J[sa, lb] -= k
    states = np.arange(64)
    ref = orc.portfolio_quality(6, states, port.returns, port.cov, om)
    assert np.max(np.abs(orc.qubo_quality(6, 0.0, h, J) - ref)) < 1e-12


def test_qubo_reads_upper_triangle_and_bit_order():
    """One coefficient at a time: h_u marks qubit u (= index bit n-1-u); J below the diagonal and
    on it is ignored."""
    n = 4
    for u in range(n):
        h = np.zeros(n)
        h[u] = 1.0
        q = orc.qubo_quality(n, 0.0, h, np.zeros((n, n)))
        assert q.tolist() == [float((i >> (n - 1 - u)) & 1) for i in range(16)]
    J = np.zeros((n, n))
    J[1, 3] = 2.0
    J[3, 1] = 100.0
    J[2, 2] = 100.0
    q = orc.qubo_quality(n, 0.5, np.zeros(n), J)
    assert q.tolist() == [0.5 + (2.0 if ((i >> 2) & 1) and (i & 1) else 0.0) for i in range(16)]


def test_qubo_fixed_point_rule():
    """The fixed-point contract: F maximal with S 2^F + 1024 <= 2^30, exact for dyadic
    coefficients, within half a grid step per coefficient otherwise, and every subset sum of the
    rounded coefficients below 2^30 in magnitude."""
    rng = np.random.default_rng(123)
    for n, scale in ((6, 1.0), (8, 1e-3), (10, 1e4)):
        c = scale * rng.standard_normal()
        h = scale * rng.standard_normal(n)
        J = np.triu(scale * rng.standard_normal((n, n)), 1)
        F, ci, hi, Ji = orc.qubo_fixed_point(n, c, h, J)
        S = abs(c) + np.sum(np.abs(h)) + np.sum(np.abs(J))
        assert S * 2.0 ** F + 1024 <= 2.0 ** 30 < S * 2.0 ** (F + 1) + 1024
        mag = abs(ci) + sum(abs(x) for x in hi) + sum(abs(x) for row in Ji for x in row)
        assert mag < 2 ** 30
        ncoef = 1 + n + n * (n - 1) // 2
        err = np.max(np.abs(orc.qubo_quality_fixed(n, c, h, J) - orc.qubo_quality(n, c, h, J)))
        assert err <= ncoef * 2.0 ** (-F - 1) * (1 + 1e-9)
        assert err > 0   # random coefficients are not on the grid
    # integer and dyadic coefficients are on the grid: exact
    G = wl.regular3_graph(12, wl.rng_for(124))
    c, h, J = _maxcut_as_qubo(12, G.eu, G.ev, None)
    assert np.array_equal(orc.qubo_quality_fixed(12, c, h, J), orc.maxcut_quality(12, G.eu, G.ev))
    F, ci, _, _ = orc.qubo_fixed_point(3, 0.75, [0.5, -0.25, 0.0], np.zeros((3, 3)))
    assert ci * 2.0 ** (-F) == 0.75
    # halves round away from zero
    F, ci, hi, _ = orc.qubo_fixed_point(2, 0.0, [1.0, -1.0], np.zeros((2, 2)))
    F2, ci2, hi2, _ = orc.qubo_fixed_point(2, 0.0, [1.0 + 2.0 ** (-F - 1), -1.0 - 2.0 ** (-F - 1)], np.zeros((2, 2)))
    assert F2 == F and hi2 == [hi[0] + 1, hi[1] - 1]


# ------------------------------------------------------------------ ex-QAOA (Sec. 2.3.2)

def _qubo_to_pauli(n, c, h, J):
    """x_u = (1 - z_u)/2 written out: q = const + sum_u a_u Z_u + sum_{u<v} b_uv Z_u Z_v."""
    const = c + 0.5 * sum(h) + 0.25 * sum(J[u][v] for u in range(n) for v in range(u + 1, n))
    tu, tv, coef = [], [], []
    for u in range(n):
        a = -0.5 * h[u] - 0.25 * sum(J[min(u, v)][max(u, v)] for v in range(n) if v != u)
        tu.append(u), tv.append(-1), coef.append(a)
    for u in range(n):
        for v in range(u + 1, n):
            if J[u][v] != 0:
                tu.append(u), tv.append(v), coef.append(0.25 * J[u][v])
    return const, tu, tv, coef


def test_pauli_z_diag_bit_order():
    # qubit 0 is the most significant bit; Z = +1 on |0>
    assert orc.pauli_z_diag(3, 0).tolist() == [1, 1, 1, 1, -1, -1, -1, -1]
    assert orc.pauli_z_diag(3, 2).tolist() == [1, -1, 1, -1, 1, -1, 1, -1]
    assert orc.pauli_z_diag(3, 0, 2).tolist() == [1, -1, 1, -1, -1, 1, -1, 1]


def test_exqaoa_equal_gammas_is_qaoa():
    """With gamma_{k,j} = gamma_k for every term of Q's Pauli decomposition, U_Qext differs from
    exp(-i gamma_k Q) by the global phase of the identity part: same state up to a phase, same
    objective, and the per-term gradients of a layer sum to the QAOA gamma gradient."""
    n, p = 7, 3
    rng = wl.rng_for(160)
    c, h, J = rng.standard_normal(), rng.standard_normal(n), np.triu(rng.standard_normal((n, n)), 1)
    const, tu, tv, coef = _qubo_to_pauli(n, c, h, J)
    terms = orc.exqaoa_term_diags(n, tu, tv, coef)
    q = orc.qubo_quality(n, c, h, J)
    assert np.max(np.abs(const + sum(terms) - q)) < 1e-12     # the decomposition itself
    prob = orc.Problem(q=q, mixer="hypercube", n=n)
    gs, ts = wl.thetas(p, wl.rng_for(161))
    G = np.repeat(np.asarray(gs)[:, None], len(terms), axis=1)
    a = orc.exqaoa_evolve(prob, terms, G, ts)
    b = orc.evolve(prob, gs, ts)
    assert abs(abs(np.vdot(a, b)) - 1.0) < 1e-12
    f, dG, dt = orc.exqaoa_gradient(prob, terms, G, ts)
    f0, dg0, dt0 = orc.gradient(prob, gs, ts)
    assert abs(f - f0) < 1e-12
    assert np.max(np.abs(dG.sum(axis=1) - dg0)) < 1e-10
    assert np.max(np.abs(dt - dt0)) < 1e-10


def test_exqaoa_vs_dense_expm():
    """n=4, p=2, distinct gamma per term: the ansatz as dense matrix exponentials of the summed
    diagonal and of W = sum_j X_j."""
    n, p = 4, 2
    tu, tv, coef = [0, 1, 0, 2, 1], [1, 3, -1, 3, -1], [0.5, -1.25, 0.75, 2.0, 0.3]
    terms = orc.exqaoa_term_diags(n, tu, tv, coef)
    G = wl.rng_for(162).uniform(0, math.pi, size=(p, len(tu)))
    ts = [0.4, 1.9]
    W = sum(_dense_pauli(n, {u: "X"}) for u in range(n))
    psi = np.full(1 << n, 0.25, dtype=np.complex128)
    for k in range(p):
        D = np.diag(sum(G[k][j] * terms[j] for j in range(len(tu))))
        psi = scipy.linalg.expm(-1j * ts[k] * W) @ (scipy.linalg.expm(-1j * D) @ psi)
    prob = orc.Problem(q=np.arange(16.0), mixer="hypercube", n=n)
    assert np.max(np.abs(orc.exqaoa_evolve(prob, terms, G, ts) - psi)) < 1e-12


def test_exqaoa_gradient_vs_richardson_fd():
    n, p = 6, 2
    G6 = wl.gnp_graph(n, 0.6, wl.rng_for(163))
    tu, tv, coef = list(G6.eu), list(G6.ev), [0.5 * w for w in G6.w]     # Example 2: 1/2 Z_u Z_v per edge
    terms = orc.exqaoa_term_diags(n, tu, tv, coef)
    prob = orc.maxcut_problem(n, G6.eu, G6.ev, G6.w)
    G = wl.rng_for(164).uniform(0, math.pi, size=(p, len(tu)))
    ts = np.array([0.7, 2.1])
    f, dG, dt = orc.exqaoa_gradient(prob, terms, G, ts)

    def obj(Gx, tx):
        return orc.expectation(orc.exqaoa_evolve(prob, terms, Gx, tx), prob.q)

    def rich(fun, h=1e-3):
        d = lambda hh: (fun(hh) - fun(-hh)) / (2 * hh)
        return (4 * d(h / 2) - d(h)) / 3

    for k in range(p):
        for j in range(len(tu)):
            def fg(hh, k=k, j=j):
                Gx = G.copy()
                Gx[k, j] += hh
                return obj(Gx, ts)
            assert abs(rich(fg) - dG[k, j]) < 1e-8
        def ft(hh, k=k):
            tx = ts.copy()
            tx[k] += hh
            return obj(G, tx)
        assert abs(rich(ft) - dt[k]) < 1e-8


# ------------------------------------------------------------------ classical optimiser (Sec. 4: BFGS)

def test_bfgs_quadratic_and_rosenbrock():
    """A positive-definite quadratic reaches its closed-form minimiser A^-1 b; the Rosenbrock
    function from (-1.2, 1) reaches (1, 1).

    Bound on the quadratic: the loop stops with max|g| <= gtol, g = A (x - x*), and A = M M^T + 6 I
    has lambda_min(A) >= 6, so max|x - x*| <= ||x - x*||_2 <= ||g||_2 / 6 <= sqrt(6) gtol / 6 =
    gtol / sqrt(6). gtol = 1e-8 is about the smallest the Armijo test can resolve here: a step
    near x* lowers f by about g^T A^-1 g / 2 ~ 1e-17 when max|g| ~ 1e-8, which is the fp64
    spacing of |f| ~ 0.1; below that no step decreases f and the search ends with stop = 2."""
    rng = wl.rng_for(200)
    M = rng.standard_normal((6, 6))
    A = M @ M.T + 6 * np.eye(6)
    b = rng.standard_normal(6)
    gtol = 1e-8
    x, f, it, ev, stop = orc.bfgs_minimize(lambda x: (0.5 * x @ A @ x - b @ x, A @ x - b), np.zeros(6), gtol=gtol)
    assert stop == 0 and it < 200   # converged, not stopped by the iteration cap or the line search
    assert np.max(np.abs(x - np.linalg.solve(A, b))) <= gtol / math.sqrt(6.0) * (1 + 1e-6)
    assert abs(f + 0.5 * b @ np.linalg.solve(A, b)) < 1e-12

    def rosen(z):
        a, c = z
        return (1 - a) ** 2 + 100 * (c - a * a) ** 2, np.array([-2 * (1 - a) - 400 * a * (c - a * a), 200 * (c - a * a)])
    x, f, it, ev, stop = orc.bfgs_minimize(rosen, np.array([-1.2, 1.0]), gtol=1e-10)
    assert np.max(np.abs(x - 1.0)) < 1e-8 and f < 1e-16


def test_bfgs_stops_on_precision_loss_at_the_best_point():
    """When no line-search step can lower f (here f is rounded to multiples of 1e-6 while its
    gradient stays exact), the search ends with stop = 2 at the last accepted point: it never moves
    to a worse point, and the returned f is the objective there."""
    D = np.array([1.0, 3.7])

    def fq(z):
        v = float(np.sum(D * (z - 1.0) ** 2))
        return math.floor(v * 1e6) / 1e6, 2.0 * D * (z - 1.0)
    x0 = np.array([3.0, -2.0])
    x, f, it, ev, stop = orc.bfgs_minimize(fq, x0, gtol=1e-12, max_iter=500)
    assert stop == 2
    assert f == fq(x)[0] and f <= fq(x0)[0]
    assert np.max(np.abs(x - 1.0)) < 2e-3            # inside the flat band around the minimiser
    assert ev <= it + 1 + (it + 1) * 31               # at most 31 trial points per iteration

    # The same bowl plus a deterministic noise of up to 1e-6 that differs at every point (a hash
    # of the point's bytes); the gradient stays that of the bowl. Every trial point the line search
    # rejects near the end is then strictly worse than the point it started from, so the point
    # returned must be the best one evaluated.
    seen = []

    def fn(z):
        h = 0
        for w in np.ascontiguousarray(z, dtype=np.float64).view(np.uint64).tolist():
            h = ((h ^ w) * 0x9E3779B97F4A7C15 + 0x632BE59BD9B4E019) % (1 << 64)
            h ^= h >> 29
        v = float(np.sum(D * (z - 1.0) ** 2)) + 1e-6 * (h % (1 << 53)) / float(1 << 53)
        seen.append(v)
        return v, 2.0 * D * (z - 1.0)
    x, f, it, ev, stop = orc.bfgs_minimize(fn, x0, gtol=1e-12, max_iter=500)
    assert stop == 2 and len(seen) == ev
    assert f == min(seen) and f == fn(x)[0]


def test_optimise_qaoa_matches_scipy_bfgs_and_closed_form():
    """p=1 QAOA on a 3-regular 8-vertex graph: from the same start the written-out BFGS and SciPy's
    BFGS (a library routine) reach the same optimum, which also equals the best value of the p=1
    closed form on a fine (gamma, t) grid refined by the same optimiser."""
    scipy_optimize = pytest.importorskip("scipy.optimize")
    n = 8
    G = wl.regular3_graph(n, wl.rng_for(201))
    prob = orc.maxcut_problem(n, G.eu, G.ev)
    g0, t0 = np.array([0.6]), np.array([0.4])
    gs, ts, f, it, ev, _ = orc.optimise(prob, g0, t0, gtol=1e-10)

    def fg(th):
        E, dg, dt = orc.gradient(prob, th[0::2], th[1::2])
        return E, np.array([dg[0], dt[0]])
    res = scipy_optimize.minimize(fg, np.array([0.6, 0.4]), jac=True, method="BFGS", options={"gtol": 1e-10})
    # same optimal value; the points themselves may differ by the ansatz's symmetries
    # (t -> t + pi, the gamma period of integer qualities), so they are not compared
    assert abs(f - res.fun) < 1e-9
    # the optimum is a stationary point of the p=1 closed form, with the same value there
    assert abs(cf.p1_maxcut_expectation(n, G.eu, G.ev, None, gs[0], ts[0]) - f) < 1e-10
    assert np.max(np.abs(cf.p1_maxcut_gradient(n, G.eu, G.ev, None, gs[0], ts[0]))) < 1e-5
    # started from the best point of a (gamma, t) grid of the closed form, it ends at or below it
    grid = np.linspace(0.0, math.pi, 41)
    best = min((cf.p1_maxcut_expectation(n, G.eu, G.ev, None, gg, tt), gg, tt) for gg in grid for tt in grid)
    gs2, ts2, f2, _, _, _ = orc.optimise(prob, np.array([best[1]]), np.array([best[2]]), gtol=1e-10)
    assert f2 <= best[0] + 1e-12
    assert abs(cf.p1_maxcut_expectation(n, G.eu, G.ev, None, gs2[0], ts2[0]) - f2) < 1e-10


def test_benchmark_depth_sweep_with_persisted_parameters():
    """Sec. 5 benchmark with param_persist: one depth and one repeat is exactly `optimise`; and when
    every new layer starts at gamma = t = 0 (an identity layer), each repeat at depth D + 1 starts
    at the best optimum of depth D, so the best objective never increases with depth."""
    n = 8
    G = wl.regular3_graph(n, wl.rng_for(203))
    prob = orc.maxcut_problem(n, G.eu, G.ev)
    g0, t0 = np.array([0.7]), np.array([0.3])
    f, best = orc.benchmark(prob, 1, 1, 1, np.concatenate([g0, t0]), gtol=1e-9)
    gs, ts, fo, _, _, _ = orc.optimise(prob, g0, t0, gtol=1e-9)
    assert f.shape == (1, 1) and f[0, 0] == fo and np.array_equal(best[0][0], gs)
    rng = wl.rng_for(204)
    repeats = 3
    init = np.concatenate([rng.uniform(0, np.pi, size=2 * repeats), np.zeros(2 * repeats * 2)])
    f, best = orc.benchmark(prob, 1, 3, repeats, init, gtol=1e-9)
    assert f.shape == (3, repeats)
    for D in range(1, 3):
        assert f[D].min() <= f[D - 1].min() + 1e-12
        # the persisted start reproduces the previous depth's best objective exactly
        g_start = np.append(best[D - 1][0], 0.0)
        t_start = np.append(best[D - 1][1], 0.0)
        assert abs(orc.objective(prob, g_start, t_start) - f[D - 1].min()) < 1e-12
    for D, (g, t) in enumerate(best, start=1):
        assert len(g) == len(t) == D
        assert abs(orc.objective(prob, g, t) - f[D - 1].min()) < 1e-12
    # With no optimiser iterations every repeat ends at its start, which shows where each start
    # value is read: at depth 1, repeat r takes init[2r] (gamma) and init[2r + 1] (t); at every
    # later depth, the best start of the previous depth plus the next pair (gamma, t) of init.
    init = rng.uniform(0.1, np.pi, size=2 * repeats + 2 * repeats * 2)
    f, best = orc.benchmark(prob, 1, 3, repeats, init, max_iter=0)
    prev = None
    for D in range(1, 4):
        starts = []
        for r in range(repeats):
            if D == 1:
                starts.append((init[2 * r: 2 * r + 1], init[2 * r + 1: 2 * r + 2]))
            else:
                base = 2 * repeats + 2 * repeats * (D - 2) + 2 * r
                starts.append((np.append(prev[0], init[base]), np.append(prev[1], init[base + 1])))
        fD = [orc.objective(prob, g, t) for g, t in starts]
        assert np.array_equal(f[D - 1], fD)
        prev = starts[int(np.argmin(fD))]
        assert np.array_equal(best[D - 1][0], prev[0]) and np.array_equal(best[D - 1][1], prev[1])
