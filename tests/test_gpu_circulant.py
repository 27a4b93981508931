"""GPU parity of the QWOA circulant (FFT) path, through the C ABI, against the fp64 oracle."""
import math

import numpy as np
import pytest

import oracle as orc
import workloads as wl
from tests.gpu_util import TOL_E, TOL_G, infidelity, lib, rel_err_E, rel_err_grad

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qvs():
    return lib()


def _torch():
    import torch
    assert torch.cuda.is_available()
    return torch


def _sim(qvs, log2n, weights, offsets, ow=None):
    torch = _torch()
    q = torch.empty(1 << log2n, dtype=torch.float32, device="cuda")
    qvs.qvs_quality_subset(log2n, weights, q, qvs.QVS_F32)
    sim = qvs.Simulator(1 << log2n, qvs.QVS_C64)
    sim.set_quality(q)
    sim.set_mixer(qvs.QVS_MIX_CIRCULANT, qvs.circulant_desc(offsets, ow))
    return sim, q


def _oracle(log2n, weights, offsets, ow=None):
    N = 1 << log2n
    q = orc.subset_quality(log2n, weights).astype(np.float32).astype(np.float64)
    if ow is None:
        row = orc.circulant_first_row_from_offsets(N, offsets)
    else:
        row = np.zeros(N)
        for s, w in zip(offsets, ow):
            row[int(s)] = w
            row[(N - int(s)) % N] = w
    return orc.Problem(q=q, mixer="circulant", lam=orc.circulant_eigenvalues(row))


@pytest.mark.parametrize("n", [20, 22])
def test_subset_quality_bit_exact(qvs, n):
    torch = _torch()
    w = wl.item_weights(n, wl.rng_for(70, n))
    q = torch.empty(1 << n, dtype=torch.float32, device="cuda")
    qvs.qvs_quality_subset(n, w, q, qvs.QVS_F32)
    assert np.array_equal(q.cpu().numpy(), orc.subset_quality(n, w).astype(np.float32))


# every column-transform geometry below 2^24: one, two and three-bit digits, odd and even n
@pytest.mark.parametrize("n,p", [(17, 2), (18, 1), (19, 2), (20, 1), (20, 3), (21, 2), (22, 2), (23, 1)])
def test_qwoa_pow2_offsets_vs_oracle(qvs, n, p):
    inst = wl.qwoa(n, p)
    sim, _ = _sim(qvs, n, inst.weights, inst.offsets)
    prob = _oracle(n, inst.weights, inst.offsets)
    E = sim.evolve(inst.gammas, inst.ts)
    ref_psi = orc.evolve(prob, inst.gammas, inst.ts)
    assert rel_err_E(E, orc.expectation(ref_psi, prob.q)) < TOL_E
    assert infidelity(sim.state(), ref_psi) < 1e-6
    E2, dg, dt = sim.gradient(inst.gammas, inst.ts)
    f, rdg, rdt = orc.gradient(prob, inst.gammas, inst.ts)
    assert rel_err_E(E2, f) < TOL_E
    assert rel_err_grad(dg, dt, rdg, rdt) < TOL_G


def test_qwoa_weighted_offsets_and_initial_state(qvs):
    n, p = 20, 2
    rng = wl.rng_for(71, 0)
    w = wl.item_weights(n, rng)
    offsets = np.array([1, 3, 77, 1000, 1 << 19])
    ow = rng.uniform(0.2, 1.5, size=offsets.shape[0])
    sim, _ = _sim(qvs, n, w, offsets, ow)
    psi0 = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    psi0 = (psi0 / np.linalg.norm(psi0)).astype(np.complex64)
    sim.set_initial_state(psi0)
    prob = _oracle(n, w, offsets, ow)
    prob.psi0 = psi0.astype(np.complex128)
    gs, ts = [0.7, 2.1], [0.4, 1.3]
    E, dg, dt = sim.gradient(gs, ts)
    f, rdg, rdt = orc.gradient(prob, gs, ts)
    assert rel_err_E(E, f) < TOL_E
    assert rel_err_grad(dg, dt, rdg, rdt) < TOL_G


def test_qwoa_24_objective(qvs):
    n, p = 24, 2
    inst = wl.qwoa(n, p)
    sim, _ = _sim(qvs, n, inst.weights, inst.offsets)
    prob = _oracle(n, inst.weights, inst.offsets)
    E = sim.evolve(inst.gammas, inst.ts)
    assert rel_err_E(E, orc.objective(prob, inst.gammas, inst.ts)) < TOL_E


# ------------------------------------------------------------------ full size N = 2^26, p = 6

@pytest.fixture(scope="module")
def full26(qvs):
    inst = wl.qwoa(26, 6)
    sim, q = _sim(qvs, 26, inst.weights, inst.offsets)
    return inst, sim, q


def test_full26_identities(full26):
    inst, sim, q = full26
    qh = q.cpu().numpy().astype(np.float64)
    # t = 0: mixer is the identity, E = <psi0|Q|psi0> = mean(q) whatever gamma
    E0 = sim.evolve(inst.gammas, np.zeros(6))
    assert rel_err_E(E0, qh.mean()) < TOL_E
    # gamma = 0: the uniform state is the k = 0 eigenvector of W, so E = mean(q) again
    E1 = sim.evolve(np.zeros(6), inst.ts)
    assert rel_err_E(E1, qh.mean()) < TOL_E


def test_full26_tensor_copies_bit_identical(qvs, full26):
    """At N=2^26 the column tiles move through tensor copies and the passes prefetch into L2
    (QVS_OPT_STAGED = 1, the default); per-thread loads and stores (0) run the same arithmetic, so
    the objective, the gradient and the final state agree bit for bit."""
    inst, sim, _ = full26
    gs, ts = np.asarray(inst.gammas, float), np.asarray(inst.ts, float)
    out = {}
    for staged in (1, 0):
        sim.set_option(qvs.QVS_OPT_STAGED, staged)
        E, dg, dt = sim.gradient(gs, ts)
        E2 = sim.evolve(gs, ts)
        out[staged] = (E, dg, dt, E2, sim.state())
    sim.set_option(qvs.QVS_OPT_STAGED, 1)
    (Ea, dga, dta, E2a, pa), (Eb, dgb, dtb, E2b, pb) = out[1], out[0]
    assert Ea == Eb and E2a == E2b
    assert np.array_equal(dga, dgb) and np.array_equal(dta, dtb)
    assert np.array_equal(pa, pb)


def test_full26_norm_bounds_and_gradient_consistency(full26):
    inst, sim, q = full26
    gs, ts = np.asarray(inst.gammas, float), np.asarray(inst.ts, float)
    E = sim.evolve(gs, ts)
    psi = sim.state()
    assert abs(np.sum(np.abs(psi.astype(np.complex128)) ** 2) - 1.0) < 1e-4
    assert float(q.min()) <= E <= float(q.max())
    Eg, dg, dt = sim.gradient(gs, ts)
    assert rel_err_E(Eg, E) < TOL_E
    # central differences of the complex64 objective (h = 1e-3): agreement to ~1e-3 of max|g|
    h = 1e-3
    fd = []
    for which in range(2):
        for k in range(6):
            g2, t2 = gs.copy(), ts.copy()
            (g2 if which == 0 else t2)[k] += h
            ep = sim.evolve(g2, t2)
            (g2 if which == 0 else t2)[k] -= 2 * h
            em = sim.evolve(g2, t2)
            fd.append((ep - em) / (2 * h))
    fd = np.array(fd)
    assert rel_err_grad(dg, dt, fd[:6], fd[6:]) < 2e-3


@pytest.mark.parametrize("n", [25, 27])
def test_large_sizes_norm_bounds_and_gradient_fd(qvs, n):
    """The largest geometries (three-bit and one-bit spectator rows): norm, E within the quality
    range, and the adjoint gradient against central differences of the same path."""
    p = 2
    inst = wl.qwoa(n, p)
    sim, q = _sim(qvs, n, inst.weights, inst.offsets)
    qh = q.cpu().numpy().astype(np.float64)
    gs, ts = np.asarray(inst.gammas, float), np.asarray(inst.ts, float)
    E = sim.evolve(gs, ts)
    psi = sim.state().astype(np.complex128)
    assert abs(np.sum(np.abs(psi) ** 2) - 1.0) < 1e-4
    assert qh.min() <= E <= qh.max()
    E2, dg, dt = sim.gradient(gs, ts)
    assert rel_err_E(E2, E) < TOL_E
    h = 1e-3
    fd = []
    for which in range(2):
        for k in range(p):
            g2, t2 = gs.copy(), ts.copy()
            (g2 if which == 0 else t2)[k] += h
            ep = sim.evolve(g2, t2)
            (g2 if which == 0 else t2)[k] -= 2 * h
            em = sim.evolve(g2, t2)
            fd.append((ep - em) / (2 * h))
    fd = np.array(fd)
    assert rel_err_grad(dg, dt, fd[:p], fd[p:]) < 2e-3
