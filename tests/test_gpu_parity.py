"""GPU parity of the QAOAz parity-ring mixer path (Sec. 2.4.1), through the C ABI, against the fp64
oracle."""
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


def _setup(qvs, n, A, port, init="parity"):
    torch = _torch()
    dim = 1 << n
    states = torch.arange(dim, dtype=torch.int64, device="cuda")
    q = torch.empty(dim, dtype=torch.float32, device="cuda")
    qvs.qvs_quality_portfolio(n, states, port.returns, port.cov, port.omega, q, qvs.QVS_F32)
    sim = qvs.Simulator(dim, qvs.QVS_C64)
    sim.set_quality(q)
    sim.set_mixer(qvs.QVS_MIX_PARITY, qvs.parity_desc(n))
    if init == "parity":
        psi0 = torch.empty(dim, dtype=torch.complex64, device="cuda")
        qvs.qvs_state_parity(n, A, psi0)
        torch.cuda.synchronize()
        sim.set_initial_state(psi0)
    return sim, q


def _oracle(n, A, port, init="parity"):
    prob = orc.qaoaz_parity_problem(n, A, port.returns, port.cov, port.omega, q_dtype=np.float32)
    if init != "parity":
        prob.psi0 = None
    return prob


@pytest.mark.parametrize("n,A", [(12, 0), (12, 2), (14, 3), (16, 8)])
def test_parity_state_vs_oracle(qvs, n, A):
    torch = _torch()
    out = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    qvs.qvs_state_parity(n, A, out)
    ref = orc.parity_state(n, A)
    got = out.cpu().numpy()
    assert np.max(np.abs(got - ref)) < 1e-7
    assert np.array_equal(np.abs(got) > 0, np.abs(ref) > 0)


# n = 14, 18: rings of 7 and 9 qubits (closed by B_last); n = 12, 16: rings of 6 and 8 (closed in B_even)
@pytest.mark.parametrize("n,A,p", [(12, 2, 1), (14, 2, 3), (16, 3, 2), (18, 2, 2)])
def test_parity_mixer_vs_oracle(qvs, n, A, p):
    port = wl.portfolio(n // 2, wl.rng_for(95, n))
    sim, _ = _setup(qvs, n, A, port)
    prob = _oracle(n, A, port)
    gs, ts = wl.thetas(p, wl.rng_for(96, n * 10 + p))
    E = sim.evolve(gs, ts)
    ref_psi = orc.evolve(prob, gs, ts)
    assert rel_err_E(E, orc.expectation(ref_psi, prob.q)) < TOL_E
    assert infidelity(sim.state(), ref_psi) < 1e-6
    assert np.max(np.abs(sim.state() - ref_psi)) < 1e-5
    E2, dg, dt = sim.gradient(gs, ts)
    f, rdg, rdt = orc.gradient(prob, gs, ts)
    assert rel_err_E(E2, f) < TOL_E
    assert rel_err_grad(dg, dt, rdg, rdt) < TOL_G


def test_parity_mixer_uniform_start_vs_oracle(qvs):
    n, p = 14, 3
    port = wl.portfolio(n // 2, wl.rng_for(97, n))
    sim, _ = _setup(qvs, n, 0, port, init="uniform")
    prob = _oracle(n, 0, port, init="uniform")
    gs, ts = wl.thetas(p, wl.rng_for(98, 0))
    E2, dg, dt = sim.gradient(gs, ts)
    f, rdg, rdt = orc.gradient(prob, gs, ts)
    assert rel_err_E(E2, f) < TOL_E
    assert rel_err_grad(dg, dt, rdg, rdt) < TOL_G


# ------------------------------------------------------------------ full size: n = 24, A = 2, p = 4

@pytest.fixture(scope="module")
def full24(qvs):
    n, A, p = 24, 2, 4
    port = wl.portfolio(n // 2, wl.rng_for(99, n))
    sim, q = _setup(qvs, n, A, port)
    gs, ts = wl.thetas(p, wl.rng_for(100, 0))
    return n, A, sim, q, np.asarray(gs, float), np.asarray(ts, float)


def test_full24_norm_and_constraint_subspace(full24):
    """The state keeps its norm and stays on weight(odd qubits) - weight(even qubits) = A."""
    n, A, sim, q, gs, ts = full24
    sim.evolve(gs, ts)
    psi = sim.state().astype(np.complex128)
    assert abs(np.sum(np.abs(psi) ** 2) - 1.0) < 1e-5
    idx = np.arange(1 << n, dtype=np.int64)
    w_odd = np.zeros(1 << n, dtype=np.int64)
    w_even = np.zeros(1 << n, dtype=np.int64)
    for qb in range(n):
        bit = (idx >> (n - 1 - qb)) & 1
        if qb % 2:
            w_odd += bit
        else:
            w_even += bit
    outside = (w_odd - w_even) != A
    assert np.max(np.abs(psi[outside])) == 0.0


def test_full24_gradient_vs_central_fd(full24):
    n, A, sim, q, gs, ts = full24
    E, dg, dt = sim.gradient(gs, ts)
    assert rel_err_E(E, sim.evolve(gs, ts)) < TOL_E
    h = 1e-3
    fd = []
    for which in range(2):
        for k in range(len(gs)):
            g2, t2 = gs.copy(), ts.copy()
            (g2 if which == 0 else t2)[k] += h
            ep = sim.evolve(g2, t2)
            (g2 if which == 0 else t2)[k] -= 2 * h
            em = sim.evolve(g2, t2)
            fd.append((ep - em) / (2 * h))
    fd = np.array(fd)
    p = len(gs)
    assert rel_err_grad(dg, dt, fd[:p], fd[p:]) < 2e-3
