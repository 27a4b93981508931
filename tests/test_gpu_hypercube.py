"""GPU parity of the QAOA hypercube path (through the C ABI) against the fp64 oracle."""
import math

import numpy as np
import pytest

import oracle as orc
import workloads as wl
from tests import closed_forms as cf
from tests.gpu_util import TOL_E, TOL_E_C128, TOL_G, infidelity, lib, rel_err_E, rel_err_grad

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qvs():
    return lib()


def _torch():
    import torch
    assert torch.cuda.is_available()
    return torch


def _sim_maxcut(qvs, n, G, precision, q_dtype):
    """Simulator whose q comes from the library's own device generator."""
    torch = _torch()
    dim = 1 << n
    if q_dtype == "i32":
        q = torch.empty(dim, dtype=torch.int32, device="cuda")
        qvs.qvs_quality_maxcut(n, G.eu, G.ev, None, q, qvs.QVS_I32)
    elif q_dtype == "f32":
        q = torch.empty(dim, dtype=torch.float32, device="cuda")
        qvs.qvs_quality_maxcut(n, G.eu, G.ev, G.w, q, qvs.QVS_F32)
    else:
        q = torch.empty(dim, dtype=torch.float64, device="cuda")
        qvs.qvs_quality_maxcut(n, G.eu, G.ev, G.w, q, qvs.QVS_F64)
    sim = qvs.Simulator(dim, precision)
    sim.set_quality(q)
    sim.set_mixer(qvs.QVS_MIX_HYPERCUBE, qvs.hypercube_desc(n))
    return sim, q


# ------------------------------------------------------------------ quality vectors: bit-exact

@pytest.mark.parametrize("n", [10, 16, 21])
def test_maxcut_quality_int_bit_exact(qvs, n):
    torch = _torch()
    G = wl.regular3_graph(n, wl.rng_for(50, n))
    q = torch.empty(1 << n, dtype=torch.int32, device="cuda")
    qvs.qvs_quality_maxcut(n, G.eu, G.ev, None, q, qvs.QVS_I32)
    ref = orc.maxcut_quality(n, G.eu, G.ev)
    assert np.array_equal(q.cpu().numpy(), ref.astype(np.int32))


@pytest.mark.parametrize("n", [12, 20])
def test_maxcut_quality_weighted_bit_exact(qvs, n):
    torch = _torch()
    G = wl.gnp_graph(n, 0.5, wl.rng_for(51, n))
    q32 = torch.empty(1 << n, dtype=torch.float32, device="cuda")
    qvs.qvs_quality_maxcut(n, G.eu, G.ev, G.w, q32, qvs.QVS_F32)
    q64 = torch.empty(1 << n, dtype=torch.float64, device="cuda")
    qvs.qvs_quality_maxcut(n, G.eu, G.ev, G.w, q64, qvs.QVS_F64)
    ref = orc.maxcut_quality(n, G.eu, G.ev, G.w)
    assert np.array_equal(q64.cpu().numpy(), ref)
    assert np.array_equal(q32.cpu().numpy(), ref.astype(np.float32))


def test_maxcut_quality_full_size_sampled(qvs):
    """n=28 weighted G(28,1/2): sampled entries against the oracle's definition (one by one)."""
    torch = _torch()
    inst = wl.wmaxcut(28, 8)
    G = inst.graph
    q = torch.empty(1 << 28, dtype=torch.float32, device="cuda")
    qvs.qvs_quality_maxcut(28, G.eu, G.ev, G.w, q, qvs.QVS_F32)
    idx = np.concatenate([np.arange(64), wl.rng_for(52, 0).integers(0, 1 << 28, 4096), [(1 << 28) - 1]])
    got = q[torch.from_numpy(idx).cuda()].cpu().numpy()
    # evaluate the oracle's definition on the sampled basis states only
    x = orc.qubit_bits(28, idx)
    ref = np.zeros(idx.shape[0])
    for e in range(G.m):
        ref += np.where(x[G.eu[e]] == x[G.ev[e]], G.w[e], 0.0)
    assert np.array_equal(got, ref.astype(np.float32))


# ------------------------------------------------------------------ small path (n <= 12)

def test_config1_maxcut10_c128_forward(qvs):
    inst = wl.maxcut10()
    G = inst.graph
    sim, _ = _sim_maxcut(qvs, 10, G, qvs.QVS_C128, "i32")
    E = sim.evolve(inst.gammas, inst.ts)
    prob = orc.maxcut_problem(10, G.eu, G.ev)
    ref_psi = orc.evolve(prob, inst.gammas, inst.ts)
    ref = orc.expectation(ref_psi, prob.q)
    assert rel_err_E(E, ref) < TOL_E_C128
    assert infidelity(sim.state(), ref_psi) < 1e-13
    E2, dg, dt = sim.gradient(inst.gammas, inst.ts)
    f, rdg, rdt = orc.gradient(prob, inst.gammas, inst.ts)
    assert rel_err_E(E2, f) < TOL_E_C128
    assert rel_err_grad(dg, dt, rdg, rdt) < 1e-11


@pytest.mark.parametrize("n,precision", [(8, "c64"), (12, "c64"), (12, "c128"), (5, "c64")])
def test_small_path_gradient(qvs, n, precision):
    G = wl.gnp_graph(n, 0.5, wl.rng_for(53, n))
    prec = qvs.QVS_C64 if precision == "c64" else qvs.QVS_C128
    sim, _ = _sim_maxcut(qvs, n, G, prec, "f32" if precision == "c64" else "f64")
    gs, ts = wl.thetas(4, wl.rng_for(54, n))
    E, dg, dt = sim.gradient(gs, ts)
    prob = orc.maxcut_problem(n, G.eu, G.ev, G.w, q_dtype=np.float32 if precision == "c64" else None)
    f, rdg, rdt = orc.gradient(prob, gs, ts)
    tol_e = TOL_E if precision == "c64" else TOL_E_C128
    assert rel_err_E(E, f) < tol_e
    assert rel_err_grad(dg, dt, rdg, rdt) < (TOL_G if precision == "c64" else 1e-11)


# ------------------------------------------------------------------ tiled path

@pytest.mark.parametrize("n,p", [(13, 1), (14, 3), (16, 2), (18, 4), (20, 5), (21, 2), (22, 3), (23, 1)])
def test_tiled_forward_and_gradient_c64(qvs, n, p):
    G = wl.gnp_graph(n, 0.5, wl.rng_for(55, n))
    sim, _ = _sim_maxcut(qvs, n, G, qvs.QVS_C64, "f32")
    gs, ts = wl.thetas(p, wl.rng_for(56, n * 10 + p))
    prob = orc.maxcut_problem(n, G.eu, G.ev, G.w, q_dtype=np.float32)
    E = sim.evolve(gs, ts)
    ref_psi = orc.evolve(prob, gs, ts)
    ref = orc.expectation(ref_psi, prob.q)
    assert rel_err_E(E, ref) < TOL_E
    assert infidelity(sim.state(), ref_psi) < 1e-6
    E2, dg, dt = sim.gradient(gs, ts)
    f, rdg, rdt = orc.gradient(prob, gs, ts)
    assert rel_err_E(E2, f) < TOL_E
    assert rel_err_grad(dg, dt, rdg, rdt) < TOL_G


# Mixer angles where the kernels shift t by pi/2 (|tan t| > 1) and carry the remaining all-bit flip
# as a frame: every layer flipped, alternating, on the |tan t| = 1 boundary, exactly pi/2 (tangent
# 0 after the shift), 0 and pi; odd and even n, two- and three-group schedules.
FRAME_TS = {
    "all_flip": [1.3, 1.9, 1.6, 1.45],
    "alternate": [0.4, 1.7, 2.9, 1.2],
    "boundary": [math.pi / 4, 3 * math.pi / 4, math.pi / 4 + 1e-9, 3 * math.pi / 4 - 1e-9],
    "exact": [math.pi / 2, 0.0, math.pi, math.pi / 2],
}


@pytest.mark.parametrize("n", [13, 14, 21, 22])
@pytest.mark.parametrize("pattern", sorted(FRAME_TS))
def test_tiled_angle_frames_c64(qvs, n, pattern):
    G = wl.gnp_graph(n, 0.5, wl.rng_for(67, n))
    sim, _ = _sim_maxcut(qvs, n, G, qvs.QVS_C64, "f32")
    ts = np.array(FRAME_TS[pattern])
    gs = np.array([0.7, 2.3, 1.1, 0.2])
    prob = orc.maxcut_problem(n, G.eu, G.ev, G.w, q_dtype=np.float32)
    E = sim.evolve(gs, ts)
    ref_psi = orc.evolve(prob, gs, ts)
    assert rel_err_E(E, orc.expectation(ref_psi, prob.q)) < TOL_E
    assert infidelity(sim.state(), ref_psi) < 1e-6
    # the returned state carries the right global phase too (not only up to a phase)
    assert np.max(np.abs(sim.state() - ref_psi)) < 5e-6 / math.sqrt(1 << n) * 64
    E2, dg, dt = sim.gradient(gs, ts)
    f, rdg, rdt = orc.gradient(prob, gs, ts)
    assert rel_err_E(E2, f) < TOL_E
    assert rel_err_grad(dg, dt, rdg, rdt) < TOL_G


@pytest.mark.parametrize("pattern", ["all_flip", "alternate"])
def test_tiled_angle_frames_c128_tight(qvs, pattern):
    n = 15
    G = wl.gnp_graph(n, 0.5, wl.rng_for(68, n))
    sim, _ = _sim_maxcut(qvs, n, G, qvs.QVS_C128, "f64")
    ts = np.array(FRAME_TS[pattern])
    gs = np.array([0.7, 2.3, 1.1, 0.2])
    prob = orc.maxcut_problem(n, G.eu, G.ev, G.w)
    E = sim.evolve(gs, ts)
    ref_psi = orc.evolve(prob, gs, ts)
    assert np.max(np.abs(sim.state() - ref_psi)) < 1e-12
    E2, dg, dt = sim.gradient(gs, ts)
    f, rdg, rdt = orc.gradient(prob, gs, ts)
    assert rel_err_E(E2, f) < 1e-11
    assert rel_err_grad(dg, dt, rdg, rdt) < 1e-10


@pytest.mark.parametrize("n", [14, 22])
def test_tiled_c128_matches_oracle_tightly(qvs, n):
    G = wl.gnp_graph(n, 0.5, wl.rng_for(57, n))
    sim, _ = _sim_maxcut(qvs, n, G, qvs.QVS_C128, "f64")
    gs, ts = wl.thetas(3, wl.rng_for(58, n))
    prob = orc.maxcut_problem(n, G.eu, G.ev, G.w)
    E, dg, dt = sim.gradient(gs, ts)
    f, rdg, rdt = orc.gradient(prob, gs, ts)
    assert rel_err_E(E, f) < 1e-11
    assert rel_err_grad(dg, dt, rdg, rdt) < 1e-10


@pytest.mark.parametrize("ckpt", [1, 2, 0, 100])
def test_checkpoint_intervals_agree(qvs, ckpt):
    n, p = 22, 6
    G = wl.gnp_graph(n, 0.5, wl.rng_for(59, 0))
    sim, _ = _sim_maxcut(qvs, n, G, qvs.QVS_C64, "f32")
    sim.set_option(qvs.QVS_OPT_CKPT_LAYERS, ckpt)
    gs, ts = wl.thetas(p, wl.rng_for(60, 0))
    prob = orc.maxcut_problem(n, G.eu, G.ev, G.w, q_dtype=np.float32)
    E, dg, dt = sim.gradient(gs, ts)
    f, rdg, rdt = orc.gradient(prob, gs, ts)
    assert rel_err_E(E, f) < TOL_E
    assert rel_err_grad(dg, dt, rdg, rdt) < TOL_G


def test_explicit_initial_state(qvs):
    n = 15
    G = wl.gnp_graph(n, 0.5, wl.rng_for(61, 0))
    sim, _ = _sim_maxcut(qvs, n, G, qvs.QVS_C64, "f32")
    rng = wl.rng_for(62, 0)
    psi0 = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    psi0 /= np.linalg.norm(psi0)
    sim.set_initial_state(psi0.astype(np.complex64))
    prob = orc.maxcut_problem(n, G.eu, G.ev, G.w, q_dtype=np.float32)
    prob.psi0 = psi0.astype(np.complex64).astype(np.complex128)
    gs, ts = [0.5, 1.9], [2.2, 0.3]
    E, dg, dt = sim.gradient(gs, ts)
    f, rdg, rdt = orc.gradient(prob, gs, ts)
    assert rel_err_E(E, f) < TOL_E
    assert rel_err_grad(dg, dt, rdg, rdt) < TOL_G


def test_integer_quality_c64(qvs):
    n = 17
    G = wl.regular3_graph(n, wl.rng_for(63, 0))
    sim, _ = _sim_maxcut(qvs, n, G, qvs.QVS_C64, "i32")
    gs, ts = wl.thetas(3, wl.rng_for(64, 0))
    prob = orc.maxcut_problem(n, G.eu, G.ev)
    E, dg, dt = sim.gradient(gs, ts)
    f, rdg, rdt = orc.gradient(prob, gs, ts)
    assert rel_err_E(E, f) < TOL_E
    assert rel_err_grad(dg, dt, rdg, rdt) < TOL_G


def test_deterministic_repeat(qvs):
    n = 20
    G = wl.gnp_graph(n, 0.5, wl.rng_for(65, 0))
    sim, _ = _sim_maxcut(qvs, n, G, qvs.QVS_C64, "f32")
    gs, ts = wl.thetas(3, wl.rng_for(66, 0))
    a = sim.gradient(gs, ts)
    b = sim.gradient(gs, ts)
    assert a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


# ------------------------------------------------------------------ full size n=28 (config: weighted G(28,1/2), p=8)

@pytest.fixture(scope="module")
def full28(qvs):
    inst = wl.wmaxcut(28, 8)
    sim, q = _sim_maxcut(qvs, 28, inst.graph, qvs.QVS_C64, "f32")
    return inst, sim, q


def test_full28_p1_closed_form(full28):
    """p=1 objective and gradient against the closed form (valid at any n)."""
    inst, sim, q = full28
    G = inst.graph
    for gamma, t in [(inst.gammas[0], inst.ts[0]), (0.05, 0.4)]:
        E, dg, dt = sim.gradient([gamma], [t])
        w32 = G.w   # q is the fp32 rounding of the fp64 weighted sum; the closed form uses fp64 weights
        ref = cf.p1_maxcut_expectation(28, G.eu, G.ev, w32, gamma, t)
        rg, rt = cf.p1_maxcut_gradient(28, G.eu, G.ev, w32, gamma, t)
        # fp32 rounding of q moves E by <= max|q| * 2^-24 relative
        assert rel_err_E(E, ref) < TOL_E
        assert rel_err_grad(np.array([dg[0]]), np.array([dt[0]]), np.array([rg]), np.array([rt])) < TOL_G


def test_full28_p1_sampled_amplitudes(full28, qvs):
    inst, sim, q = full28
    gamma, t = 0.31, 0.77
    sim.evolve([gamma], [t])
    psi = sim.state()
    qh = q.cpu().numpy().astype(np.float64)
    for i in [0, 12345, (1 << 28) - 1, 1 << 27]:
        a = cf.p1_hypercube_amplitude(28, qh, gamma, t, i)
        assert abs(psi[i] - a) < 1e-6 * max(abs(a), 1.0 / math.sqrt(1 << 28)) * 50


def test_full28_p8_invariants(full28):
    inst, sim, q = full28
    gs, ts = inst.gammas, inst.ts
    E = sim.evolve(gs, ts)
    psi = sim.state()
    norm = float(np.sum(np.abs(psi.astype(np.complex128)) ** 2))
    assert abs(norm - 1.0) < 1e-4
    qmin, qmax = float(q.min()), float(q.max())
    assert qmin <= E <= qmax
    # hypercube: exp(-i pi X) = -I, so E is unchanged by t_k -> t_k + pi
    ts2 = np.array(ts, dtype=float)
    ts2[3] += math.pi
    assert rel_err_E(sim.evolve(gs, ts2), E) < TOL_E
    # real psi0 and real q: E(-gamma, -t) = E(gamma, t)
    assert rel_err_E(sim.evolve(-np.asarray(gs), -np.asarray(ts)), E) < TOL_E
    Eg, dg, dt = sim.gradient(gs, ts)
    assert rel_err_E(Eg, E) < TOL_E


def test_full28_p8_gradient_vs_c128_central_fd(full28, qvs):
    """All 16 adjoint gradient entries (complex64) against central differences of the complex128
    path (h = 1e-4, truncation error ~1e-9), both through the C ABI."""
    torch = _torch()
    inst, sim, q = full28
    gs, ts = np.asarray(inst.gammas, float), np.asarray(inst.ts, float)
    E, dg, dt = sim.gradient(gs, ts)
    q64 = torch.empty(1 << 28, dtype=torch.float64, device="cuda")
    q64.copy_(q)
    s128 = qvs.Simulator(1 << 28, qvs.QVS_C128)
    s128.set_quality(q64)
    s128.set_mixer(qvs.QVS_MIX_HYPERCUBE, qvs.hypercube_desc(28))
    del q64
    h = 1e-4

    def fd(which, k):
        def ev(delta):
            g2, t2 = gs.copy(), ts.copy()
            (g2 if which == 0 else t2)[k] += delta
            return s128.evolve(g2, t2)
        return (ev(h) - ev(-h)) / (2 * h)

    rdg = np.array([fd(0, k) for k in range(8)])
    rdt = np.array([fd(1, k) for k in range(8)])
    s128.close()
    assert rel_err_grad(dg, dt, rdg, rdt) < TOL_G


@pytest.mark.parametrize("n,p", [(13, 3), (14, 2), (16, 4), (19, 3), (21, 2), (25, 2)])
def test_staged_passes_bit_identical_to_per_tile(qvs, n, p):
    """The TMA-staged persistent passes (QVS_OPT_STAGED = 1) read the same inputs from a shared
    stage instead of global memory and do the same arithmetic, so objective and gradient equal the
    one-CTA-per-tile kernels' bit for bit; covers chunk widths s = 11 (n = 13) down to s = 4 and
    both frames (random t spans |tan t| > 1)."""
    import torch
    G = wl.gnp_graph(n, 0.5, wl.rng_for(260, n))
    q = torch.empty(1 << n, dtype=torch.float32, device="cuda")
    qvs.qvs_quality_maxcut(n, G.eu, G.ev, G.w, q, qvs.QVS_F32)
    gs, ts = wl.thetas(p, wl.rng_for(261, n))
    out = []
    for staged in (0, 1):
        sim = qvs.Simulator(1 << n, qvs.QVS_C64)
        sim.set_quality(q).set_mixer(qvs.QVS_MIX_HYPERCUBE, qvs.hypercube_desc(n))
        sim.set_option(qvs.QVS_OPT_STAGED, staged)
        out.append(sim.gradient(gs, ts))
        sim.close()
    (E0, dg0, dt0), (E1, dg1, dt1) = out
    assert E0 == E1 and np.array_equal(dg0, dg1) and np.array_equal(dt0, dt1)
    prob = orc.maxcut_problem(n, G.eu, G.ev, G.w, q_dtype=np.float32)
    if n <= 21:
        f, rdg, rdt = orc.gradient(prob, gs, ts)
        assert rel_err_E(E1, f) < TOL_E and rel_err_grad(dg1, dt1, rdg, rdt) < TOL_G
