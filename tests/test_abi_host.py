"""Host-side checks of the C ABI (no GPU needed): the library builds, loads and exports every
function that include/qvs.h declares; host-only entry points are compared with the oracle."""
import os
import re

import numpy as np
import pytest

import oracle as orc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(qvs_\w+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def qvs():
    from paper_2110_03963_gb300 import _build
    _build.build()
    import paper_2110_03963_gb300 as q
    q.load()
    return q


def test_exports_every_declared_symbol(qvs):
    import ctypes
    lib = ctypes.CDLL(qvs.LIB_PATH)
    declared = _declared()
    assert len(declared) >= 16
    for name in declared:
        assert hasattr(lib, name), name


def test_binding_names_match_header(qvs):
    declared = set(_declared())
    assert declared == set(qvs.EXPORTED)
    for name in declared:
        assert callable(getattr(qvs, name)), name


def test_strerror(qvs):
    assert qvs.strerror(0) == "ok"
    assert "invalid" in qvs.strerror(-1)
    assert qvs.strerror(12345) == "unknown status"


def test_create_rejects_bad_arguments_without_gpu(qvs):
    import ctypes
    lib = qvs.load()
    h = ctypes.c_void_p()
    no_a, no_d = qvs.ALLOC_FN(), qvs.DEALLOC_FN()
    assert lib.qvs_create(ctypes.byref(h), 1, qvs.QVS_C64, None, no_a, no_d, None) == qvs.QVS_EINVAL
    assert lib.qvs_create(ctypes.byref(h), 1024, 7, None, no_a, no_d, None) == qvs.QVS_EINVAL
    assert lib.qvs_create(None, 1024, qvs.QVS_C64, None, no_a, no_d, None) == qvs.QVS_EINVAL
    assert lib.qvs_destroy(None) == qvs.QVS_OK
    assert lib.qvs_evolve(None, 1, None, None) == qvs.QVS_EINVAL
    assert lib.qvs_set_initial_state(None, qvs.QVS_INIT_UNIFORM, None, 0) == qvs.QVS_EINVAL


def test_create_rejects_half_an_allocator_without_gpu(qvs):
    """The device-memory hooks come as a pair: alloc without dealloc (or the reverse) is refused
    before any CUDA call, and no hook is ever called for a refused handle."""
    import ctypes
    lib = qvs.load()
    calls = []
    a = qvs.ALLOC_FN(lambda nbytes, ctx: calls.append(nbytes) or None)
    d = qvs.DEALLOC_FN(lambda ptr, ctx: calls.append(ptr))
    h = ctypes.c_void_p()
    assert lib.qvs_create(ctypes.byref(h), 1024, qvs.QVS_C64, None, a, qvs.DEALLOC_FN(), None) == qvs.QVS_EINVAL
    assert lib.qvs_create(ctypes.byref(h), 1024, qvs.QVS_C64, None, qvs.ALLOC_FN(), d, None) == qvs.QVS_EINVAL
    assert h.value is None and calls == []


@pytest.mark.parametrize("n,k", [(6, 3), (8, 4), (9, 2), (12, 6), (7, 1), (7, 6), (5, 0), (5, 5), (3, 1)])
def test_xy_ring_csr_matches_oracle_operator(qvs, n, k):
    states, rowptr, colind = qvs.qvs_xy_ring_csr(n, k)
    ref_states = orc.subspace_states(n, k)
    assert np.array_equal(states, ref_states)
    rng = np.random.default_rng(n * 100 + k)
    v = rng.standard_normal(states.shape[0]) + 1j * rng.standard_normal(states.shape[0])
    rows = np.repeat(np.arange(states.shape[0]), np.diff(rowptr))
    y = np.zeros_like(v)
    np.add.at(y, rows, 2.0 * v[colind])
    assert np.max(np.abs(y - orc.xy_ring_apply(v, n, states))) < 1e-12


def test_xy_ring_csr_full_size_counts(qvs):
    import math
    import ctypes
    lib = qvs.load()
    dim = ctypes.c_int64()
    nnz = ctypes.c_int64()
    assert lib.qvs_xy_ring_csr(24, 12, None, None, None, ctypes.byref(dim), ctypes.byref(nnz)) == 0
    assert dim.value == math.comb(24, 12)
    assert nnz.value == 2 * 24 * math.comb(22, 11)


def test_qubo_from_maxcut_matches_oracle_maxcut(qvs):
    """The host conversion of a (weighted) edge list gives a quadratic form whose qualities equal
    the oracle's edge-sum max-cut cost."""
    import workloads as wl
    G = wl.regular3_graph(10, wl.rng_for(130))
    c, h, J = qvs.qvs_qubo_from_maxcut(10, G.eu, G.ev)
    assert np.array_equal(orc.qubo_quality(10, c, h, J), orc.maxcut_quality(10, G.eu, G.ev))
    Gw = wl.gnp_graph(11, 0.5, wl.rng_for(131))
    c, h, J = qvs.qvs_qubo_from_maxcut(11, Gw.eu, Gw.ev, Gw.w)
    assert np.max(np.abs(orc.qubo_quality(11, c, h, J) - orc.maxcut_quality(11, Gw.eu, Gw.ev, Gw.w))) < 1e-12
    assert np.all(np.tril(J) == 0)
    with pytest.raises(qvs.QvsError):
        qvs.qvs_qubo_from_maxcut(4, [0], [0])
    with pytest.raises(qvs.QvsError):
        qvs.qvs_qubo_from_maxcut(4, [0], [4])


def test_new_entry_points_reject_bad_arguments_without_gpu(qvs):
    """Argument checks of the quadratic-quality, ex-QAOA and parity-state entry points run before
    any device work, so they are exercised here without a GPU."""
    import ctypes
    lib = qvs.load()
    D = ctypes.POINTER(ctypes.c_double)
    h = np.zeros(4)
    J = np.zeros(16)
    hp, Jp = h.ctypes.data_as(D), J.ctypes.data_as(D)
    dummy = ctypes.c_void_p(1)   # never dereferenced: every call below fails its checks first
    for n in (0, 33):
        assert lib.qvs_quality_qubo(n, 0.0, hp, Jp, qvs.QVS_F32, dummy, None) == qvs.QVS_EINVAL
    assert lib.qvs_quality_qubo(4, 0.0, hp, Jp, qvs.QVS_F32, None, None) == qvs.QVS_EINVAL
    bad = np.array([0.0, np.inf, 0.0, 0.0])
    assert lib.qvs_quality_qubo(4, 0.0, bad.ctypes.data_as(D), Jp, qvs.QVS_F32, dummy, None) == qvs.QVS_EINVAL
    assert lib.qvs_set_quality_qubo(None, 4, 0.0, hp, Jp) == qvs.QVS_EINVAL
    i32 = ctypes.POINTER(ctypes.c_int32)
    u = np.zeros(1, dtype=np.int32)
    assert lib.qvs_set_phase_terms(None, 1, u.ctypes.data_as(i32), u.ctypes.data_as(i32), hp) == qvs.QVS_EINVAL
    g = np.zeros(4)
    E = ctypes.c_double()
    assert lib.qvs_evolve_ex(None, 1, g.ctypes.data_as(D), g.ctypes.data_as(D)) == qvs.QVS_EINVAL
    assert lib.qvs_gradient_ex(None, 1, g.ctypes.data_as(D), g.ctypes.data_as(D), ctypes.byref(E),
                               g.ctypes.data_as(D), g.ctypes.data_as(D)) == qvs.QVS_EINVAL
    for n, A in ((13, 1), (12, 7), (12, -1), (0, 0)):
        assert lib.qvs_state_parity(n, A, dummy, None) == qvs.QVS_EINVAL


def test_bfgs_minimize_matches_oracle(qvs):
    """The library's host BFGS (no GPU involved) against the oracle's written-out BFGS on the same
    functions: a positive-definite quadratic and Rosenbrock."""
    rng = np.random.default_rng(202)
    M = rng.standard_normal((5, 5))
    A = M @ M.T + 5 * np.eye(5)
    b = rng.standard_normal(5)
    quad = lambda x: (0.5 * x @ A @ x - b @ x, A @ x - b)
    # gtol well above the fp64 resolution of the Armijo test (|f| ~ 0.1, so decreases below ~1e-17
    # are invisible and a tighter gtol would only run into the iteration cap)
    x, f, it, ev, stop = qvs.qvs_bfgs_minimize(quad, np.zeros(5), gtol=1e-8)
    xo, fo, ito, evo, stopo = orc.bfgs_minimize(quad, np.zeros(5), gtol=1e-8)
    assert np.max(np.abs(A @ x - b)) <= 1e-8 and it < 200 and stop == stopo == 0
    assert np.max(np.abs(x - np.linalg.solve(A, b))) < 1e-8
    assert (it, ev) == (ito, evo) and abs(f - fo) < 1e-14 and np.max(np.abs(x - xo)) < 1e-12

    def rosen(z):
        a, c = z
        return (1 - a) ** 2 + 100 * (c - a * a) ** 2, np.array([-2 * (1 - a) - 400 * a * (c - a * a), 200 * (c - a * a)])
    x, f, it, ev, stop = qvs.qvs_bfgs_minimize(rosen, np.array([-1.2, 1.0]), gtol=1e-10)
    xo, fo, ito, evo, stopo = orc.bfgs_minimize(rosen, np.array([-1.2, 1.0]), gtol=1e-10)
    assert np.max(np.abs(x - 1.0)) < 1e-8
    assert abs(it - ito) <= 2 and np.max(np.abs(x - xo)) < 1e-8


def test_bfgs_precision_loss_stop_matches_oracle(qvs):
    """Both BFGS loops end with stop = 2 at the same last accepted point when no line-search step
    can lower a rounded objective."""
    import math

    D = np.array([1.0, 3.7])

    def fq(z):
        v = float(np.sum(D * (z - 1.0) ** 2))
        return math.floor(v * 1e6) / 1e6, 2.0 * D * (z - 1.0)
    x0 = np.array([3.0, -2.0])
    x, f, it, ev, stop = qvs.qvs_bfgs_minimize(fq, x0, gtol=1e-12, max_iter=500)
    xo, fo, ito, evo, stopo = orc.bfgs_minimize(fq, x0, gtol=1e-12, max_iter=500)
    assert stop == stopo == 2
    assert (it, ev) == (ito, evo) and f == fo and np.array_equal(x, xo)

    # a bowl with a deterministic noise of up to 1e-6 per point: every rejected trial point is
    # worse than its start, so the library must return the best point it evaluated
    seen = []

    def fn(z):
        h = 0
        for w in np.ascontiguousarray(z, dtype=np.float64).view(np.uint64).tolist():
            h = ((h ^ w) * 0x9E3779B97F4A7C15 + 0x632BE59BD9B4E019) % (1 << 64)
            h ^= h >> 29
        v = float(np.sum(D * (z - 1.0) ** 2)) + 1e-6 * (h % (1 << 53)) / float(1 << 53)
        seen.append(v)
        return v, 2.0 * D * (z - 1.0)
    x, f, it, ev, stop = qvs.qvs_bfgs_minimize(fn, x0, gtol=1e-12, max_iter=500)
    assert stop == 2 and len(seen) == ev and f == min(seen)
    seen.clear()
    xo, fo, ito, evo, stopo = orc.bfgs_minimize(fn, x0, gtol=1e-12, max_iter=500)
    assert (it, ev, stop) == (ito, evo, stopo) and f == fo and np.array_equal(x, xo)


def test_bfgs_minimize_argument_errors_and_callback_failure(qvs):
    with pytest.raises(qvs.QvsError):
        qvs.qvs_bfgs_minimize(lambda x: (0.0, x), np.zeros(0))
    with pytest.raises(ZeroDivisionError):
        qvs.qvs_bfgs_minimize(lambda x: (1.0 / 0.0, x), np.ones(2))


def test_optimise_rejects_bad_arguments_without_gpu(qvs):
    import ctypes
    lib = qvs.load()
    D = ctypes.POINTER(ctypes.c_double)
    g = np.zeros(2)
    f = ctypes.c_double()
    it = ctypes.c_int()
    assert lib.qvs_optimise(None, 1, g.ctypes.data_as(D), g.ctypes.data_as(D), 1e-6, 10, ctypes.byref(f),
                            ctypes.byref(it), ctypes.byref(it), ctypes.byref(it)) == qvs.QVS_EINVAL
    with pytest.raises(qvs.QvsError):
        qvs.qvs_bfgs_minimize(lambda x: (0.0, x), np.zeros(3), gtol=-1.0)


@pytest.mark.parametrize("a,b,t,tol", [(0.0, 30.645, 0.7, 1e-7), (1.5, 3.0, -2.0, 1e-10), (-4.0, 10.0, 2.9, 1e-6),
                                       (2.0, 0.0, 1.3, 1e-7)])
def test_chebyshev_coefficients_vs_bessel_and_expm(qvs, a, b, t, tol):
    """The series coefficients the sparse mixer uses, on the host: equal to the Jacobi-Anger
    coefficients from SciPy's Bessel functions; K the first index whose tail bound drops below tol;
    and the truncated series reproduces scipy's expm on a dense symmetric matrix whose spectrum lies
    in [a - b, a + b] to within that bound."""
    sp = pytest.importorskip("scipy.special")
    la = pytest.importorskip("scipy.linalg")
    c, tail = qvs.qvs_chebyshev_coefficients(a, b, t, tol)
    K = len(c) - 1
    m = np.arange(K + 1)
    ref = np.where(m == 0, 1.0, 2.0) * (-1j) ** m * sp.jv(m, b * t) * np.exp(-1j * t * a)
    assert np.max(np.abs(c - ref)) < 1e-13
    rest = 2.0 * np.abs(sp.jv(np.arange(K + 1, K + 400), b * t))
    assert abs(tail - rest.sum()) < 1e-15 + 1e-9 * tail
    assert tail < tol and (K == 0 or tail + 2.0 * abs(sp.jv(K, b * t)) >= tol)

    rng = np.random.default_rng(205)
    Q, _ = np.linalg.qr(rng.standard_normal((24, 24)))
    lam = a + b * rng.uniform(-1.0, 1.0, 24)
    W = (Q * lam) @ Q.T
    v = rng.standard_normal(24) + 1j * rng.standard_normal(24)
    v /= np.linalg.norm(v)
    Wt = (W - a * np.eye(24)) / b if b > 0 else np.zeros((24, 24))
    t_prev, t_cur = v, Wt @ v
    y = c[0] * t_prev + (c[1] * t_cur if K >= 1 else 0.0)
    for k in range(2, K + 1):
        t_prev, t_cur = t_cur, 2.0 * (Wt @ t_cur) - t_prev
        y = y + c[k] * t_cur
    assert np.linalg.norm(y - la.expm(-1j * t * W) @ v) <= tail + 1e-12


def test_chebyshev_coefficients_argument_errors(qvs):
    for args in [(0.0, -1.0, 1.0, 1e-7), (0.0, 1.0, float("nan"), 1e-7), (0.0, 1.0, 1.0, 0.0)]:
        with pytest.raises(qvs.QvsError):
            qvs.qvs_chebyshev_coefficients(*args)
    with pytest.raises(qvs.QvsError) as e:
        qvs.qvs_chebyshev_coefficients(0.0, 100.0, 10.0, 1e-7, max_terms=50)   # needs ~1000 terms
    assert e.value.status == qvs.QVS_ENUMERIC


def test_qubo_fixed_point_equals_oracle(qvs):
    """The library's host quantiser of quadratic qualities against the oracle's fixed-point rule,
    integer for integer: random forms over six decades of scale, dyadic coefficients with exact
    halves, an all-zero form (F at its upper clamp) and one whose sum S forces F below zero."""
    rng = np.random.default_rng(206)
    cases = []
    for n, scale in ((1, 1.0), (5, 1e-4), (9, 1.0), (16, 1e2), (24, 3e3), (32, 0.5)):
        cases.append((n, scale * rng.standard_normal(), scale * rng.standard_normal(n),
                      np.triu(scale * rng.standard_normal((n, n)), 1) + np.tril(rng.standard_normal((n, n)))))
    # S ~ 3.75 gives F = 28; odd multiples of 2^-29 then sit exactly half-way between grid points
    halves = np.zeros((4, 4))
    halves[0, 1], halves[1, 3] = 3 * 2.0 ** -29, -5 * 2.0 ** -29
    cases.append((4, 0.75, [2.0 ** -29, -(2.0 ** -29), 3.0, 0.0], halves))
    cases.append((3, 0.0, np.zeros(3), np.zeros((3, 3))))
    cases.append((6, 5e9, 1e9 * np.ones(6), np.zeros((6, 6))))
    for n, c, h, J in cases:
        F, ci, hi, Ji = qvs.qvs_qubo_fixed_point(n, c, h, J)
        Fo, cio, hio, Jio = orc.qubo_fixed_point(n, c, h, J)
        assert (F, ci) == (Fo, cio), (n, F, Fo)
        assert hi.tolist() == hio and Ji.tolist() == Jio, n
    F, ci, hi, Ji = qvs.qvs_qubo_fixed_point(4, 0.75, [2.0 ** -29, -(2.0 ** -29), 3.0, 0.0], halves)
    assert F == 28 and hi[:2].tolist() == [1, -1] and (Ji[0, 1], Ji[1, 3]) == (2, -3)   # away from zero
    assert qvs.qvs_qubo_fixed_point(3, 0.0, np.zeros(3), np.zeros((3, 3)))[0] == 40
    assert qvs.qvs_qubo_fixed_point(6, 5e9, 1e9 * np.ones(6), np.zeros((6, 6)))[0] < 0
    with pytest.raises(qvs.QvsError):
        qvs.qvs_qubo_fixed_point(3, float("inf"), np.zeros(3), np.zeros((3, 3)))


@pytest.mark.parametrize("n", [12, 13, 16, 21, 24, 25, 26, 27, 28, 29, 30])
def test_parity_plan_reproduces_the_printed_product(qvs, n):
    """The library's packing of one parity-mixer layer into shared-memory passes (host only), against
    the oracle's factors (B_odd, B_even, B_last of both rings in the printed order): the same gates,
    and every two gates that share a qubit in the printed relative order, so the product is the same
    unitary (gates on disjoint qubits commute). Each pass's gates lie in its 12-bit tile, which holds
    the 4 lowest index bits first; the sweeps cover the gates in order, two at a time when the kind
    says so, with the kind matching how the two gates share bits."""
    plan = qvs.qvs_parity_plan(n)
    printed = [frozenset(pq) for r in orc.parity_ring_rounds(n) for pq in r]
    assert len(set(printed)) == len(printed)
    got = [frozenset((n - 1 - a, n - 1 - b)) for P in plan for (a, b) in P["gates"]]
    assert sorted(map(sorted, got)) == sorted(map(sorted, printed))
    pos = {g: i for i, g in enumerate(got)}
    for i, g in enumerate(printed):
        for h in printed[i + 1:]:
            if g & h:
                assert pos[g] < pos[h], (sorted(g), sorted(h))
    for P in plan:
        tile, gates = P["tile"], P["gates"]
        assert len(set(tile)) == 12 and tile[:4] == [0, 1, 2, 3] and max(tile) < n
        assert all(a in tile and b in tile and a != b for a, b in gates)
        covered = []
        for kind, first in P["sweeps"]:
            assert first == len(covered)
            if kind == 0:
                covered.append(first)
                nxt = first + 1
                assert nxt == len(gates) or set(gates[first]) == set(gates[nxt])
            else:
                shared = len(set(gates[first]) & set(gates[first + 1]))
                assert (kind, shared) in ((1, 0), (2, 1))
                covered += [first, first + 1]
        assert covered == list(range(len(gates)))
    if n == 24:
        assert len(plan) == 3
    if n in (26, 27, 28):
        assert len(plan) == 4


def test_parity_plan_argument_errors(qvs):
    import ctypes
    lib = qvs.load()
    npass = ctypes.c_int()
    for n in (11, 31):
        assert lib.qvs_parity_plan(n, 0, ctypes.byref(npass), None, None, None, None, None, None) == qvs.QVS_EINVAL
    assert lib.qvs_parity_plan(24, 0, None, None, None, None, None, None, None) == qvs.QVS_EINVAL
    buf = (ctypes.c_int32 * 1024)()
    assert lib.qvs_parity_plan(24, 2, ctypes.byref(npass), buf, buf, buf, buf, buf, buf) == qvs.QVS_EINVAL


@pytest.mark.parametrize("n", list(range(12, 33)))
def test_hypercube_plan_composes_the_ansatz(qvs, n):
    """The hypercube pass schedule (host only) composes exactly prod_k exp(-i t_k W) exp(-i g_k Q):
    rotations of different bits commute and the phase is diagonal, so it suffices that each layer's
    phase comes after every rotation of the previous layer, in layer order, and that every index bit
    is rotated exactly once per layer, after that layer's phase. Also: the first pass generates the
    initial state and carries phase 0, the last computes the objective and carries no phase, and
    with three tile types every pass with a phase runs on a high tile type (not the 12 lowest bits)."""
    full = (1 << n) - 1
    for p in (1, 2, 3, 5, 8):
        plan = qvs.qvs_hypercube_plan(n, p)
        three = any(P["type"] == 2 for P in plan)
        rotated = [0] * p
        phases = []

        def rotate(k, bits):
            assert 0 <= k < p and phases and phases[-1] == k   # after phase k, before phase k + 1
            assert rotated[k] & bits == 0, (n, p, k)
            rotated[k] |= bits

        for j, P in enumerate(plan):
            assert P["bits"] != 0 and P["bits"] & ~full == 0
            if P["type"] == 0:
                assert P["bits"] == 0xFFF
            if P["before"] >= 0:
                rotate(P["before"], P["bits"])
            if P["phase"] >= 0:
                k = P["phase"]
                assert k == len(phases) and (k == 0 or rotated[k - 1] == full), (n, p, j)
                phases.append(k)
                assert P["after"] == k
            if P["after"] >= 0:
                rotate(P["after"], P["bits"])
            assert (P["shape"] == 0) == (j == 0) and (P["shape"] == 3) == (j == len(plan) - 1)
            assert (P["phase"] >= 0) == (P["shape"] in (0, 1))
            if three and P["shape"] in (0, 1, 3):
                assert P["type"] != 0, (n, p, j)
        assert phases == list(range(p)) and rotated == [full] * p


def test_hypercube_plan_argument_errors(qvs):
    import ctypes
    lib = qvs.load()
    m = ctypes.c_int()
    for n, p in ((11, 2), (33, 2), (20, 0)):
        assert lib.qvs_hypercube_plan(n, p, 0, ctypes.byref(m), *([None] * 6)) == qvs.QVS_EINVAL
    buf32 = (ctypes.c_int32 * 8)()
    bufu = (ctypes.c_uint32 * 8)()
    assert lib.qvs_hypercube_plan(28, 8, 8, ctypes.byref(m), buf32, buf32, bufu, buf32, buf32, buf32) == qvs.QVS_EINVAL


def test_host_allocation_failure_returns_enomem():
    """No C++ exception crosses the C ABI: in a child process whose address space is capped at
    3 GiB, the XY-ring CSR builder asked for C(33,16) states (a 9.4 GB state list) returns
    QVS_ENOMEM instead of aborting the process."""
    import subprocess
    import sys
    import textwrap
    pytest.importorskip("resource")
    code = textwrap.dedent("""
        import ctypes, resource
        resource.setrlimit(resource.RLIMIT_AS, (3 << 30, 3 << 30))
        import paper_2110_03963_gb300 as q
        lib = q.load()
        dim, nnz = ctypes.c_int64(), ctypes.c_int64()
        print(lib.qvs_xy_ring_csr(33, 16, None, None, None, ctypes.byref(dim), ctypes.byref(nnz)))
    """)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=root, timeout=120)
    assert r.returncode == 0, r.stderr[-500:]
    assert int(r.stdout.strip().splitlines()[-1]) == -2   # QVS_ENOMEM


def _prototypes():
    """{name: [parameter declarations]} of every function include/qvs.h declares."""
    src = open(os.path.join(ROOT, "include", "qvs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for m in re.finditer(r"\b(qvs_\w+)\s*\(", src):
        name, i, depth = m.group(1), m.end(), 1
        j = i
        while depth:
            depth += {"(": 1, ")": -1}.get(src[j], 0)
            j += 1
        if src[j:].lstrip().startswith(";"):
            params, cur, depth = [], "", 0
            for ch in src[i:j - 1]:
                depth += {"(": 1, ")": -1}.get(ch, 0)
                if ch == "," and depth == 0:
                    params.append(cur.strip())
                    cur = ""
                else:
                    cur += ch
            params.append(cur.strip())
            out[name] = [p for p in params if p and p != "void"]
    return out


def test_binding_signatures_match_the_header(qvs):
    """Every ctypes signature the binding sets has the header's parameter count, and each argument
    the header's kind: fp64 by value, 32- or 64-bit integer by value, or a pointer (handles,
    arrays, callbacks)."""
    import ctypes
    lib = qvs.load()
    protos = _prototypes()
    assert set(protos) == set(qvs.EXPORTED)
    pointer_like = (ctypes.c_void_p, ctypes.c_char_p)
    for name, params in protos.items():
        argtypes = getattr(lib, name).argtypes
        assert argtypes is not None and len(argtypes) == len(params), (name, params, argtypes)
        for decl, t in zip(params, argtypes):
            if "*" in decl or "(" in decl or decl.split()[0] in ("qvs_t", "qvs_batch_t", "qvs_fg_fn"):
                ok = (t in pointer_like or issubclass(t, ctypes._Pointer) or issubclass(t, ctypes._CFuncPtr))
                # a typed pointer points to the header's element type
                base = decl.replace("const", "").split("*")[0].split()
                if ok and issubclass(t, ctypes._Pointer) and "(" not in decl and base:
                    want = {"double": ctypes.c_double, "float": ctypes.c_float, "int": ctypes.c_int,
                            "int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "uint32_t": ctypes.c_uint32,
                            "qvs_t": ctypes.c_void_p, "qvs_batch_t": ctypes.c_void_p,
                            "qvs_mixer_desc": qvs.MixerDesc, "qvs_batch_info_t": qvs.BatchInfo}.get(base[0])
                    ok = want is not None and ctypes.sizeof(t._type_) == ctypes.sizeof(want) and (
                        t._type_ is want or (issubclass(want, ctypes._SimpleCData) and
                                             issubclass(t._type_, ctypes._SimpleCData) and
                                             t._type_._type_ == want._type_))
            elif decl.split()[0] == "double":
                ok = t is ctypes.c_double
            elif decl.split()[0] == "int64_t":
                ok = ctypes.sizeof(t) == 8 and issubclass(t, ctypes._SimpleCData) and t not in (ctypes.c_double,)
            elif decl.split()[0] in ("int", "int32_t"):
                ok = t in (ctypes.c_int, ctypes.c_int32)
            else:
                ok = False
            assert ok, (name, decl, t)
    assert lib.qvs_strerror.restype is ctypes.c_char_p


def test_binding_structs_match_the_header(qvs, tmp_path):
    """The binding's ctypes mirrors of qvs_mixer_desc and qvs_batch_info_t have the C structs'
    size and field offsets, as a C compiler lays them out from include/qvs.h."""
    import ctypes
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"qvs_mixer_desc": qvs.MixerDesc, "qvs_batch_info_t": qvs.BatchInfo}
    lines = ['#include <stddef.h>', '#include <stdio.h>', f'#include "{os.path.join(ROOT, "include", "qvs.h")}"',
             "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-o", str(exe), str(src)], check=True, capture_output=True, timeout=60)
    got = {}
    for ln in subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=30).stdout.splitlines():
        cname, field, value = ln.split()
        got[(cname, field)] = int(value)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def test_host_entry_points_degenerate_inputs(qvs):
    """No edges: the quadratic form is zero. No iterations: BFGS returns its start, as the oracle's.
    t = 0: the series is the single coefficient 1."""
    c, h, J = qvs.qvs_qubo_from_maxcut(5, [], [])
    assert c == 0.0 and not h.any() and not J.any()
    quad = lambda x: (float(x @ x), 2.0 * x)
    x0 = np.array([1.0, -2.0])
    x, f, it, ev, stop = qvs.qvs_bfgs_minimize(quad, x0, gtol=1e-8, max_iter=0)
    xo, fo, ito, evo, stopo = orc.bfgs_minimize(quad, x0, gtol=1e-8, max_iter=0)
    assert np.array_equal(x, x0) and (f, it, ev, stop) == (fo, ito, evo, stopo) == (5.0, 0, 1, 1)
    c, tail = qvs.qvs_chebyshev_coefficients(1.5, 10.0, 0.0, 1e-7)
    assert len(c) == 1 and c[0] == 1.0 and tail == 0.0
