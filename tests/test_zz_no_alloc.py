"""The allocation-free small-state solve (qvs_gradient_small_noalloc) against the handle-based
qvs_gradient, through the C ABI, twice in a row (the static scratch keeps the previous call's
contents, which must not leak into the next result).

It serves callers that cannot allocate device memory when they need a solve (allocator
callbacks, fixed-budget real-time loops, runtimes that own all device memory). This file
is collected last so that a failure here comes after every other test has run."""
import numpy as np
import pytest

import oracle as orc
import workloads as wl
from tests.gpu_util import TOL_E, TOL_G, lib, rel_err_E, rel_err_grad

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qvs():
    return lib()


@pytest.mark.parametrize("precision,n,p", [("c64", 10, 3), ("c128", 10, 3), ("c64", 12, 5)])
def test_noalloc_matches_handle_solve_twice(qvs, precision, n, p):
    import torch
    prec = qvs.QVS_C64 if precision == "c64" else qvs.QVS_C128
    tdt = torch.float32 if precision == "c64" else torch.float64
    G = wl.gnp_graph(n, 0.5, wl.rng_for(90, n))
    q = torch.empty(1 << n, dtype=tdt, device="cuda")
    qvs.qvs_quality_maxcut(n, G.eu, G.ev, G.w, q, qvs.QVS_F32 if precision == "c64" else qvs.QVS_F64)
    sim = qvs.Simulator(1 << n, prec)
    sim.set_quality(q).set_mixer(qvs.QVS_MIX_HYPERCUBE, qvs.hypercube_desc(n))
    tol_e, tol_g = (TOL_E, TOL_G) if precision == "c64" else (1e-12, 1e-11)
    for call in range(2):
        gs, ts = wl.thetas(p, wl.rng_for(91, 10 * n + call))
        E, dg, dt = sim.gradient(gs, ts)
        out = torch.full((1 + 2 * p,), float("nan"), dtype=torch.float64, device="cuda")
        qvs.qvs_gradient_small_noalloc(n, prec, q, gs, ts, out)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        assert rel_err_E(o[0], E) < tol_e
        assert rel_err_grad(o[1:1 + p], o[1 + p:], dg, dt) < tol_g
    sim.close()


@pytest.mark.parametrize("precision,n,p", [("c64", 10, 4), ("c128", 10, 4), ("c64", 12, 3), ("c128", 12, 3)])
def test_noalloc_matches_the_oracle(qvs, precision, n, p):
    """The allocation-free solve against the fp64 oracle directly, on two calls in a row with
    different graphs and parameters; the second call also takes no memory from PyTorch or the
    device."""
    import torch
    prec = qvs.QVS_C64 if precision == "c64" else qvs.QVS_C128
    tdt = torch.float32 if precision == "c64" else torch.float64
    tol_e, tol_g = (TOL_E, TOL_G) if precision == "c64" else (1e-12, 1e-11)
    for call in range(2):
        G = wl.gnp_graph(n, 0.5, wl.rng_for(92, 10 * n + call))
        q = torch.empty(1 << n, dtype=tdt, device="cuda")
        qvs.qvs_quality_maxcut(n, G.eu, G.ev, G.w, q, qvs.QVS_F32 if precision == "c64" else qvs.QVS_F64)
        gs, ts = wl.thetas(p, wl.rng_for(93, 10 * n + call))
        out = torch.full((1 + 2 * p,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        stats0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
        free0, _ = torch.cuda.mem_get_info()
        qvs.qvs_gradient_small_noalloc(n, prec, q, gs, ts, out)
        torch.cuda.synchronize()
        if call == 1:
            assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == stats0
            assert torch.cuda.mem_get_info()[0] == free0
        o = out.cpu().numpy()
        prob = orc.maxcut_problem(n, G.eu, G.ev, G.w, q_dtype=np.float32 if precision == "c64" else None)
        f, rdg, rdt = orc.gradient(prob, gs, ts)
        assert rel_err_E(o[0], f) < tol_e
        assert rel_err_grad(o[1:1 + p], o[1 + p:], rdg, rdt) < tol_g


def test_noalloc_rejects_sizes_beyond_the_scratch(qvs):
    import torch
    n = 12
    q = torch.zeros(1 << n, dtype=torch.float64, device="cuda")
    out = torch.zeros(1 + 2 * 65, dtype=torch.float64, device="cuda")
    # 65 complex128 states of 2^12 amplitudes need 4.06 MiB > the 4 MiB scratch
    with pytest.raises(qvs.QvsError) as e:
        qvs.qvs_gradient_small_noalloc(n, qvs.QVS_C128, q, np.zeros(65), np.zeros(65), out)
    assert e.value.status == qvs.QVS_EINVAL
    with pytest.raises(qvs.QvsError):
        qvs.qvs_gradient_small_noalloc(13, qvs.QVS_C64, q, [0.1], [0.2], out)
