"""GPU check of the host BFGS loop over the device objective and gradient (qvs_optimise, Sec. 4)
against the oracle's BFGS on the fp64 objective."""
import numpy as np
import pytest

import oracle as orc
import workloads as wl
from tests.gpu_util import lib, rel_err_E

pytestmark = pytest.mark.gpu


def test_optimise_qaoa_p1_matches_oracle():
    import torch
    qvs = lib()
    n = 13
    G = wl.gnp_graph(n, 0.5, wl.rng_for(210, n))
    q = torch.empty(1 << n, dtype=torch.float32, device="cuda")
    qvs.qvs_quality_maxcut(n, G.eu, G.ev, G.w, q, qvs.QVS_F32)
    sim = qvs.Simulator(1 << n, qvs.QVS_C64)
    sim.set_quality(q).set_mixer(qvs.QVS_MIX_HYPERCUBE, qvs.hypercube_desc(n))
    gs, ts, f, it, ev, stop = sim.optimise(np.array([0.6]), np.array([0.4]), gtol=1e-4, max_iter=100)
    prob = orc.maxcut_problem(n, G.eu, G.ev, G.w, q_dtype=np.float32)
    go, to, fo, ito, evo, _ = orc.optimise(prob, np.array([0.6]), np.array([0.4]), gtol=1e-8)
    assert rel_err_E(f, fo) < 1e-5
    # the returned parameters reproduce the returned objective, and the optimum was descended to
    assert rel_err_E(sim.evolve(gs, ts), f) < 1e-6
    assert f < orc.objective(prob, [0.6], [0.4])
    sim.close()
