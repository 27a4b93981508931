"""GPU checks of the C-ABI boundary: the device-memory hooks of qvs_create, the initial-state kinds
of qvs_set_initial_state and the differentiable objective (torch.autograd) against the fp64 oracle.
The failing allocator is a host-side fake (its alloc returns NULL); no device fault is involved."""
import ctypes
import gc

import numpy as np
import pytest

import oracle as orc
import workloads as wl
from tests.gpu_util import TOL_E, TOL_G, lib, rel_err_E, rel_err_grad

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qvs():
    return lib()


class CountingAllocator:
    """Hooks that serve blocks from the PyTorch caching allocator and record every call."""

    def __init__(self, qvs, fail_after=None, misalign=False):
        import torch
        self.torch = torch
        self.fail_after = fail_after
        self.misalign = misalign
        self.allocs, self.frees, self.live = [], [], {}
        self.alloc_fn = qvs.ALLOC_FN(self._alloc)
        self.dealloc_fn = qvs.DEALLOC_FN(self._dealloc)

    def _alloc(self, nbytes, ctx):
        if self.fail_after is not None and len(self.allocs) >= self.fail_after:
            self.allocs.append(None)
            return None
        ptr = self.torch.cuda.caching_allocator_alloc(int(nbytes) + (256 if self.misalign else 0))
        self.allocs.append(int(nbytes))
        out = ptr + (8 if self.misalign else 0)
        self.live[out] = ptr
        return out

    def _dealloc(self, ptr, ctx):
        self.frees.append(ptr)
        self.torch.cuda.caching_allocator_delete(self.live.pop(ptr))


def _maxcut(qvs, n, seed):
    import torch
    G = wl.gnp_graph(n, 0.5, wl.rng_for(seed, n))
    q = torch.empty(1 << n, dtype=torch.float32, device="cuda")
    qvs.qvs_quality_maxcut(n, G.eu, G.ev, G.w, q, qvs.QVS_F32)
    return G, q


@pytest.mark.parametrize("n", [10, 16])
def test_every_handle_buffer_goes_through_the_hooks(qvs, n):
    """All device buffers of a handle come from the hooks and go back to them at qvs_destroy; the
    results equal those of a handle on cudaMalloc and the oracle's."""
    G, q = _maxcut(qvs, n, 220)
    gs, ts = wl.thetas(3, wl.rng_for(221, n))
    al = CountingAllocator(qvs)
    sim = qvs.Simulator(1 << n, qvs.QVS_C64, allocator=al)
    sim.set_quality(q).set_mixer(qvs.QVS_MIX_HYPERCUBE, qvs.hypercube_desc(n))
    E, dg, dt = sim.gradient(gs, ts)
    assert len(al.allocs) > 0 and all(a is not None for a in al.allocs)
    ref = qvs.Simulator(1 << n, qvs.QVS_C64, allocator=None)
    ref.set_quality(q).set_mixer(qvs.QVS_MIX_HYPERCUBE, qvs.hypercube_desc(n))
    E2, dg2, dt2 = ref.gradient(gs, ts)
    assert E == E2 and np.array_equal(dg, dg2) and np.array_equal(dt, dt2)
    prob = orc.maxcut_problem(n, G.eu, G.ev, G.w, q_dtype=np.float32)
    f, rdg, rdt = orc.gradient(prob, gs, ts)
    assert rel_err_E(E, f) < TOL_E and rel_err_grad(dg, dt, rdg, rdt) < TOL_G
    sim.close()
    ref.close()
    assert len(al.frees) == len(al.allocs) and not al.live


def test_failing_hook_gives_enomem_and_the_handle_recovers(qvs):
    """A hook that refuses memory makes the call that needed it return QVS_ENOMEM; nothing leaks,
    and the same handle works once memory is available again."""
    n = 12
    G, q = _maxcut(qvs, n, 222)
    al = CountingAllocator(qvs, fail_after=0)
    sim = qvs.Simulator(1 << n, qvs.QVS_C64, allocator=al)
    with pytest.raises(qvs.QvsError) as e:
        sim.set_quality(q)
    assert e.value.status == qvs.QVS_ENOMEM
    al.fail_after = None
    sim.set_quality(q).set_mixer(qvs.QVS_MIX_HYPERCUBE, qvs.hypercube_desc(n))
    al.fail_after = len(al.allocs)          # the solve's first buffer is refused
    with pytest.raises(qvs.QvsError) as e:
        sim.gradient([0.3], [0.7])
    assert e.value.status == qvs.QVS_ENOMEM
    al.fail_after = None
    E, dg, dt = sim.gradient([0.3], [0.7])
    prob = orc.maxcut_problem(n, G.eu, G.ev, G.w, q_dtype=np.float32)
    f, rdg, rdt = orc.gradient(prob, [0.3], [0.7])
    assert rel_err_E(E, f) < TOL_E and rel_err_grad(dg, dt, rdg, rdt) < TOL_G
    sim.close()
    assert not al.live


def test_misaligned_hook_block_is_refused(qvs):
    n = 10
    _, q = _maxcut(qvs, n, 223)
    al = CountingAllocator(qvs, misalign=True)
    sim = qvs.Simulator(1 << n, qvs.QVS_C64, allocator=al)
    with pytest.raises(qvs.QvsError) as e:
        sim.set_quality(q)
    assert e.value.status == qvs.QVS_EINVAL
    assert not al.live and len(al.frees) == 1
    sim.close()


def test_default_simulator_uses_the_torch_caching_allocator(qvs):
    import torch
    n = 18
    _, q = _maxcut(qvs, n, 224)
    gc.collect()   # transient tensors of the set-up must not count in the baseline
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    sim = qvs.Simulator(1 << n, qvs.QVS_C64)
    sim.set_quality(q).set_mixer(qvs.QVS_MIX_HYPERCUBE, qvs.hypercube_desc(n))
    sim.gradient([0.3, 0.9], [0.7, 0.2])
    # q copy (1 MiB) + state + adjoint vector (2 MiB each) at least, all counted by PyTorch
    assert torch.cuda.memory_allocated() - before >= 5 * (1 << 20)
    assert sim.allocator.live > 0
    sim.close()
    assert sim.allocator.live == 0
    gc.collect()
    assert torch.cuda.memory_allocated() <= before   # every block the handle took is back


def test_initial_state_kinds(qvs):
    import torch
    n = 14
    G, q = _maxcut(qvs, n, 225)
    sim = qvs.Simulator(1 << n, qvs.QVS_C64)
    sim.set_quality(q).set_mixer(qvs.QVS_MIX_HYPERCUBE, qvs.hypercube_desc(n))
    prob = orc.maxcut_problem(n, G.eu, G.ev, G.w, q_dtype=np.float32)
    gs, ts = [0.4, 1.1], [0.9, 0.3]
    rng = wl.rng_for(226)
    psi0 = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    psi0 = (psi0 / np.linalg.norm(psi0)).astype(np.complex64)
    lib_ = qvs.load()
    # explicit from device memory
    dev = torch.from_numpy(psi0).cuda()
    assert lib_.qvs_set_initial_state(sim.h, qvs.QVS_INIT_EXPLICIT, ctypes.c_void_p(dev.data_ptr()), 1) == 0
    prob.psi0 = psi0.astype(np.complex128)
    assert rel_err_E(sim.evolve(gs, ts), orc.objective(prob, gs, ts)) < TOL_E
    # back to the uniform state
    assert lib_.qvs_set_initial_state(sim.h, qvs.QVS_INIT_UNIFORM, None, 0) == 0
    prob.psi0 = None
    assert rel_err_E(sim.evolve(gs, ts), orc.objective(prob, gs, ts)) < TOL_E
    # bad combinations
    assert lib_.qvs_set_initial_state(sim.h, qvs.QVS_INIT_UNIFORM, ctypes.c_void_p(dev.data_ptr()), 1) == qvs.QVS_EINVAL
    assert lib_.qvs_set_initial_state(sim.h, qvs.QVS_INIT_EXPLICIT, None, 0) == qvs.QVS_EINVAL
    assert lib_.qvs_set_initial_state(sim.h, 7, None, 0) == qvs.QVS_EINVAL
    sim.close()


@pytest.mark.parametrize("dtype", ["float64", "float32"])
def test_autograd_objective_matches_oracle_gradient(qvs, dtype):
    """torch.autograd.grad through QAOAObjective.function gives the oracle's gradient (scaled by
    the upstream gradient) in the dtype and on the device of the parameters."""
    import torch
    n = 13
    G, q = _maxcut(qvs, n, 227)
    sim = qvs.Simulator(1 << n, qvs.QVS_C64)
    sim.set_quality(q).set_mixer(qvs.QVS_MIX_HYPERCUBE, qvs.hypercube_desc(n))
    gs, ts = wl.thetas(3, wl.rng_for(228))
    tdt = getattr(torch, dtype)
    g = torch.tensor(gs, dtype=tdt, device="cuda", requires_grad=True)
    t = torch.tensor(ts, dtype=tdt, device="cuda", requires_grad=True)
    E = qvs.QAOAObjective.function(sim)(g, t)
    loss = 2.5 * E
    dg, dt = torch.autograd.grad(loss, (g, t))
    assert dg.dtype == tdt and dg.device == g.device and dt.shape == t.shape
    prob = orc.maxcut_problem(n, G.eu, G.ev, G.w, q_dtype=np.float32)
    f, rdg, rdt = orc.gradient(prob, g.detach().cpu().double().numpy(), t.detach().cpu().double().numpy())
    assert rel_err_E(float(E.detach()), f) < TOL_E
    assert rel_err_grad(dg.cpu().double().numpy() / 2.5, dt.cpu().double().numpy() / 2.5, rdg, rdt) < TOL_G
    sim.close()
