"""Python binding of libqvs: a single-GPU (sm_103a) state-vector engine for quantum variational
algorithms (QAOA, QWOA, QAOAz; Matwiejew & Wang, arXiv 2110.03963).

The binding only marshals arguments: every step of the evolution, objective and gradient runs in
the CUDA kernels of ``libqvs.so`` (built in-tree by ``_build.py``). PyTorch supplies device memory
for inputs/outputs given as tensors and the CUDA stream. Loading fails loudly if the library is
missing; there is no CPU fallback. Before each call, every buffer passed as a bare pointer is
checked against the element count, dtype and side (host or device) the library will use, taken
from what the binding recorded when it created the handle or batch.

Function names match the C ABI in ``include/qvs.h``.
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libqvs.so")

QVS_OK, QVS_EINVAL, QVS_ENOMEM, QVS_ECUDA, QVS_ESTATE, QVS_ENUMERIC, QVS_ETIMEOUT, QVS_EUNSUPPORTED = \
    0, -1, -2, -3, -4, -5, -6, -7
QVS_C64, QVS_C128 = 1, 2
QVS_I32, QVS_F32, QVS_F64 = 1, 2, 3
QVS_INIT_UNIFORM, QVS_INIT_EXPLICIT = 0, 1
QVS_MIX_HYPERCUBE, QVS_MIX_CIRCULANT, QVS_MIX_CSR, QVS_MIX_PARITY, QVS_MIX_XY_RING = 1, 2, 3, 4, 5
QVS_OPT_CKPT_LAYERS = 1
QVS_OPT_PROFILE = 2
QVS_OPT_STAGED = 3

EXPORTED = [
    "qvs_create", "qvs_destroy", "qvs_set_quality", "qvs_set_mixer", "qvs_set_initial_state",
    "qvs_set_option", "qvs_evolve", "qvs_expectation", "qvs_gradient", "qvs_get_state",
    "qvs_last_launch_count", "qvs_kernel_stats", "qvs_quality_maxcut", "qvs_quality_subset", "qvs_quality_portfolio",
    "qvs_xy_ring_csr", "qvs_chebyshev_coefficients", "qvs_parity_plan", "qvs_hypercube_plan", "qvs_tile_layout", "qvs_state_parity", "qvs_batch_create", "qvs_batch_set_quality", "qvs_batch_gradient",
    "qvs_batch_info", "qvs_batch_destroy", "qvs_gradient_small_noalloc", "qvs_strerror",
    "qvs_set_quality_qubo", "qvs_quality_qubo", "qvs_qubo_fixed_point", "qvs_qubo_from_maxcut",
    "qvs_set_phase_terms", "qvs_evolve_ex", "qvs_gradient_ex", "qvs_bfgs_minimize", "qvs_optimise",
    "qvs_batch_set_quality_shared", "qvs_batch_optimise", "qvs_benchmark", "qvs_batch_set_schedule",
]


class QvsError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {strerror(status)} ({status})")


class MixerDesc(ctypes.Structure):
    _fields_ = [
        ("n_qubits", ctypes.c_int),
        ("n_offsets", ctypes.c_int),
        ("offsets", ctypes.POINTER(ctypes.c_int64)),
        ("offset_weights", ctypes.POINTER(ctypes.c_double)),
        ("rowptr", ctypes.c_void_p),
        ("colind", ctypes.c_void_p),
        ("values", ctypes.c_void_p),
        ("implicit_value", ctypes.c_float),
        ("nnz", ctypes.c_int64),
        ("csr_on_device", ctypes.c_int),
        ("spec_lo", ctypes.c_double),
        ("spec_hi", ctypes.c_double),
        ("cheb_tol", ctypes.c_double),
        ("hamming_weight", ctypes.c_int),
    ]


class BatchInfo(ctypes.Structure):
    _fields_ = [
        ("ctas_per_sm", ctypes.c_int),
        ("shared_quality", ctypes.c_int),
        ("trial_ms", ctypes.c_double * 2),
        ("bytes_per_solve", ctypes.c_double),
        ("fma_per_solve", ctypes.c_double),
        ("amp_layers", ctypes.c_double),
        ("ckpt_policy", ctypes.c_int),
        ("from_cache", ctypes.c_int),
        ("trial_ms_all", ctypes.c_double * 4),
    ]


_lib = None

# device-memory hooks of qvs_create: alloc(bytes, ctx) -> pointer or NULL; dealloc(pointer, ctx)
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
DEALLOC_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

# objective-and-gradient callback of qvs_bfgs_minimize: (x, f, g, user) -> status
FG_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                         ctypes.POINTER(ctypes.c_double), ctypes.c_void_p)


def load(path: str = LIB_PATH):
    """Load libqvs.so (raises if it is missing: build it with ``_build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libqvs.so not built at {path}; run paper_2110_03963_gb300._build.build()")
    lib = ctypes.CDLL(path)
    P, I, I64, D, V = ctypes.POINTER, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
    sig = {
        "qvs_create": (I, [P(V), I64, I, V, ALLOC_FN, DEALLOC_FN, V]),
        "qvs_destroy": (I, [V]),
        "qvs_set_quality": (I, [V, V, I, I]),
        "qvs_set_mixer": (I, [V, I, P(MixerDesc)]),
        "qvs_set_initial_state": (I, [V, I, V, I]),
        "qvs_set_option": (I, [V, I, I64]),
        "qvs_evolve": (I, [V, I, P(D), P(D)]),
        "qvs_expectation": (I, [V, P(D)]),
        "qvs_gradient": (I, [V, I, P(D), P(D), P(D), P(D), P(D)]),
        "qvs_get_state": (I, [V, V, I]),
        "qvs_last_launch_count": (I, [V, P(I64)]),
        "qvs_kernel_stats": (I, [V, I, ctypes.c_char_p, I, P(I64), P(D), P(D)]),
        "qvs_quality_maxcut": (I, [I, I, P(ctypes.c_int32), P(ctypes.c_int32), P(D), I, V, V]),
        "qvs_quality_subset": (I, [I, P(D), I, V, V]),
        "qvs_quality_portfolio": (I, [I, I64, V, P(D), P(D), D, I, V, V]),
        "qvs_xy_ring_csr": (I, [I, I, V, V, V, P(I64), P(I64)]),
        "qvs_chebyshev_coefficients": (I, [D, D, D, D, I, P(D), P(I), P(D)]),
        "qvs_parity_plan": (I, [I, I, P(I)] + [P(ctypes.c_int32)] * 6),
        "qvs_tile_layout": (I, [I, I, I, P(ctypes.c_int32), P(ctypes.c_int32), P(ctypes.c_int32), P(I), P(I), P(I)]),
        "qvs_hypercube_plan": (I, [I, I, I, P(I), P(ctypes.c_int32), P(ctypes.c_int32), P(ctypes.c_uint32),
                                   P(ctypes.c_int32), P(ctypes.c_int32), P(ctypes.c_int32)]),
        "qvs_state_parity": (I, [I, I, V, V]),
        "qvs_gradient_small_noalloc": (I, [I, I, I, V, P(D), P(D), V, V]),
        "qvs_batch_create": (I, [P(V), I, P(ctypes.c_int32), P(ctypes.c_int32), V]),
        "qvs_batch_set_quality": (I, [V, V, I]),
        "qvs_batch_set_quality_shared": (I, [V, V, I]),
        "qvs_benchmark": (I, [I, V, I, I, I, I, P(D), D, I, P(D), P(D), V]),
        "qvs_batch_optimise": (I, [V, P(D), P(D), D, I, P(D), P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_int)]),
        "qvs_batch_gradient": (I, [V, P(D), P(D), P(D), P(D), P(D)]),
        "qvs_batch_info": (I, [V, P(BatchInfo)]),
        "qvs_batch_set_schedule": (I, [V, I, I]),
        "qvs_batch_destroy": (I, [V]),
        "qvs_strerror": (ctypes.c_char_p, [I]),
        "qvs_set_quality_qubo": (I, [V, I, D, P(D), P(D)]),
        "qvs_quality_qubo": (I, [I, D, P(D), P(D), I, V, V]),
        "qvs_qubo_fixed_point": (I, [I, D, P(D), P(D), P(I), P(ctypes.c_int32), P(ctypes.c_int32), P(ctypes.c_int32)]),
        "qvs_qubo_from_maxcut": (I, [I, I, P(ctypes.c_int32), P(ctypes.c_int32), P(D), P(D), P(D), P(D)]),
        "qvs_set_phase_terms": (I, [V, I, P(ctypes.c_int32), P(ctypes.c_int32), P(D)]),
        "qvs_evolve_ex": (I, [V, I, P(D), P(D)]),
        "qvs_gradient_ex": (I, [V, I, P(D), P(D), P(D), P(D), P(D)]),
        "qvs_bfgs_minimize": (I, [I, P(D), FG_FN, V, D, I, P(D), P(I), P(I), P(I)]),
        "qvs_optimise": (I, [V, I, P(D), P(D), D, I, P(D), P(I), P(I), P(I)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def strerror(status: int) -> str:
    return load().qvs_strerror(status).decode()


def _check(status: int, what: str):
    if status != QVS_OK:
        raise QvsError(status, what)


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ptr_of(x):
    """(pointer, on_device) of a numpy array or a torch tensor."""
    if isinstance(x, np.ndarray):
        return ctypes.c_void_p(x.ctypes.data), 0
    import torch
    if isinstance(x, torch.Tensor):
        return ctypes.c_void_p(x.data_ptr()), 1 if x.is_cuda else 0
    raise TypeError(type(x))


def _check_buffer(x, count: int, dtypes, what: str, device: Optional[bool] = None, exact: bool = False):
    """The library receives bare pointers and reads or writes ``count`` elements: refuse (QVS_EINVAL)
    a buffer that is not contiguous, holds fewer elements (or, with ``exact``, another number), has
    another dtype (names as numpy or torch print them, without the "torch." prefix), or lives on the
    wrong side (``device`` True / False; None: either)."""
    if isinstance(x, np.ndarray):
        n, dt, on_dev, contig = x.size, str(x.dtype), False, x.flags["C_CONTIGUOUS"]
    else:
        import torch
        if not isinstance(x, torch.Tensor):
            raise QvsError(QVS_EINVAL, f"{what}: a numpy array or a torch tensor is required")
        n, dt, on_dev, contig = x.numel(), str(x.dtype).replace("torch.", ""), x.is_cuda, x.is_contiguous()
    if not contig:
        raise QvsError(QVS_EINVAL, f"{what} must be contiguous")
    if device is not None and on_dev != device:
        raise QvsError(QVS_EINVAL, f"{what} must be a {'device tensor' if device else 'host array'}")
    if (n != count) if exact else (n < count):
        raise QvsError(QVS_EINVAL, f"{what} holds {n} values, {count} needed")
    if dt not in dtypes:
        raise QvsError(QVS_EINVAL, f"{what} has dtype {dt}, expected one of {sorted(dtypes)}")


def _quality_dtype(dtype: int) -> str:
    name = {QVS_I32: "int32", QVS_F32: "float32", QVS_F64: "float64"}.get(int(dtype))
    if name is None:
        raise QvsError(QVS_EINVAL, f"unknown quality dtype {dtype}")
    return name


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return ctypes.c_void_p(0)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


# ---------------------------------------------------------------- what the binding knows of a handle
#
# The library takes bare pointers and reads or writes as many elements as the handle's dimension,
# precision, ex-QAOA term count or batch layout says. The wrappers below keep those figures for
# every live handle they created, so that each call can refuse a short or mistyped buffer first.

class _HandleInfo:
    __slots__ = ("dim", "precision", "n_terms")

    def __init__(self, dim: int, precision: int):
        self.dim, self.precision, self.n_terms = int(dim), int(precision), 0

    @property
    def complex_dtype(self) -> str:
        return "complex64" if self.precision == QVS_C64 else "complex128"


_HANDLES: dict = {}   # qvs_create handle address -> _HandleInfo
_BATCHES: dict = {}   # qvs_batch_create handle address -> (qubit counts, layers), int64 arrays


def _addr(h) -> int:
    if isinstance(h, ctypes.c_void_p):
        return int(h.value or 0)
    return int(h or 0)


def _handle_info(h) -> _HandleInfo:
    info = _HANDLES.get(_addr(h))
    if info is None:
        raise QvsError(QVS_EINVAL, "not a live handle of qvs_create")
    return info


def _batch_info(b):
    info = _BATCHES.get(_addr(b))
    if info is None:
        raise QvsError(QVS_EINVAL, "not a live handle of qvs_batch_create")
    return info


def _edges(eu, ev, w):
    """Edge endpoint arrays (int32) and optional weights (fp64) of one length."""
    eu = np.ascontiguousarray(eu, dtype=np.int32).reshape(-1)
    ev = np.ascontiguousarray(ev, dtype=np.int32).reshape(-1)
    if eu.shape != ev.shape:
        raise QvsError(QVS_EINVAL, f"eu ({eu.shape[0]}) and ev ({ev.shape[0]}) differ in length")
    if w is not None:
        w = np.ascontiguousarray(w, dtype=np.float64).reshape(-1)
        if w.shape != eu.shape:
            raise QvsError(QVS_EINVAL, f"w holds {w.shape[0]} weights for {eu.shape[0]} edges")
    return eu, ev, w


# ---------------------------------------------------------------- thin wrappers, same names


class TorchAllocator:
    """Device-memory hooks for qvs_create that take every handle buffer from the PyTorch caching
    allocator on the handle's stream (so library buffers share PyTorch's pool and its stream-ordered
    reuse). Keep the object alive as long as the handle."""

    def __init__(self, stream=None, device=None):
        import torch
        self.device = torch.cuda.current_device() if device is None else int(device)
        self.stream = _stream_ptr(stream).value or 0
        self.live = 0
        self.alloc_fn = ALLOC_FN(self._alloc)
        self.dealloc_fn = DEALLOC_FN(self._dealloc)

    def _alloc(self, nbytes, _ctx):
        import torch
        try:
            ptr = torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream)
        except Exception:          # out of memory (or any failure): the library returns QVS_ENOMEM
            return None
        self.live += 1
        return ptr

    def _dealloc(self, ptr, _ctx):
        import torch
        torch.cuda.caching_allocator_delete(ptr)
        self.live -= 1


def qvs_create(dim: int, precision: int = QVS_C64, stream=None, allocator=None) -> ctypes.c_void_p:
    """allocator: None (the library's cudaMalloc) or an object with ``alloc_fn`` / ``dealloc_fn``
    ctypes callbacks (ALLOC_FN / DEALLOC_FN), e.g. TorchAllocator; the caller keeps it alive."""
    h = ctypes.c_void_p()
    af = allocator.alloc_fn if allocator is not None else ALLOC_FN()
    df = allocator.dealloc_fn if allocator is not None else DEALLOC_FN()
    _check(load().qvs_create(ctypes.byref(h), int(dim), int(precision), _stream_ptr(stream), af, df, None),
           "qvs_create")
    _HANDLES[_addr(h)] = _HandleInfo(dim, precision)
    return h


def qvs_destroy(h):
    _check(load().qvs_destroy(h), "qvs_destroy")
    _HANDLES.pop(_addr(h), None)


def qvs_set_quality(h, q, dtype: Optional[int] = None):
    """q: dim values (host array or device tensor) of type dtype (None: taken from q's dtype)."""
    info = _handle_info(h)
    if dtype is None:
        dt = str(getattr(q, "dtype", "")).replace("torch.", "")
        dtype = {"int32": QVS_I32, "float32": QVS_F32, "float64": QVS_F64}.get(dt)
        if dtype is None:
            raise QvsError(QVS_EINVAL, f"quality vector has dtype {dt or type(q).__name__}")
    _check_buffer(q, info.dim, {_quality_dtype(dtype)}, "quality vector", exact=True)
    p, dev = _ptr_of(q)
    _check(load().qvs_set_quality(h, p, int(dtype), dev), "qvs_set_quality")


def qvs_set_mixer(h, kind: int, desc: MixerDesc):
    _check(load().qvs_set_mixer(h, int(kind), ctypes.byref(desc)), "qvs_set_mixer")


def qvs_set_initial_state(h, psi0=None):
    """psi0 None: the equal superposition (QVS_INIT_UNIFORM); else the explicit state (host array or
    device tensor of dim complex values in the handle's precision)."""
    info = _handle_info(h)
    if psi0 is None:
        _check(load().qvs_set_initial_state(h, QVS_INIT_UNIFORM, None, 0), "qvs_set_initial_state")
        return
    _check_buffer(psi0, info.dim, {info.complex_dtype}, "initial state", exact=True)
    p, dev = _ptr_of(psi0)
    _check(load().qvs_set_initial_state(h, QVS_INIT_EXPLICIT, p, dev), "qvs_set_initial_state")


def qvs_set_option(h, option: int, value: int):
    _check(load().qvs_set_option(h, int(option), int(value)), "qvs_set_option")


def _params(gammas, ts):
    g = np.ascontiguousarray(gammas, dtype=np.float64).reshape(-1)
    t = np.ascontiguousarray(ts, dtype=np.float64).reshape(-1)
    if g.shape != t.shape:
        raise QvsError(QVS_EINVAL, f"gammas ({g.shape[0]}) and ts ({t.shape[0]}) differ in length")
    return g, t


def qvs_evolve(h, gammas, ts):
    g, t = _params(gammas, ts)
    _check(load().qvs_evolve(h, len(g), _dptr(g), _dptr(t)), "qvs_evolve")


def qvs_expectation(h) -> float:
    e = ctypes.c_double()
    _check(load().qvs_expectation(h, ctypes.byref(e)), "qvs_expectation")
    return e.value


def qvs_gradient(h, gammas, ts):
    """Returns (E, dgamma[p], dt[p])."""
    g, t = _params(gammas, ts)
    p = len(g)
    e = ctypes.c_double()
    dg = np.zeros(p)
    dt = np.zeros(p)
    _check(load().qvs_gradient(h, p, _dptr(g), _dptr(t), ctypes.byref(e), _dptr(dg), _dptr(dt)),
           "qvs_gradient")
    return e.value, dg, dt


def qvs_get_state(h, out):
    """Copy the state (dim complex values in the handle's precision) into out (host or device)."""
    info = _handle_info(h)
    _check_buffer(out, info.dim, {info.complex_dtype}, "state output")
    p, dev = _ptr_of(out)
    _check(load().qvs_get_state(h, p, dev), "qvs_get_state")
    return out


def qvs_last_launch_count(h) -> int:
    c = ctypes.c_int64()
    _check(load().qvs_last_launch_count(h, ctypes.byref(c)), "qvs_last_launch_count")
    return c.value


def qvs_kernel_stats(h):
    """List of dicts {name, launches, ms, bytes} gathered while QVS_OPT_PROFILE is on."""
    out = []
    lib = load()
    slot = 0
    while True:
        name = ctypes.create_string_buffer(128)
        n = ctypes.c_int64()
        ms = ctypes.c_double()
        by = ctypes.c_double()
        if lib.qvs_kernel_stats(h, slot, name, 128, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by)) != QVS_OK:
            break
        out.append({"name": name.value.decode(), "launches": n.value, "ms": ms.value, "bytes": by.value})
        slot += 1
    return out


def qvs_quality_maxcut(n: int, eu, ev, w, out, dtype: int, stream=None):
    eu, ev, w = _edges(eu, ev, w)
    wp = None if w is None else _dptr(w)
    _check_buffer(out, 1 << int(n), {_quality_dtype(dtype)}, "quality output", device=True)
    p, dev = _ptr_of(out)
    _check(load().qvs_quality_maxcut(n, len(eu), eu.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                     ev.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), wp, int(dtype), p,
                                     _stream_ptr(stream)), "qvs_quality_maxcut")
    return out


def _qubo_arrays(n, hlin, J):
    hl = np.ascontiguousarray(hlin, dtype=np.float64).reshape(-1)
    Jm = np.ascontiguousarray(J, dtype=np.float64).reshape(-1)
    if hl.shape[0] != int(n) or Jm.shape[0] != int(n) * int(n):
        raise QvsError(QVS_EINVAL, f"a quadratic form on {int(n)} qubits needs {int(n)} linear and "
                                   f"{int(n)} x {int(n)} pair coefficients")
    return hl, Jm


def qvs_set_quality_qubo(h, n_qubits: int, c: float, hlin, J):
    hl, Jm = _qubo_arrays(n_qubits, hlin, J)
    _check(load().qvs_set_quality_qubo(h, int(n_qubits), float(c), _dptr(hl), _dptr(Jm)), "qvs_set_quality_qubo")


def qvs_quality_qubo(n_qubits: int, c: float, hlin, J, out, dtype: int, stream=None):
    hl, Jm = _qubo_arrays(n_qubits, hlin, J)
    _check_buffer(out, 1 << int(n_qubits), {_quality_dtype(dtype)}, "quality output", device=True)
    p, dev = _ptr_of(out)
    _check(load().qvs_quality_qubo(int(n_qubits), float(c), _dptr(hl), _dptr(Jm), int(dtype), p,
                                   _stream_ptr(stream)), "qvs_quality_qubo")
    return out


def qvs_qubo_fixed_point(n_qubits: int, c: float, hlin, J):
    """(F, ci, hi[n], Ji[n, n]) of the quadratic form's fixed-point coefficients (host, no GPU)."""
    n = int(n_qubits)
    hl, Jm = _qubo_arrays(n, hlin, J)
    F, ci = ctypes.c_int(), ctypes.c_int32()
    hi = np.zeros(n, dtype=np.int32)
    Ji = np.zeros(n * n, dtype=np.int32)
    I32 = ctypes.POINTER(ctypes.c_int32)
    _check(load().qvs_qubo_fixed_point(n, float(c), _dptr(hl), _dptr(Jm), ctypes.byref(F), ctypes.byref(ci),
                                       hi.ctypes.data_as(I32), Ji.ctypes.data_as(I32)), "qvs_qubo_fixed_point")
    return F.value, ci.value, hi, Ji.reshape(n, n)


def qvs_qubo_from_maxcut(n: int, eu, ev, w=None):
    """(c, hlin[n], J[n, n]) of the max-cut cost (host, no GPU needed)."""
    eu, ev, w = _edges(eu, ev, w)
    wp = None if w is None else _dptr(w)
    c = ctypes.c_double()
    hl = np.zeros(n, dtype=np.float64)
    J = np.zeros(n * n, dtype=np.float64)
    _check(load().qvs_qubo_from_maxcut(n, len(eu), eu.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                       ev.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), wp, ctypes.byref(c),
                                       _dptr(hl), _dptr(J)), "qvs_qubo_from_maxcut")
    return c.value, hl, J.reshape(n, n)


def qvs_set_phase_terms(h, u, v, coef):
    """ex-QAOA terms coef[j] Z_u[j] Z_v[j] (v[j] = -1: a single Z)."""
    info = _handle_info(h)
    u = np.ascontiguousarray(u, dtype=np.int32).reshape(-1)
    v = np.ascontiguousarray(v, dtype=np.int32).reshape(-1)
    c = np.ascontiguousarray(coef, dtype=np.float64).reshape(-1)
    if not u.shape == v.shape == c.shape:
        raise QvsError(QVS_EINVAL, f"u, v and coef differ in length ({u.shape[0]}, {v.shape[0]}, {c.shape[0]})")
    _check(load().qvs_set_phase_terms(h, len(c), u.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                      v.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dptr(c)),
           "qvs_set_phase_terms")
    info.n_terms = int(c.shape[0])


def _ex_params(h, gammas, ts):
    """gammas (p x n_terms values, layer-major) and ts (p values) for the handle's ex-QAOA terms."""
    info = _handle_info(h)
    G = np.ascontiguousarray(gammas, dtype=np.float64)
    t = np.ascontiguousarray(ts, dtype=np.float64).reshape(-1)
    if info.n_terms > 0 and G.size != t.shape[0] * info.n_terms:
        raise QvsError(QVS_EINVAL, f"gammas hold {G.size} values, {t.shape[0]} x {info.n_terms} needed")
    return G, t


def qvs_evolve_ex(h, gammas, ts) -> float:
    """gammas: (p, n_terms) array; returns the objective."""
    G, t = _ex_params(h, gammas, ts)
    _check(load().qvs_evolve_ex(h, len(t), _dptr(G), _dptr(t)), "qvs_evolve_ex")
    E = ctypes.c_double()
    _check(load().qvs_expectation(h, ctypes.byref(E)), "qvs_expectation")
    return E.value


def qvs_gradient_ex(h, gammas, ts):
    """gammas: (p, n_terms) array; returns (E, dgamma (p, n_terms), dt (p,))."""
    G, t = _ex_params(h, gammas, ts)
    p = len(t)
    E = ctypes.c_double()
    dG = np.zeros(G.shape, dtype=np.float64)
    dt = np.zeros(p, dtype=np.float64)
    _check(load().qvs_gradient_ex(h, p, _dptr(G), _dptr(t), ctypes.byref(E), _dptr(dG), _dptr(dt)), "qvs_gradient_ex")
    return E.value, dG, dt


def qvs_bfgs_minimize(fg, x0, gtol: float = 1e-8, max_iter: int = 1000):
    """BFGS on the host with a Python objective: fg(x) -> (f, g). Returns (x, f, iterations,
    evaluations, stop) with stop 0 = gradient below gtol, 1 = max_iter reached, 2 = line search
    could not decrease f (precision loss)."""
    x = np.ascontiguousarray(x0, dtype=np.float64).copy()
    n = x.shape[0]
    err = []

    def cb(xp, fp, gp, _user):
        try:
            xv = np.ctypeslib.as_array(xp, shape=(n,)).copy()
            f, g = fg(xv)
            fp[0] = float(f)
            gv = np.asarray(g, dtype=np.float64)
            for i in range(n):
                gp[i] = float(gv[i])
            return QVS_OK
        except Exception as e:   # reported after the call; a non-zero status stops the loop
            err.append(e)
            return -1
    cfn = FG_FN(cb)
    f = ctypes.c_double()
    it = ctypes.c_int()
    ev = ctypes.c_int()
    stop = ctypes.c_int()
    st = load().qvs_bfgs_minimize(n, _dptr(x), cfn, None, float(gtol), int(max_iter), ctypes.byref(f),
                                  ctypes.byref(it), ctypes.byref(ev), ctypes.byref(stop))
    if err:
        raise err[0]
    _check(st, "qvs_bfgs_minimize")
    return x, f.value, it.value, ev.value, stop.value


def qvs_optimise(h, gammas0, ts0, gtol: float = 1e-6, max_iter: int = 200):
    """BFGS over theta = (gamma_1, t_1, ...) with the device gradient. Returns
    (gammas, ts, f, iterations, evaluations, stop)."""
    g = np.ascontiguousarray(gammas0, dtype=np.float64).copy()
    t = np.ascontiguousarray(ts0, dtype=np.float64).copy()
    f = ctypes.c_double()
    it = ctypes.c_int()
    ev = ctypes.c_int()
    stop = ctypes.c_int()
    _check(load().qvs_optimise(h, len(g), _dptr(g), _dptr(t), float(gtol), int(max_iter), ctypes.byref(f),
                               ctypes.byref(it), ctypes.byref(ev), ctypes.byref(stop)), "qvs_optimise")
    return g, t, f.value, it.value, ev.value, stop.value


def qvs_quality_subset(n: int, w, out, dtype: int, stream=None):
    w = np.ascontiguousarray(w, dtype=np.float64).reshape(-1)
    if w.shape[0] != int(n):
        raise QvsError(QVS_EINVAL, f"{w.shape[0]} item weights for {int(n)} qubits")
    _check_buffer(out, 1 << int(n), {_quality_dtype(dtype)}, "quality output", device=True)
    p, dev = _ptr_of(out)
    _check(load().qvs_quality_subset(n, _dptr(w), int(dtype), p, _stream_ptr(stream)), "qvs_quality_subset")
    return out


def qvs_quality_portfolio(n_qubits: int, states_dev, returns, cov, omega: float, out, dtype: int, stream=None):
    r = np.ascontiguousarray(returns, dtype=np.float64).reshape(-1)
    c = np.ascontiguousarray(cov, dtype=np.float64)
    M = int(n_qubits) // 2           # the library reads M returns and the M x M covariance, row-major
    if r.shape[0] != M or c.size != M * M:
        raise QvsError(QVS_EINVAL, f"{M} assets need {M} returns and an {M} x {M} covariance")
    dim = int(states_dev.shape[0])
    _check_buffer(states_dev, dim, {"int64"}, "states", device=True)
    _check_buffer(out, dim, {_quality_dtype(dtype)}, "quality output", device=True)
    sp, sdev = _ptr_of(states_dev)
    op, odev = _ptr_of(out)
    _check(load().qvs_quality_portfolio(n_qubits, dim, sp, _dptr(r), _dptr(c), float(omega), int(dtype), op,
                                        _stream_ptr(stream)), "qvs_quality_portfolio")
    return out


def qvs_state_parity(n_qubits: int, A: int, out, stream=None):
    """The QAOAz parity initial state written into the complex64 device tensor ``out``."""
    _check_buffer(out, 1 << int(n_qubits), {"complex64"}, "parity state output", device=True)
    op, odev = _ptr_of(out)
    _check(load().qvs_state_parity(int(n_qubits), int(A), op, _stream_ptr(stream)), "qvs_state_parity")
    return out


def qvs_chebyshev_coefficients(a: float, b: float, t: float, tol: float, max_terms: int = 20000):
    """(c[K + 1] complex, tail bound) of exp(-i t W) = sum_m c_m T_m((W - a) / b) (host, no GPU)."""
    n = ctypes.c_int()
    tail = ctypes.c_double()
    _check(load().qvs_chebyshev_coefficients(float(a), float(b), float(t), float(tol), int(max_terms), None,
                                             ctypes.byref(n), ctypes.byref(tail)), "qvs_chebyshev_coefficients")
    c = np.zeros(2 * n.value, dtype=np.float64)
    _check(load().qvs_chebyshev_coefficients(float(a), float(b), float(t), float(tol), int(max_terms), _dptr(c),
                                             ctypes.byref(n), ctypes.byref(tail)), "qvs_chebyshev_coefficients")
    return c[0::2] + 1j * c[1::2], tail.value


def qvs_hypercube_plan(n_qubits: int, p: int):
    """The hypercube mixer's forward pass schedule (host, no GPU): a list of dicts per pass with its
    shape, tile type, rotated index bits (a mask) and the layers of its rotations and phase."""
    m = ctypes.c_int()
    _check(load().qvs_hypercube_plan(int(n_qubits), int(p), 0, ctypes.byref(m), None, None, None, None, None, None),
           "qvs_hypercube_plan")
    F = m.value
    shape, typ, lb, la, lg = (np.zeros(F, np.int32) for _ in range(5))
    bits = np.zeros(F, np.uint32)
    I32, U32 = ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_uint32)
    _check(load().qvs_hypercube_plan(int(n_qubits), int(p), F, ctypes.byref(m), shape.ctypes.data_as(I32),
                                     typ.ctypes.data_as(I32), bits.ctypes.data_as(U32), lb.ctypes.data_as(I32),
                                     la.ctypes.data_as(I32), lg.ctypes.data_as(I32)), "qvs_hypercube_plan")
    return [{"shape": int(shape[j]), "type": int(typ[j]), "bits": int(bits[j]), "before": int(lb[j]),
             "after": int(la[j]), "phase": int(lg[j])} for j in range(F)]


QVS_LAYOUT_HYPERCUBE, QVS_LAYOUT_CIRCULANT_COLUMN, QVS_LAYOUT_CIRCULANT_ROW, QVS_LAYOUT_CIRCULANT_BOX = 1, 2, 3, 4


def qvs_tile_layout(family: int, log2n: int, layout: int):
    """A tiled kernel's register layout (host, no GPU): (index[threads, regs], slot[tile], global[tile],
    column_bits) -- the tile index of each thread register, the shared-memory slot and the
    state-vector offset (first tile) of each tile index."""
    I32 = ctypes.POINTER(ctypes.c_int32)
    index = np.zeros(512 * 32, np.int32)
    slot = np.zeros(1 << 14, np.int32)
    glob = np.zeros(1 << 14, np.int32)
    th, rg, cb = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().qvs_tile_layout(int(family), int(log2n), int(layout), index.ctypes.data_as(I32),
                                  slot.ctypes.data_as(I32), glob.ctypes.data_as(I32), ctypes.byref(th),
                                  ctypes.byref(rg), ctypes.byref(cb)), "qvs_tile_layout")
    tile = th.value * rg.value
    return index[:tile].reshape(th.value, rg.value), slot[:tile], glob[:tile], cb.value


PARITY_TILE_BITS, PARITY_MAX_GATES = 12, 40


def qvs_parity_plan(n_qubits: int):
    """The parity-ring mixer's passes for one layer (host, no GPU): a list of dicts with the tile's
    index bits, the gates as index-bit pairs in order, and the sweeps as (kind, first gate)."""
    n = int(n_qubits)
    npass = ctypes.c_int()
    _check(load().qvs_parity_plan(n, 0, ctypes.byref(npass), None, None, None, None, None, None), "qvs_parity_plan")
    m = npass.value
    T, G = PARITY_TILE_BITS, PARITY_MAX_GATES
    ng, ns = np.zeros(m, np.int32), np.zeros(m, np.int32)
    tb, gb = np.zeros(m * T, np.int32), np.zeros(m * G * 2, np.int32)
    sk, sf = np.zeros(m * G, np.int32), np.zeros(m * G, np.int32)
    I32 = ctypes.POINTER(ctypes.c_int32)
    _check(load().qvs_parity_plan(n, m, ctypes.byref(npass), *(a.ctypes.data_as(I32) for a in (ng, tb, gb, ns, sk, sf))),
           "qvs_parity_plan")
    out = []
    for i in range(m):
        g = gb[i * G * 2:(i + 1) * G * 2].reshape(G, 2)[:ng[i]]
        out.append({"tile": tb[i * T:(i + 1) * T].tolist(), "gates": [tuple(x) for x in g.tolist()],
                    "sweeps": list(zip(sk[i * G:i * G + ns[i]].tolist(), sf[i * G:i * G + ns[i]].tolist()))})
    return out


def qvs_xy_ring_csr(n: int, k: int):
    """Returns (states int64[dim], rowptr int64[dim+1], colind int32[nnz]) as numpy arrays."""
    lib = load()
    dim = ctypes.c_int64()
    nnz = ctypes.c_int64()
    _check(lib.qvs_xy_ring_csr(n, k, None, None, None, ctypes.byref(dim), ctypes.byref(nnz)), "qvs_xy_ring_csr")
    states = np.zeros(dim.value, dtype=np.int64)
    rowptr = np.zeros(dim.value + 1, dtype=np.int64)
    colind = np.zeros(nnz.value, dtype=np.int32)
    _check(lib.qvs_xy_ring_csr(n, k, ctypes.c_void_p(states.ctypes.data), ctypes.c_void_p(rowptr.ctypes.data),
                               ctypes.c_void_p(colind.ctypes.data), ctypes.byref(dim), ctypes.byref(nnz)),
           "qvs_xy_ring_csr")
    return states, rowptr, colind


def qvs_gradient_small_noalloc(n: int, precision: int, q_dev, gammas, ts, out_dev, stream=None):
    """Allocation-free small-state solve (n <= 12): writes E, dgamma[p], dt[p] into the device
    tensor out_dev (1 + 2p float64) on the stream; see include/qvs.h for the limits. The sizes and
    dtypes of q_dev and out_dev are checked here, since the library receives bare pointers."""
    import torch
    g, t = _params(gammas, ts)
    p = g.shape[0]
    want = torch.float32 if precision == QVS_C64 else torch.float64
    for name, x in (("q", q_dev), ("out", out_dev)):
        if not (isinstance(x, torch.Tensor) and x.is_cuda and x.is_contiguous()):
            raise QvsError(QVS_EINVAL, f"{name} must be a contiguous CUDA tensor")
    if not 1 <= int(n) <= 30 or q_dev.dtype != want or q_dev.numel() != (1 << int(n)):
        raise QvsError(QVS_EINVAL, f"q must hold 2^n {want} values")
    if out_dev.dtype != torch.float64 or out_dev.numel() < 1 + 2 * p:
        raise QvsError(QVS_EINVAL, "out must hold at least 1 + 2p float64 values")
    qp, _ = _ptr_of(q_dev)
    op, _ = _ptr_of(out_dev)
    _check(load().qvs_gradient_small_noalloc(int(n), int(precision), p, qp, _dptr(g), _dptr(t), op,
                                             _stream_ptr(stream)), "qvs_gradient_small_noalloc")
    return out_dev


def qvs_batch_create(n_qubits, layers, stream=None):
    ns = np.ascontiguousarray(n_qubits, dtype=np.int32).reshape(-1)
    ps = np.ascontiguousarray(layers, dtype=np.int32).reshape(-1)
    h = ctypes.c_void_p()
    if ns.shape != ps.shape:
        raise QvsError(QVS_EINVAL, f"n_qubits ({ns.shape[0]}) and layers ({ps.shape[0]}) differ in length")
    _check(load().qvs_batch_create(ctypes.byref(h), len(ns), ns.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   ps.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _stream_ptr(stream)),
           "qvs_batch_create")
    _BATCHES[_addr(h)] = (ns.astype(np.int64), ps.astype(np.int64))
    return h


def qvs_batch_set_quality(b, q):
    """The instances' fp32 qualities concatenated in instance order (host or device)."""
    ns, _ = _batch_info(b)
    _check_buffer(q, int(np.sum(np.int64(1) << ns)), {"float32"}, "concatenated qualities", exact=True)
    p, dev = _ptr_of(q)
    _check(load().qvs_batch_set_quality(b, p, dev), "qvs_batch_set_quality")


def qvs_batch_set_quality_shared(b, q):
    """One quality vector (2^n fp32 values) read by every instance of the batch (all of one n)."""
    ns, _ = _batch_info(b)
    _check_buffer(q, 1 << int(ns.max()), {"float32"}, "shared quality vector", exact=True)
    p, dev = _ptr_of(q)
    _check(load().qvs_batch_set_quality_shared(b, p, dev), "qvs_batch_set_quality_shared")


def _batch_params(b, gammas, ts, count: int):
    """Concatenated per-instance parameters: sum of the instances' layers each, count instances."""
    ns, ps = _batch_info(b)
    g, t = _params(gammas, ts)
    if int(count) != ns.shape[0] or g.shape[0] != int(ps.sum()):
        raise QvsError(QVS_EINVAL, f"{g.shape[0]} parameters for {int(count)} instances; the batch has "
                                   f"{ns.shape[0]} instances and {int(ps.sum())} layers")
    return g, t


def qvs_batch_optimise(b, gammas, ts, count: int, gtol: float = 1e-6, max_iter: int = 200):
    """Device BFGS of every instance at once. gammas, ts: concatenated start points. Returns
    (gammas, ts, f[count], iterations[count], evaluations[count], stop[count])."""
    g, t = _batch_params(b, gammas, ts, count)
    g, t = g.copy(), t.copy()
    f = np.zeros(count)
    it = np.zeros(count, dtype=np.int32)
    ev = np.zeros(count, dtype=np.int32)
    stop = np.zeros(count, dtype=np.int32)
    IP = ctypes.POINTER(ctypes.c_int)
    _check(load().qvs_batch_optimise(b, _dptr(g), _dptr(t), float(gtol), int(max_iter), _dptr(f),
                                     it.ctypes.data_as(IP), ev.ctypes.data_as(IP), stop.ctypes.data_as(IP)),
           "qvs_batch_optimise")
    return g, t, f, it, ev, stop


def qvs_benchmark(n: int, q, d_min: int, d_max: int, repeats: int, init, gtol: float = 1e-6, max_iter: int = 200,
                  stream=None):
    """Depth sweep with persisted parameters (see include/qvs.h). init: the start values (repeats x
    2 d_min for the first depth, then repeats x 2 per later depth). Returns (f[depth][repeat],
    list of best (gammas, ts) per depth)."""
    nd = d_max - d_min + 1
    need = repeats * 2 * d_min + repeats * 2 * (nd - 1)
    x0 = np.ascontiguousarray(init, dtype=np.float64).reshape(-1)
    if x0.shape[0] != need:
        raise QvsError(QVS_EINVAL, f"init needs {need} values")
    f = np.zeros(nd * repeats)
    best = np.zeros(sum(2 * D for D in range(d_min, d_max + 1)))
    _check_buffer(q, 1 << int(n), {"float32"}, "quality vector", exact=True)
    qp, dev = _ptr_of(q)
    _check(load().qvs_benchmark(int(n), qp, dev, int(d_min), int(d_max), int(repeats), _dptr(x0), float(gtol),
                                int(max_iter), _dptr(f), _dptr(best), _stream_ptr(stream)), "qvs_benchmark")
    out, o = [], 0
    for D in range(d_min, d_max + 1):
        out.append((best[o:o + D].copy(), best[o + D:o + 2 * D].copy()))
        o += 2 * D
    return f.reshape(nd, repeats), out


def qvs_batch_gradient(b, gammas, ts, count: int):
    """gammas, ts: concatenated per-instance parameters. Returns (E[count], dgamma, dt) concatenated."""
    g, t = _batch_params(b, gammas, ts, count)
    E = np.zeros(count)
    dg = np.zeros(len(g))
    dt = np.zeros(len(g))
    _check(load().qvs_batch_gradient(b, _dptr(g), _dptr(t), _dptr(E), _dptr(dg), _dptr(dt)), "qvs_batch_gradient")
    return E, dg, dt


def qvs_batch_info(b):
    info = BatchInfo()
    _check(load().qvs_batch_info(b, ctypes.byref(info)), "qvs_batch_info")
    return {"ctas_per_sm": info.ctas_per_sm, "trial_ms": [info.trial_ms[0], info.trial_ms[1]],
            "bytes_per_solve": info.bytes_per_solve, "fma_per_solve": info.fma_per_solve,
            "amp_layers": info.amp_layers, "shared_quality": bool(info.shared_quality),
            "ckpt_policy": info.ckpt_policy, "from_cache": bool(info.from_cache),
            "trial_ms_all": [info.trial_ms_all[k] for k in range(4)]}


def qvs_batch_set_schedule(b, ctas_per_sm: int, ckpt_policy: int):
    _check(load().qvs_batch_set_schedule(b, int(ctas_per_sm), int(ckpt_policy)), "qvs_batch_set_schedule")


def qvs_batch_destroy(b):
    _check(load().qvs_batch_destroy(b), "qvs_batch_destroy")
    _BATCHES.pop(_addr(b), None)


class Batch:
    """Many QAOA hypercube instances (n >= 12) solved by one persistent launch."""

    def __init__(self, n_qubits, layers, stream=None):
        self.ns = np.asarray(n_qubits, dtype=np.int64)
        self.ps = np.asarray(layers, dtype=np.int64)
        self.qoff = np.concatenate([[0], np.cumsum(1 << self.ns)])
        self.poff = np.concatenate([[0], np.cumsum(self.ps)])
        self.h = qvs_batch_create(self.ns, self.ps, stream)

    def close(self):
        if self.h is not None:
            qvs_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_quality(self, q_concat):
        _check_buffer(q_concat, int(self.qoff[-1]), {"float32"}, "concatenated qualities", exact=True)
        qvs_batch_set_quality(self.h, q_concat)
        return self

    def _per_instance(self, gammas_list, ts_list):
        """Per-instance parameter arrays, one of each instance's depth, concatenated."""
        lg = np.fromiter(map(len, gammas_list), dtype=np.int64, count=len(gammas_list))
        lt = np.fromiter(map(len, ts_list), dtype=np.int64, count=len(ts_list))
        if lg.shape != self.ps.shape or lt.shape != self.ps.shape or np.any(lg != self.ps) or np.any(lt != self.ps):
            raise QvsError(QVS_EINVAL, "one gamma and one t array per instance, of that instance's depth")
        return np.concatenate(gammas_list), np.concatenate(ts_list)

    def gradient(self, gammas_list, ts_list):
        """Lists of per-instance parameter arrays -> (E array, list of dgamma, list of dt)."""
        E, dg, dt = qvs_batch_gradient(self.h, *self._per_instance(gammas_list, ts_list), len(self.ns))
        cut = lambda v: [v[self.poff[i]:self.poff[i + 1]] for i in range(len(self.ns))]
        return E, cut(dg), cut(dt)

    def set_quality_shared(self, q):
        _check_buffer(q, 1 << int(self.ns.max()), {"float32"}, "shared quality vector", exact=True)
        qvs_batch_set_quality_shared(self.h, q)
        return self

    def optimise(self, gammas_list, ts_list, gtol: float = 1e-6, max_iter: int = 200):
        """Lists of per-instance start points -> (list of gammas, list of ts, f, iterations,
        evaluations, stop), per instance."""
        g, t, f, it, ev, stop = qvs_batch_optimise(self.h, *self._per_instance(gammas_list, ts_list), len(self.ns),
                                                   gtol, max_iter)
        cut = lambda v: [v[self.poff[i]:self.poff[i + 1]] for i in range(len(self.ns))]
        return cut(g), cut(t), f, it, ev, stop

    def set_schedule(self, ctas_per_sm: int, ckpt_policy: int):
        qvs_batch_set_schedule(self.h, ctas_per_sm, ckpt_policy)
        return self

    def info(self):
        return qvs_batch_info(self.h)


def qvs_strerror(status: int) -> str:
    return strerror(status)


# ---------------------------------------------------------------- convenience layer


def parity_desc(n: int) -> MixerDesc:
    d = MixerDesc()
    d.n_qubits = n
    return d


def xy_ring_desc(n: int, k: int, spec=(0.0, 0.0), tol: float = 0.0) -> MixerDesc:
    """The XY ring on the Hamming-weight-k states of n qubits, applied without a stored matrix."""
    d = MixerDesc()
    d.n_qubits = n
    d.hamming_weight = k
    d.spec_lo, d.spec_hi = spec
    d.cheb_tol = tol
    return d


def hypercube_desc(n: int) -> MixerDesc:
    d = MixerDesc()
    d.n_qubits = n
    return d


def circulant_desc(offsets, weights=None) -> MixerDesc:
    """Connection offsets and (optionally) one weight per offset; the library reads n_offsets of
    each, so the two arrays must have one length."""
    d = MixerDesc()
    off = np.ascontiguousarray(offsets, dtype=np.int64).reshape(-1)
    d.n_offsets = len(off)
    d._off = off   # keep alive
    d.offsets = off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    if weights is not None:
        w = np.ascontiguousarray(weights, dtype=np.float64).reshape(-1)
        if w.shape != off.shape:
            raise QvsError(QVS_EINVAL, f"{w.shape[0]} weights for {off.shape[0]} offsets")
        d._w = w
        d.offset_weights = w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return d


def csr_desc(rowptr, colind, values=None, implicit_value: float = 1.0, spec=(0.0, 0.0), tol: float = 0.0) -> MixerDesc:
    d = MixerDesc()
    rp, dev1 = _ptr_of(rowptr)
    ci, dev2 = _ptr_of(colind)
    if dev1 != dev2:
        raise QvsError(QVS_EINVAL, "rowptr and colind must both be host arrays or both device tensors")
    nnz = int(colind.shape[0])
    _check_buffer(rowptr, int(rowptr.shape[0]), {"int64"}, "rowptr")
    _check_buffer(colind, nnz, {"int32"}, "colind")
    if values is not None:
        _check_buffer(values, nnz, {"float32"}, "values", device=bool(dev1), exact=True)
    d._keep = (rowptr, colind, values)
    d.rowptr = rp.value
    d.colind = ci.value
    if values is not None:
        vp, _ = _ptr_of(values)
        d.values = vp.value
    d.implicit_value = implicit_value
    d.nnz = int(colind.shape[0])
    d.csr_on_device = dev1
    d.spec_lo, d.spec_hi = spec
    d.cheb_tol = tol
    return d


class Simulator:
    """Owns one qvs handle: quality vector + mixer + optional initial state."""

    def __init__(self, dim: int, precision: int = QVS_C64, stream=None, allocator="torch"):
        """allocator: "torch" (default: device buffers from the PyTorch caching allocator on the
        handle's stream), None (the library's cudaMalloc) or a hooks object (see qvs_create)."""
        self.dim = int(dim)
        self.precision = precision
        self.h = None
        if allocator == "torch":
            allocator = TorchAllocator(stream)
        self.allocator = allocator
        self.h = qvs_create(dim, precision, stream, allocator)

    def close(self):
        if self.h is not None:
            qvs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_quality(self, q, dtype=None):
        _check_buffer(q, self.dim, {"int32", "float32", "float64"}, "quality vector", exact=True)
        qvs_set_quality(self.h, q, dtype)
        return self

    def set_quality_qubo(self, n_qubits: int, c: float, hlin, J):
        qvs_set_quality_qubo(self.h, n_qubits, c, hlin, J)
        return self

    def set_phase_terms(self, u, v, coef):
        qvs_set_phase_terms(self.h, u, v, coef)
        return self

    def optimise(self, gammas0, ts0, gtol: float = 1e-6, max_iter: int = 200):
        return qvs_optimise(self.h, gammas0, ts0, gtol, max_iter)

    def evolve_ex(self, gammas, ts) -> float:
        return qvs_evolve_ex(self.h, gammas, ts)

    def gradient_ex(self, gammas, ts):
        return qvs_gradient_ex(self.h, gammas, ts)

    def set_mixer(self, kind: int, desc: MixerDesc):
        if int(kind) == QVS_MIX_CSR:   # the library copies dim + 1 row pointers
            rowptr = desc._keep[0]
            if int(rowptr.shape[0]) != self.dim + 1:
                raise QvsError(QVS_EINVAL, f"rowptr holds {int(rowptr.shape[0])} entries, {self.dim + 1} needed")
        qvs_set_mixer(self.h, kind, desc)
        return self

    def set_initial_state(self, psi0=None):
        if psi0 is not None:
            want = "complex64" if self.precision == QVS_C64 else "complex128"
            _check_buffer(psi0, self.dim, {want}, "initial state", exact=True)
        qvs_set_initial_state(self.h, psi0)
        return self

    def set_option(self, option, value):
        qvs_set_option(self.h, option, value)
        return self

    def evolve(self, gammas, ts) -> float:
        qvs_evolve(self.h, gammas, ts)
        return qvs_expectation(self.h)

    def gradient(self, gammas, ts):
        return qvs_gradient(self.h, gammas, ts)

    def state(self) -> np.ndarray:
        out = np.zeros(self.dim, dtype=np.complex64 if self.precision == QVS_C64 else np.complex128)
        qvs_get_state(self.h, out)
        return out

    def launches(self) -> int:
        return qvs_last_launch_count(self.h)


class QAOAObjective:
    """The objective E(gammas, ts) = <theta|Q|theta> of a Simulator as a differentiable PyTorch
    function: the forward pass runs the device solve (qvs_gradient: forward sweep, objective and
    adjoint sweep), the backward pass returns grad_out * (dE/dgamma, dE/dt) from that same solve,
    in the dtype and on the device of the inputs."""

    @staticmethod
    def function(sim: Simulator):
        import torch

        class _Evolve(torch.autograd.Function):
            @staticmethod
            def forward(ctx, gammas, ts):
                E, dg, dt = sim.gradient(gammas.detach().cpu().double().numpy(),
                                         ts.detach().cpu().double().numpy())
                ctx.save_for_backward(torch.from_numpy(dg).to(gammas.device, gammas.dtype),
                                      torch.from_numpy(dt).to(ts.device, ts.dtype))
                return torch.tensor(E, dtype=torch.float64, device=gammas.device)

            @staticmethod
            def backward(ctx, grad_out):
                dg, dt = ctx.saved_tensors
                return grad_out.to(dg.dtype) * dg, grad_out.to(dt.dtype) * dt

        return _Evolve.apply
