"""Shared helpers for the GPU tests (import only from tests marked gpu)."""
from __future__ import annotations

import numpy as np

TOL_E = 1e-5        # |dE| / |E| for complex64 results (target tolerance of the hot path)
TOL_G = 1e-4        # max_k |g_k - g_ref_k| / max_k |g_ref_k|
TOL_E_C128 = 1e-12  # complex128 path


def rel_err_E(E, ref):
    return abs(E - ref) / max(abs(ref), 1e-30)


def rel_err_grad(dg, dt, rdg, rdt):
    g = np.concatenate([dg, dt])
    r = np.concatenate([rdg, rdt])
    return float(np.max(np.abs(g - r)) / max(np.max(np.abs(r)), 1e-30))


def infidelity(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return 1.0 - abs(np.vdot(a, b)) / (np.linalg.norm(a) * np.linalg.norm(b))


def lib():
    import paper_2110_03963_gb300 as qvs
    from paper_2110_03963_gb300 import _build
    _build.build()
    qvs.load()
    return qvs
