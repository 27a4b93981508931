"""Seeded synthetic problem instances shared by the oracle tests, the GPU tests and the bench.

This module holds only random instance data (graphs, weights, item values, returns and
covariances, variational parameters) drawn from seeded numpy generators. It contains none of the
simulation arithmetic: quality vectors, mixers, phases, expectations and gradients are computed
separately by ``oracle/`` (fp64 CPU) and by the CUDA library, from these raw inputs.

Instance shapes follow the workloads the paper simulates (Sec. 6.1 max-cut on regular and random
graphs, Sec. 6.2 portfolio rebalancing, Sec. 7 scaling runs with random qualities and parameters):

* ``maxcut3``   - random 3-regular graph (pairing model with rejection), unit weights.
* ``maxcut_gnp`` - Erdos-Renyi G(n, 1/2) with edge weights uniform on [0, 1].
* ``subset``     - n Gaussian item weights (QWOA quality = sum of selected weights).
* ``portfolio``  - Gaussian returns and a random positive-definite covariance (Sec. 6.2).
* ``thetas``     - gamma_k, t_k uniform on [0, pi].

The master seed is 211003963; each named workload draws from
``Generator(PCG64(SeedSequence([MASTER_SEED, workload_id, instance])))``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASTER_SEED = 211003963

# workload ids (stable: changing one changes every seeded instance of that workload)
WL_MAXCUT10 = 1      # QAOA max-cut, n=10, 3-regular, complex128, p=2
WL_WMAXCUT28 = 2     # QAOA weighted max-cut, G(28, 1/2), p=8
WL_QWOA26 = 3        # QWOA circulant, N=2^26, p=6
WL_BATCH = 4         # batched QAOA, 4096 instances, n in 12..20, p in 2..8
WL_QAOAZ24 = 5       # QAOAz XY-ring on the Hamming-weight-12 subspace of 24 qubits, p=4


def rng_for(workload: int, instance: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([MASTER_SEED, workload, instance])))


@dataclass
class Graph:
    n: int
    eu: np.ndarray            # int32 [m] first endpoint (qubit index)
    ev: np.ndarray            # int32 [m] second endpoint
    w: np.ndarray | None = None   # float64 [m] edge weights, None = unit weights

    @property
    def m(self) -> int:
        return int(self.eu.shape[0])


def regular3_graph(n: int, rng: np.random.Generator, max_tries: int = 10000) -> Graph:
    """Random 3-regular simple graph by the pairing (configuration) model with rejection.

    For odd n a 3-regular graph does not exist; one vertex then gets degree 2 (all others 3).
    """
    degrees = [3] * n
    if (3 * n) % 2 == 1:
        degrees[-1] = 2
    stubs = np.repeat(np.arange(n, dtype=np.int64), degrees)
    for _ in range(max_tries):
        perm = rng.permutation(stubs)
        pairs = perm.reshape(-1, 2)
        u = np.minimum(pairs[:, 0], pairs[:, 1])
        v = np.maximum(pairs[:, 0], pairs[:, 1])
        if np.any(u == v):
            continue
        key = u * n + v
        if np.unique(key).shape[0] != key.shape[0]:
            continue
        order = np.argsort(key)
        return Graph(n, u[order].astype(np.int32), v[order].astype(np.int32), None)
    raise RuntimeError("pairing model did not produce a simple graph")


def gnp_graph(n: int, prob: float, rng: np.random.Generator, weighted: bool = True) -> Graph:
    """Erdos-Renyi G(n, prob); weights uniform on [0, 1] when ``weighted``."""
    iu, iv = np.triu_indices(n, k=1)
    keep = rng.random(iu.shape[0]) < prob
    eu, ev = iu[keep].astype(np.int32), iv[keep].astype(np.int32)
    w = rng.random(eu.shape[0]) if weighted else None
    return Graph(n, eu, ev, w)


def thetas(p: int, rng: np.random.Generator) -> tuple[np.ndarray, np.ndarray]:
    """gamma_k and t_k, each uniform on [0, pi] (layer k = 1..p)."""
    g = rng.uniform(0.0, math.pi, size=p)
    t = rng.uniform(0.0, math.pi, size=p)
    return g, t


def item_weights(k: int, rng: np.random.Generator) -> np.ndarray:
    """k Gaussian item weights N(0, 1) (QWOA subset-sum style qualities)."""
    return rng.standard_normal(k)


@dataclass
class Portfolio:
    n_assets: int
    returns: np.ndarray      # [M] expected returns r_i ~ N(0,1)
    cov: np.ndarray          # [M, M] covariance, A A^T / M + 1e-3 I with A_ij ~ N(0,1)
    omega: float = 0.5


def portfolio(n_assets: int, rng: np.random.Generator, omega: float = 0.5) -> Portfolio:
    r = rng.standard_normal(n_assets)
    a = rng.standard_normal((n_assets, n_assets))
    cov = a @ a.T / n_assets + 1e-3 * np.eye(n_assets)
    return Portfolio(n_assets, r, cov, omega)


def circulant_offsets_pow2(log2n: int) -> np.ndarray:
    """Connection offsets {1, 2, 4, ..., 2^(log2n-1)} of the circulant QWOA graph on N = 2^log2n.

    Each offset s couples vertex j with j+s and j-s (mod N); the offset N/2 couples each vertex
    with a single partner.
    """
    return (1 << np.arange(log2n, dtype=np.int64))


# ---------------------------------------------------------------- named workloads

@dataclass
class MaxCutInstance:
    graph: Graph
    p: int
    gammas: np.ndarray
    ts: np.ndarray


def maxcut10(instance: int = 0) -> MaxCutInstance:
    """QAOA max-cut, n=10, random 3-regular graph, integer qualities, p=2."""
    rng = rng_for(WL_MAXCUT10, instance)
    g = regular3_graph(10, rng)
    gam, t = thetas(2, rng)
    return MaxCutInstance(g, 2, gam, t)


def wmaxcut(n: int = 28, p: int = 8, instance: int = 0) -> MaxCutInstance:
    """QAOA weighted max-cut on G(n, 1/2), weights U[0,1], p layers."""
    rng = rng_for(WL_WMAXCUT28, instance * 1000 + n)
    g = gnp_graph(n, 0.5, rng, weighted=True)
    gam, t = thetas(p, rng)
    return MaxCutInstance(g, p, gam, t)


def maxcut3(n: int, p: int, instance: int = 0) -> MaxCutInstance:
    """QAOA max-cut on a random 3-regular graph with unit weights (batched workload member)."""
    rng = rng_for(WL_BATCH, instance * 1000 + n)
    g = regular3_graph(n, rng)
    gam, t = thetas(p, rng)
    return MaxCutInstance(g, p, gam, t)


@dataclass
class BatchSpec:
    ns: np.ndarray      # int [B] qubit counts
    ps: np.ndarray      # int [B] depths


def batch_spec(count: int = 4096, nmin: int = 12, nmax: int = 20, pmin: int = 2, pmax: int = 8,
               instance: int = 0) -> BatchSpec:
    rng = rng_for(WL_BATCH, 10_000_000 + instance)
    ns = rng.integers(nmin, nmax + 1, size=count)
    ps = rng.integers(pmin, pmax + 1, size=count)
    return BatchSpec(ns.astype(np.int32), ps.astype(np.int32))


@dataclass
class SubsetInstance:
    log2n: int
    weights: np.ndarray
    offsets: np.ndarray
    p: int
    gammas: np.ndarray
    ts: np.ndarray


def qwoa(log2n: int = 26, p: int = 6, instance: int = 0) -> SubsetInstance:
    """QWOA on the circulant graph with offsets 2^m, qualities = Gaussian item-weight sums."""
    rng = rng_for(WL_QWOA26, instance * 1000 + log2n)
    w = item_weights(log2n, rng)
    gam, t = thetas(p, rng)
    return SubsetInstance(log2n, w, circulant_offsets_pow2(log2n), p, gam, t)


@dataclass
class PortfolioInstance:
    n_qubits: int
    weight: int
    port: Portfolio
    p: int
    gammas: np.ndarray
    ts: np.ndarray


def qaoaz(n_qubits: int = 24, weight: int | None = None, p: int = 4, instance: int = 0) -> PortfolioInstance:
    """QAOAz on the Hamming-weight subspace; 2 qubits per asset (long, short)."""
    if weight is None:
        weight = n_qubits // 2
    rng = rng_for(WL_QAOAZ24, instance * 1000 + n_qubits)
    port = portfolio(n_qubits // 2, rng)
    gam, t = thetas(p, rng)
    return PortfolioInstance(n_qubits, weight, port, p, gam, t)
