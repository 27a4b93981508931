"""The seeded synthetic inputs have the shapes and distributions the workload recipe states (CPU)."""
import math

import numpy as np
import pytest

import workloads as wl


@pytest.mark.parametrize("n", [8, 10, 13, 19, 20])
def test_regular3_graph(n):
    G = wl.regular3_graph(n, wl.rng_for(300, n))
    deg = np.bincount(np.concatenate([G.eu, G.ev]), minlength=n)
    assert sorted(deg.tolist()) == ([2] + [3] * (n - 1) if n % 2 else [3] * n)
    pairs = {(min(u, v), max(u, v)) for u, v in zip(G.eu.tolist(), G.ev.tolist())}
    assert len(pairs) == G.m and all(u != v for u, v in pairs) and G.w is None


def test_gnp_graph_weights_and_density():
    G = wl.gnp_graph(28, 0.5, wl.rng_for(301))
    assert np.all(G.eu < G.ev) and G.eu.dtype == np.int32
    assert np.all((G.w >= 0) & (G.w < 1)) and G.w.shape == G.eu.shape
    m = 28 * 27 // 2
    assert abs(G.m - m / 2) < 4 * math.sqrt(m / 4)          # Binomial(378, 1/2) within 4 sigma
    assert wl.wmaxcut(28, 8).graph.m == 190                  # the benchmark instance


def test_portfolio_and_items():
    P = wl.portfolio(12, wl.rng_for(302))
    assert P.cov.shape == (12, 12) and np.allclose(P.cov, P.cov.T)
    assert np.linalg.eigvalsh(P.cov).min() >= 1e-3 - 1e-12   # A A^T / M + 1e-3 I
    assert P.omega == 0.5 and P.returns.shape == (12,)
    w = wl.item_weights(4096, wl.rng_for(303))
    assert abs(w.mean()) < 0.1 and abs(w.std() - 1.0) < 0.1


def test_parameters_batch_and_offsets():
    g, t = wl.thetas(1000, wl.rng_for(304))
    assert np.all((g >= 0) & (g <= math.pi)) and np.all((t >= 0) & (t <= math.pi))
    spec = wl.batch_spec()
    assert spec.ns.shape == (4096,) and spec.ns.min() == 12 and spec.ns.max() == 20
    assert spec.ps.min() == 2 and spec.ps.max() == 8
    assert wl.circulant_offsets_pow2(5).tolist() == [1, 2, 4, 8, 16]


def test_seeded_streams_are_reproducible_and_distinct():
    a = wl.rng_for(305, 1).standard_normal(8)
    assert np.array_equal(a, wl.rng_for(305, 1).standard_normal(8))
    assert not np.array_equal(a, wl.rng_for(305, 2).standard_normal(8))
    assert not np.array_equal(a, wl.rng_for(306, 1).standard_normal(8))
