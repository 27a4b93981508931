"""Closed-form results used to pin the oracle (and, at sizes the oracle cannot reach, the GPU path).

Nothing here calls the oracle or the CUDA library.
"""
from __future__ import annotations

import math

import numpy as np


def p1_maxcut_expectation(n: int, eu, ev, w, gamma: float, t: float) -> float:
    """<Q> after one QAOA layer, Q = sum_e w_e (1 + Z_u Z_v)/2, state exp(-itB) exp(-i gamma Q)|+>.

    Derived in the Heisenberg picture (the weighted generalisation of Wang, Hadfield, Jiang,
    Rieffel, PRA 97, 022304 (2018), which it reproduces for unit weights):
    with a_w = gamma*w_uw, b_w = gamma*w_vw and F = common neighbours of u and v,
      <Z_u Z_v> = 1/2 sin(4t) sin(gamma w_uv) [prod_{N(u)\\v} cos a_w + prod_{N(v)\\u} cos b_w]
                - 1/2 sin^2(2t) prod_{N(u)\\v\\F} cos a_w prod_{N(v)\\u\\F} cos b_w
                      [prod_F cos(a_w + b_w) - prod_F cos(a_w - b_w)].
    Works at any n (cost O(|E| * degree)).
    """
    if w is None:
        w = np.ones(len(eu))
    nbr = [dict() for _ in range(n)]
    for a, b, ww in zip(eu, ev, w):
        nbr[int(a)][int(b)] = float(ww)
        nbr[int(b)][int(a)] = float(ww)
    total = 0.0
    for a, b, ww in zip(eu, ev, w):
        u, v, wuv = int(a), int(b), float(ww)
        Nu = set(nbr[u]) - {v}
        Nv = set(nbr[v]) - {u}
        F = Nu & Nv
        pu = math.prod(math.cos(gamma * nbr[u][x]) for x in Nu)
        pv = math.prod(math.cos(gamma * nbr[v][x]) for x in Nv)
        ru = math.prod(math.cos(gamma * nbr[u][x]) for x in Nu - F)
        rv = math.prod(math.cos(gamma * nbr[v][x]) for x in Nv - F)
        fp = math.prod(math.cos(gamma * (nbr[u][x] + nbr[v][x])) for x in F)
        fm = math.prod(math.cos(gamma * (nbr[u][x] - nbr[v][x])) for x in F)
        zz = 0.5 * math.sin(4 * t) * math.sin(gamma * wuv) * (pu + pv) \
            - 0.5 * math.sin(2 * t) ** 2 * ru * rv * (fp - fm)
        total += wuv * 0.5 * (1.0 + zz)
    return total


def p1_maxcut_gradient(n, eu, ev, w, gamma, t, h=1e-5):
    """(dE/dgamma, dE/dt) of the p=1 closed form by Richardson central differences (the closed
    form is analytic, so this is accurate to ~1e-10)."""
    def d(fn, x, hh):
        return (fn(x + hh) - fn(x - hh)) / (2 * hh)

    fg = lambda g: p1_maxcut_expectation(n, eu, ev, w, g, t)
    ft = lambda tt: p1_maxcut_expectation(n, eu, ev, w, gamma, tt)
    dg = (4 * d(fg, gamma, h / 2) - d(fg, gamma, h)) / 3
    dt = (4 * d(ft, t, h / 2) - d(ft, t, h)) / 3
    return dg, dt


def p1_hypercube_amplitude(n: int, q: np.ndarray, gamma: float, t: float, i: int) -> complex:
    """<i| exp(-itB) exp(-i gamma Q) |+> as an explicit O(2^n) sum:
    <i|exp(-itB)|j> = cos(t)^(n-d) (-i sin t)^d with d = popcount(i xor j)."""
    N = 1 << n
    j = np.arange(N, dtype=np.int64)
    x = j ^ int(i)
    d = np.zeros(N, dtype=np.int64)
    for b in range(n):
        d += (x >> b) & 1
    amp = (np.cos(t) ** (n - d)) * ((-1j * np.sin(t)) ** d)
    return complex(np.sum(amp * np.exp(-1j * gamma * q)) / math.sqrt(N))


def complete_graph_mix(psi: np.ndarray, t: float) -> np.ndarray:
    """exp(-it(J - I)) psi = e^{it} [psi + (e^{-itN} - 1) mean(psi) 1] (J = all-ones)."""
    N = psi.shape[0]
    return np.exp(1j * t) * (psi + (np.exp(-1j * t * N) - 1.0) * psi.mean())


def pow2_circulant_eigs(log2n: int) -> np.ndarray:
    """Eigenvalues of the circulant graph on N = 2^m with offsets 2^0..2^(m-1):
    offsets s < N/2 contribute 2 cos(2 pi j s / N); s = N/2 contributes (-1)^j once."""
    N = 1 << log2n
    j = np.arange(N, dtype=np.int64)
    lam = np.zeros(N)
    for m in range(log2n - 1):
        s = 1 << m
        lam += 2 * np.cos(2 * math.pi * ((j * s) % N) / N)
    lam += np.where(j % 2 == 0, 1.0, -1.0)
    return lam


def givens_xy(t: float) -> np.ndarray:
    """exp(-i t (XX + YY)) on span{|01>, |10>}: [[cos 2t, -i sin 2t], [-i sin 2t, cos 2t]]."""
    c, s = math.cos(2 * t), math.sin(2 * t)
    return np.array([[c, -1j * s], [-1j * s, c]])
