"""Oracle: a plain, slow, fp64 (complex128) CPU state-vector simulator of the QVA hot path.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference legs of ``bench.py`` may import this package. It shares no code with the CUDA library
(``paper_2110_03963_gb300``) and never imports it; the two meet only in the seeded raw inputs of
``workloads``.

What it computes (paper: Matwiejew & Wang, "QuOp_MPI: a framework for parallel simulation of
quantum variational algorithms", arXiv 2110.03963):

* Sec. 2.1, generic ansatz: |theta> = prod_k U(theta_k) |psi0>, objective f = <theta|Q|theta>
  with Q diagonal (the quality vector q).
* Sec. 2.1 / Sec. 3, phase shift: U_phase(gamma) = exp(-i gamma Q) acts elementwise,
  c_i <- exp(-i gamma q_i) c_i.
* Sec. 2.1, mixer: U_mix(t) = exp(-i t W); three forms
    - Sec. 2.3.1 QAOA: W = sum_j X_j (hypercube adjacency; the printed "X^{tensor N}" is read as
      the sum of single-qubit X, which is the hypercube coupling of the same section). The oracle
      applies it as the product of the commuting single-qubit rotations exp(-i t X_j).
    - Sec. 2.4.2 / Sec. 3 QWOA: W circulant. Eigenvalues from the first row by the DFT relation of
      Sec. 3 (written out as a direct sum), action F^-1 exp(-i t Lambda) F (Sec. 3 prints
      exp(+i t Lambda); exp(-i t Lambda) is what equals exp(-i t W) of Sec. 2.1).
    - Sec. 2.4.1 QAOAz: W = sum over ring edges (a, a+1 mod n) of X_a X_{a+1} + Y_a Y_{a+1},
      restricted to a Hamming-weight subspace; exp(-i t W) v by a truncated Taylor series with
      step splitting (the scaling family of Sec. 3's sparse method).
* Layer order: phase first, then mixer, parameters interleaved (gamma_1, t_1, gamma_2, t_2, ...),
  as fixed by Example 1 (Sec. 6.1.1).
* Gradient: the adjoint recurrences of the alternating ansatz, every intermediate state stored
  (no uncompute), and Richardson-extrapolated central finite differences (Sec. 4 uses finite
  differences for the gradient).

Conventions: qubit u is bit (n-1-u) of the basis index (most significant first, as
``np.binary_repr`` in Example 3 and q_90 = 0 for (0,1,0,1,1,0,1,0) in Sec. 6.1.1).

Every function below is pinned by ``tests/test_oracle_pins.py`` against values the paper prints,
closed forms, dense matrix exponentials, and invariants; ``tests/test_oracle_mutants.py`` plants
one mistake at a time in these functions and checks that a pin fails.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# ============================================================== quality vectors (Sec. 2.2, Sec. 6)


def qubit_bits(n: int, idx: np.ndarray) -> np.ndarray:
    """x[u, i] = value of qubit u in basis state idx[i] (qubit u = bit n-1-u)."""
    idx = np.asarray(idx, dtype=np.int64)
    return np.stack([(idx >> (n - 1 - u)) & 1 for u in range(n)], axis=0)


def maxcut_quality(n: int, eu, ev, w=None) -> np.ndarray:
    """Sec. 6.1, max-cut cost C(s) = sum_{edges} 1/2 (I + Z_u Z_v) = (weighted) number of UNCUT edges.

    Unit weights give integers (Example 3 counts n_edges minus cut edges). With weights, each
    uncut edge contributes w_e; the terms are summed in edge order in fp64.
    """
    N = 1 << n
    idx = np.arange(N, dtype=np.int64)
    q = np.zeros(N, dtype=np.float64)
    for e in range(len(eu)):
        bu = (idx >> (n - 1 - int(eu[e]))) & 1
        bv = (idx >> (n - 1 - int(ev[e]))) & 1
        same = (bu == bv)
        q += np.where(same, 1.0 if w is None else float(w[e]), 0.0)
    return q


def subset_quality(n: int, weights) -> np.ndarray:
    """q_i = sum_b w_b x_b(i): item b is selected when qubit b is 1 (summed in item order, fp64)."""
    N = 1 << n
    idx = np.arange(N, dtype=np.int64)
    q = np.zeros(N, dtype=np.float64)
    for b in range(n):
        q += np.where(((idx >> (n - 1 - b)) & 1) == 1, float(weights[b]), 0.0)
    return q


def subspace_states(n: int, k: int) -> np.ndarray:
    """All n-bit basis states with exactly k ones, in increasing integer order."""
    idx = np.arange(1 << n, dtype=np.int64)
    pc = np.zeros_like(idx)
    for b in range(n):
        pc += (idx >> b) & 1
    return idx[pc == k]


def portfolio_quality(n_qubits: int, states: np.ndarray, returns, cov, omega: float) -> np.ndarray:
    """Sec. 6.2, discrete mean-variance cost omega * sum_ij sigma_ij z_i z_j - (1-omega) sum_i r_i z_i.

    Two qubits per asset a: qubit 2a is the 'long' qubit, qubit 2a+1 the 'short' one;
    |10> -> long (z=+1), |01> -> short (z=-1), |00>,|11> -> no position (z=0).
    """
    M = n_qubits // 2
    x = qubit_bits(n_qubits, states)
    z = np.stack([x[2 * a] - x[2 * a + 1] for a in range(M)], axis=0).astype(np.float64)
    q = np.zeros(states.shape[0], dtype=np.float64)
    for i in range(M):
        for j in range(M):
            q += omega * float(cov[i][j]) * z[i] * z[j]
    for i in range(M):
        q -= (1.0 - omega) * float(returns[i]) * z[i]
    return q


def qubo_quality(n: int, c: float, h, J) -> np.ndarray:
    """Qualities written as a quadratic form of the qubit values (Sec. 2.2: q is any function of the
    basis state; the max-cut, subset-sum and portfolio costs of Sec. 6 are all of this form):

        q(x) = c + sum_u h_u x_u + sum_{u<v} J_uv x_u x_v     (x_u = value of qubit u)

    J is read above its diagonal only. fp64, terms in the order c, h_0..h_{n-1}, then J by rows.
    """
    N = 1 << n
    x = qubit_bits(n, np.arange(N, dtype=np.int64)).astype(np.float64)
    q = np.full(N, float(c), dtype=np.float64)
    for u in range(n):
        q += float(h[u]) * x[u]
    for u in range(n):
        for v in range(u + 1, n):
            q += float(J[u][v]) * x[u] * x[v]
    return q


def qubo_fixed_point(n: int, c: float, h, J):
    """Fixed-point form of a quadratic quality, the contract of qvs_set_quality_qubo /
    qvs_quality_qubo (not a step of the paper: the device evaluates q(x) exactly on this grid).

    S = |c| + sum_u |h_u| + sum_{u<v} |J_uv| (fp64, that order); F = the largest integer in
    [-30, 40] with S * 2^F + 1024 <= 2^30; every coefficient is rounded to the nearest integer
    multiple of 2^-F, halves away from zero. Any sum of the rounded coefficients is then an integer
    of magnitude below 2^30 (so exact in 32-bit integers). Returns (F, ci, hi, Ji) with integer
    ci, hi[u], Ji[u][v] (u < v; zero elsewhere).
    """
    S = abs(float(c))
    for u in range(n):
        S += abs(float(h[u]))
    for u in range(n):
        for v in range(u + 1, n):
            S += abs(float(J[u][v]))
    F = 40
    while F > -30 and S * 2.0 ** F + 1024.0 > 2.0 ** 30:
        F -= 1

    def rnd(x):
        y = abs(float(x)) * 2.0 ** F
        r = math.floor(y + 0.5)
        return int(r) if x >= 0 else -int(r)

    ci = rnd(c)
    hi = [rnd(h[u]) for u in range(n)]
    Ji = [[rnd(J[u][v]) if v > u else 0 for v in range(n)] for u in range(n)]
    return F, ci, hi, Ji


def qubo_quality_fixed(n: int, c: float, h, J) -> np.ndarray:
    """q(x) of the fixed-point coefficients of ``qubo_fixed_point``, summed exactly in integers and
    scaled by 2^-F (exact in fp64: the integers stay below 2^30)."""
    F, ci, hi, Ji = qubo_fixed_point(n, c, h, J)
    N = 1 << n
    x = qubit_bits(n, np.arange(N, dtype=np.int64))
    qi = np.full(N, ci, dtype=np.int64)
    for u in range(n):
        qi += hi[u] * x[u]
    for u in range(n):
        for v in range(u + 1, n):
            qi += Ji[u][v] * x[u] * x[v]
    return qi.astype(np.float64) * 2.0 ** (-F)


# ============================================================== unitaries (Sec. 2.1, Sec. 3)


def phase(psi: np.ndarray, q: np.ndarray, gamma: float) -> np.ndarray:
    """Sec. 3: U_phase(gamma) psi = sum_i exp(-i gamma q_i) c_i |i>."""
    return psi * (np.cos(gamma * q) - 1j * np.sin(gamma * q))


def mix_hypercube(psi: np.ndarray, n: int, t: float) -> np.ndarray:
    """Sec. 2.3.1: exp(-i t sum_j X_j) = prod_j (cos t I - i sin t X_j), one qubit at a time."""
    c, s = math.cos(t), math.sin(t)
    out = psi.copy()
    for b in range(n):
        v = out.reshape(-1, 2, 1 << b)      # axis 1 = bit b
        a0 = v[:, 0, :].copy()
        a1 = v[:, 1, :].copy()
        v[:, 0, :] = c * a0 - 1j * s * a1
        v[:, 1, :] = c * a1 - 1j * s * a0
    return out


def apply_hypercube_W(psi: np.ndarray, n: int) -> np.ndarray:
    """W psi with W = sum_j X_j (X_j flips bit j)."""
    idx = np.arange(psi.shape[0], dtype=np.int64)
    out = np.zeros_like(psi)
    for b in range(n):
        out += psi[idx ^ (1 << b)]
    return out


def circulant_first_row_from_offsets(N: int, offsets, weight: float = 1.0) -> np.ndarray:
    """Symmetric circulant adjacency: w_s = w_{N-s} = weight for each offset s (0 < s < N)."""
    row = np.zeros(N, dtype=np.float64)
    for s in offsets:
        s = int(s) % N
        if s == 0:
            continue
        row[s] = weight
        row[(N - s) % N] = weight
    return row


def circulant_eigenvalues(first_row: np.ndarray) -> np.ndarray:
    """Sec. 3: lambda_j = sum_k w_k omega^{jk}, omega = exp(2 pi i / M), summed directly over the
    nonzero entries of the first row. Requires a symmetric first row (w_k = w_{M-k}), so the
    eigenvalues are real; the exponent j*k is reduced mod M in integers before the cosine.
    """
    M = first_row.shape[0]
    ks = np.nonzero(first_row)[0]
    assert np.allclose(first_row, np.roll(first_row[::-1], 1)), "circulant must be symmetric"
    j = np.arange(M, dtype=np.int64)
    lam = np.zeros(M, dtype=np.float64)
    for k in ks:
        lam += first_row[k] * np.cos(2.0 * math.pi * ((j * int(k)) % M) / M)
    return lam


def mix_circulant(psi: np.ndarray, lam: np.ndarray, t: float) -> np.ndarray:
    """Sec. 3: U_mix(t) psi = F^-1 exp(-i t Lambda) F psi (F = unitary DFT; numpy's FFT pair)."""
    return np.fft.ifft(np.exp(-1j * t * lam) * np.fft.fft(psi))


def apply_circulant_W(psi: np.ndarray, lam: np.ndarray) -> np.ndarray:
    return np.fft.ifft(lam * np.fft.fft(psi))


def xy_ring_apply(psi: np.ndarray, n: int, states: np.ndarray) -> np.ndarray:
    """Sec. 2.4.1 operator family: W = sum_{a=0}^{n-1} (X_a X_{a+1} + Y_a Y_{a+1}), a+1 taken mod n,
    on the subspace spanned by ``states``. (XX+YY)|01> = 2|10>, (XX+YY)|00> = (XX+YY)|11> = 0.
    """
    out = np.zeros_like(psi)
    for a in range(n):
        b = (a + 1) % n
        ba, bb = n - 1 - a, n - 1 - b
        differ = (((states >> ba) ^ (states >> bb)) & 1) == 1
        src = np.nonzero(differ)[0]
        flipped = states[src] ^ ((1 << ba) | (1 << bb))
        dst = np.searchsorted(states, flipped)
        assert np.all(states[dst] == flipped)
        np.add.at(out, dst, 2.0 * psi[src])
    return out


def mix_xy_ring(psi: np.ndarray, n: int, states: np.ndarray, t: float) -> np.ndarray:
    """exp(-i t W) psi by a Taylor series with step splitting: s substeps of tau = t/s with
    |tau| * ||W||_1 <= 1 (||W||_1 <= 2n: at most n differing ring pairs, each entry 2); each
    substep sums terms until one falls below 1e-18 of the vector's max norm.
    """
    s = max(1, math.ceil(abs(t) * 2 * n))
    tau = t / s
    v = psi.copy()
    for _ in range(s):
        term = v.copy()
        acc = v.copy()
        m = 1
        while True:
            term = (-1j * tau / m) * xy_ring_apply(term, n, states)
            acc = acc + term
            if np.max(np.abs(term)) < 1e-18 * max(np.max(np.abs(acc)), 1e-300) or m > 60:
                break
            m += 1
        v = acc
    return v


# ============================================================== QAOAz parity-ring mixer (Sec. 2.4.1)


def parity_ring_rounds(n: int):
    """Sec. 2.4.1, Eqs. for B_odd, B_even, B_last and U_parity: the qubit pairs of the three
    factors, for the two rings of an n-qubit register (one ring on the even qubits 0, 2, ..., one on
    the odd qubits 1, 3, ...). On a ring of N qubits with 1-indexed positions k:
      B_odd  couples (k, k+1) for odd k < N,
      B_even couples (k, k+1) for even k < N, and the closing pair (N, 1) when N is even,
      B_last couples (N, 1) when N is odd (identity when N is even).
    Returns [pairs of B_odd, pairs of B_even, pairs of B_last] as global qubit pairs; the pairs of
    one factor are disjoint, and the two rings share no qubit."""
    rounds = [[], [], []]
    for ring in ([q for q in range(0, n, 2)], [q for q in range(1, n, 2)]):
        N = len(ring)
        pos = lambda k: ring[k - 1]   # 1-indexed position on the ring -> qubit
        for k in range(1, N):
            rounds[0 if k % 2 == 1 else 1].append((pos(k), pos(k + 1)))
        if N >= 2:
            rounds[1 if N % 2 == 0 else 2].append((pos(N), pos(1)))
    return rounds


def xy_pairs_apply(psi: np.ndarray, n: int, pairs) -> np.ndarray:
    """B psi for B = sum over the pairs (u, v) of X_u X_v + Y_u Y_v: (XX+YY)|01> = 2|10>,
    (XX+YY)|10> = 2|01>, zero on |00> and |11> (qubit u = bit n-1-u)."""
    N = psi.shape[0]
    idx = np.arange(N, dtype=np.int64)
    out = np.zeros_like(psi, dtype=np.complex128)
    for u, v in pairs:
        bu, bv = n - 1 - u, n - 1 - v
        differ = (((idx >> bu) ^ (idx >> bv)) & 1) == 1
        out[differ] += 2.0 * psi[idx[differ] ^ ((1 << bu) | (1 << bv))]
    return out


def xy_pairs_exp(psi: np.ndarray, n: int, pairs, t: float) -> np.ndarray:
    """exp(-i t B) psi for disjoint pairs: one Givens rotation per pair on its |01>, |10>
    amplitudes, [[cos 2t, -i sin 2t], [-i sin 2t, cos 2t]] (exp(-i t (XX+YY)) on that plane)."""
    N = psi.shape[0]
    idx = np.arange(N, dtype=np.int64)
    out = np.asarray(psi, dtype=np.complex128).copy()
    c, s = math.cos(2.0 * t), math.sin(2.0 * t)
    for u, v in pairs:
        bu, bv = n - 1 - u, n - 1 - v
        lo = idx[(((idx >> bu) & 1) == 0) & (((idx >> bv) & 1) == 1)]
        hi = lo ^ ((1 << bu) | (1 << bv))
        a, b = out[lo].copy(), out[hi].copy()
        out[lo] = c * a - 1j * s * b
        out[hi] = c * b - 1j * s * a
    return out


def mix_parity(psi: np.ndarray, n: int, t: float) -> np.ndarray:
    """U_parity(t) = exp(-i t B_last) exp(-i t B_even) exp(-i t B_odd) on both rings (the rings act
    on disjoint qubits and commute); one t for every factor."""
    for pairs in parity_ring_rounds(n):
        psi = xy_pairs_exp(psi, n, pairs, t)
    return psi


def parity_state(n: int, A: int) -> np.ndarray:
    """Sec. 6.2 QAOAz initial state: |01>^{(x)A} ((|00> + |11>)/sqrt 2)^{(x)(M-A)}, M = n/2 assets,
    one pair of qubits (2a, 2a+1) per asset in qubit order (qubit u = bit n-1-u)."""
    M = n // 2
    state = np.array([1.0 + 0j])
    for a in range(M):
        pair = np.zeros(4, dtype=np.complex128)   # index = 2 * x_{2a} + x_{2a+1}
        if a < A:
            pair[0b01] = 1.0
        else:
            pair[0b00] = pair[0b11] = 1.0 / math.sqrt(2.0)
        state = np.kron(state, pair)
    return state


def mix_dense(psi: np.ndarray, W: np.ndarray, t: float) -> np.ndarray:
    """Sec. 2.1 / Sec. 3: exp(-i t W) psi for a real symmetric W given densely, from the definition
    of the matrix exponential of a symmetric matrix: W = V diag(w) V^T, exp(-i t W) = V diag(exp(-i t w)) V^T
    (numpy eigh as the library step)."""
    w, V = np.linalg.eigh(np.asarray(W, dtype=np.float64))
    return V @ (np.exp(-1j * t * w) * (V.T @ np.asarray(psi, dtype=np.complex128)))


# ============================================================== problems and the ansatz


@dataclass
class Problem:
    """One QVA instance: quality vector q (fp64), a mixer, and an initial state (None = uniform)."""
    q: np.ndarray
    mixer: str                     # "hypercube" | "circulant" | "xy_ring" | "dense" | "parity"
    n: int = 0                     # qubits (hypercube, xy_ring)
    lam: np.ndarray | None = None  # circulant eigenvalues
    states: np.ndarray | None = None   # xy_ring subspace basis
    psi0: np.ndarray | None = None
    W: np.ndarray | None = None        # dense real symmetric mixer matrix

    @property
    def dim(self) -> int:
        return int(self.q.shape[0])

    def initial_state(self) -> np.ndarray:
        """Sec. 2.3.1 / Sec. 2.4.2: equal superposition over the simulated space, 1/sqrt(dim)."""
        if self.psi0 is not None:
            return np.asarray(self.psi0, dtype=np.complex128).copy()
        return np.full(self.dim, 1.0 / math.sqrt(self.dim), dtype=np.complex128)

    def mix(self, psi: np.ndarray, t: float) -> np.ndarray:
        if self.mixer == "hypercube":
            return mix_hypercube(psi, self.n, t)
        if self.mixer == "circulant":
            return mix_circulant(psi, self.lam, t)
        if self.mixer == "xy_ring":
            return mix_xy_ring(psi, self.n, self.states, t)
        if self.mixer == "dense":
            return mix_dense(psi, self.W, t)
        if self.mixer == "parity":
            return mix_parity(psi, self.n, t)
        raise ValueError(self.mixer)

    def apply_W(self, psi: np.ndarray) -> np.ndarray:
        if self.mixer == "hypercube":
            return apply_hypercube_W(psi, self.n)
        if self.mixer == "circulant":
            return apply_circulant_W(psi, self.lam)
        if self.mixer == "xy_ring":
            return xy_ring_apply(psi, self.n, self.states)
        if self.mixer == "dense":
            return np.asarray(self.W, dtype=np.float64) @ psi
        raise ValueError(self.mixer)


def evolve(prob: Problem, gammas, ts) -> np.ndarray:
    """Sec. 2.1 / Eqs. of Sec. 2.3-2.4: psi_p = prod_{k=1..p} U_mix(t_k) U_phase(gamma_k) psi0."""
    psi = prob.initial_state()
    for g, t in zip(gammas, ts):
        psi = phase(psi, prob.q, float(g))
        psi = prob.mix(psi, float(t))
    return psi


def expectation(psi: np.ndarray, q: np.ndarray) -> float:
    """Sec. 2.1: f = <psi|Q|psi> = sum_i q_i |c_i|^2."""
    return float(np.sum(q * (psi.real ** 2 + psi.imag ** 2)))


def objective(prob: Problem, gammas, ts) -> float:
    return expectation(evolve(prob, gammas, ts), prob.q)


def gradient(prob: Problem, gammas, ts):
    """Adjoint gradient of f = <psi_p|Q|psi_p> with every state stored.

    Forward: phi_k = P_k psi_{k-1}, psi_k = M_k phi_k.
    With lambda_p = Q psi_p and lambda_{k-1} = P_k^dag M_k^dag lambda_k:
      df/dt_k     = 2 Im <lambda_k | W psi_k>
      df/dgamma_k = 2 Im <M_k^dag lambda_k | Q phi_k>
    Returns (f, dgamma[p], dt[p]).
    """
    if prob.mixer == "parity":
        return _gradient_factored(prob, gammas, ts)
    p = len(gammas)
    psi = prob.initial_state()
    phis, psis = [], []
    for k in range(p):
        phi = phase(psi, prob.q, float(gammas[k]))
        psi = prob.mix(phi, float(ts[k]))
        phis.append(phi)
        psis.append(psi)
    f = expectation(psi, prob.q)
    lam = prob.q * psi
    dg = np.zeros(p)
    dt = np.zeros(p)
    for k in range(p - 1, -1, -1):
        dt[k] = 2.0 * np.vdot(lam, prob.apply_W(psis[k])).imag
        lam = prob.mix(lam, -float(ts[k]))                # M_k^dag
        dg[k] = 2.0 * np.vdot(lam, prob.q * phis[k]).imag
        lam = phase(lam, prob.q, -float(gammas[k]))       # P_k^dag
    return f, dg, dt


def _gradient_factored(prob: Problem, gammas, ts):
    """Adjoint gradient for a mixer that is a product of exponentials sharing one t,
    M(t) = exp(-i t B_F) ... exp(-i t B_1) (the parity mixer). Every factor's input state is stored;
    with lambda moved back through the factors,
      df/dt_k     = sum_f 2 Im <lambda_{k,f} | B_f psi_{k,f}>   (both at factor f's output)
      df/dgamma_k = 2 Im <M_k^dag lambda_k | Q phi_k>."""
    p = len(gammas)
    rounds = parity_ring_rounds(prob.n)
    psi = prob.initial_state()
    phis, outs = [], []   # outs[k][f] = state after factor f of layer k
    for k in range(p):
        phi = phase(psi, prob.q, float(gammas[k]))
        phis.append(phi)
        cur, lst = phi, []
        for pairs in rounds:
            cur = xy_pairs_exp(cur, prob.n, pairs, float(ts[k]))
            lst.append(cur)
        outs.append(lst)
        psi = cur
    f = expectation(psi, prob.q)
    lam = prob.q * psi
    dg = np.zeros(p)
    dt = np.zeros(p)
    for k in range(p - 1, -1, -1):
        for fi in range(len(rounds) - 1, -1, -1):
            dt[k] += 2.0 * np.vdot(lam, xy_pairs_apply(outs[k][fi], prob.n, rounds[fi])).imag
            lam = xy_pairs_exp(lam, prob.n, rounds[fi], -float(ts[k]))
        dg[k] = 2.0 * np.vdot(lam, prob.q * phis[k]).imag
        lam = phase(lam, prob.q, -float(gammas[k]))
    return f, dg, dt


# ============================================================== ex-QAOA (Sec. 2.3.2)


def pauli_z_diag(n: int, u: int, v: int = -1) -> np.ndarray:
    """Diagonal of Z_u (v < 0) or Z_u Z_v on n qubits: Z has eigenvalue +1 on |0>, -1 on |1>."""
    x = qubit_bits(n, np.arange(1 << n, dtype=np.int64))
    z = 1.0 - 2.0 * x[u].astype(np.float64)
    if v >= 0:
        z = z * (1.0 - 2.0 * x[v].astype(np.float64))
    return z


def exqaoa_term_diags(n: int, tu, tv, coef):
    """Sec. 2.3.2: the terms Sigma_j = coef_j Z_u Z_v (tv[j] < 0: coef_j Z_u) as diagonals."""
    return [float(coef[j]) * pauli_z_diag(n, int(tu[j]), int(tv[j])) for j in range(len(coef))]


def exqaoa_phase(psi: np.ndarray, terms, gam) -> np.ndarray:
    """Eq. of U_Qext: prod_j exp(-i gamma_j Sigma_j), each diagonal factor applied in turn."""
    for j, S in enumerate(terms):
        psi = psi * np.exp(-1j * float(gam[j]) * S)
    return psi


def exqaoa_evolve(prob: Problem, terms, G, ts) -> np.ndarray:
    """Sec. 2.3.2: psi = prod_k U_X(t_k) U_Qext(gamma_{k,:}) |+>; G[k][j] = gamma_{k,j}."""
    psi = prob.initial_state()
    for k in range(len(ts)):
        psi = exqaoa_phase(psi, terms, G[k])
        psi = prob.mix(psi, float(ts[k]))
    return psi


def exqaoa_gradient(prob: Problem, terms, G, ts):
    """Adjoint gradient of f = <psi_p|Q|psi_p> for ex-QAOA, every state stored. With
    phi_k = U_Qext,k psi_{k-1}, psi_k = M_k phi_k, lambda_p = Q psi_p:
      df/dt_k         = 2 Im <lambda_k | W psi_k>
      df/dgamma_{k,j} = 2 Im <M_k^dag lambda_k | Sigma_j phi_k>
    Returns (f, dG[p][J], dt[p])."""
    p = len(ts)
    J = len(terms)
    psi = prob.initial_state()
    phis, psis = [], []
    for k in range(p):
        phi = exqaoa_phase(psi, terms, G[k])
        psi = prob.mix(phi, float(ts[k]))
        phis.append(phi)
        psis.append(psi)
    f = expectation(psi, prob.q)
    lam = prob.q * psi
    dG = np.zeros((p, J))
    dt = np.zeros(p)
    for k in range(p - 1, -1, -1):
        dt[k] = 2.0 * np.vdot(lam, prob.apply_W(psis[k])).imag
        lam = prob.mix(lam, -float(ts[k]))
        for j in range(J):
            dG[k, j] = 2.0 * np.vdot(lam, terms[j] * phis[k]).imag
        lam = exqaoa_phase(lam, terms, -np.asarray(G[k], dtype=np.float64))
    return f, dG, dt


def central_fd(prob: Problem, gammas, ts, h: float = 1e-3):
    """Richardson-extrapolated central differences: D(h) = (f(x+h)-f(x-h))/2h,
    estimate = (4 D(h/2) - D(h)) / 3 (error O(h^4))."""
    gammas = np.asarray(gammas, dtype=np.float64)
    ts = np.asarray(ts, dtype=np.float64)
    p = len(gammas)

    def d(vec_is_gamma, k, hh):
        g1, t1 = gammas.copy(), ts.copy()
        g2, t2 = gammas.copy(), ts.copy()
        if vec_is_gamma:
            g1[k] += hh
            g2[k] -= hh
        else:
            t1[k] += hh
            t2[k] -= hh
        return (objective(prob, g1, t1) - objective(prob, g2, t2)) / (2 * hh)

    dg = np.array([(4 * d(True, k, h / 2) - d(True, k, h)) / 3 for k in range(p)])
    dt = np.array([(4 * d(False, k, h / 2) - d(False, k, h)) / 3 for k in range(p)])
    return dg, dt


# ============================================================== classical optimiser (Sec. 4)


BFGS_MAX_HALVINGS = 30   # line-search step sizes 1, 1/2, ..., 2^-30


def bfgs_minimize(fg, x0, gtol: float = 1e-8, max_iter: int = 1000, c1: float = 1e-4):
    """BFGS quasi-Newton minimisation, the paper's default classical optimiser (Sec. 4 uses
    SciPy's BFGS through `minimize`), written out step by step:

    * search direction d = -H g with H the inverse-Hessian estimate (H_0 = I);
    * backtracking line search from step 1, halving until the Armijo condition
      f(x + a d) <= f(x) + c1 a g.d holds, for at most BFGS_MAX_HALVINGS halvings;
    * with s = x_new - x and y = g_new - g, the inverse update
      H <- (I - rho s y^T) H (I - rho y s^T) + rho s s^T, rho = 1 / y.s, skipped when y.s <= 0
      (the curvature condition fails) so that H stays positive definite;
    * stop when max |g| <= gtol (stop = 0), after max_iter iterations (stop = 1), or when no step
      of the line search decreases f enough (stop = 2: the objective's rounding hides any further
      descent; x, f, g stay at the last accepted point, as SciPy's BFGS ends with its
      precision-loss message).

    fg(x) returns (f, g). Returns (x, f, iterations, evaluations, stop)."""
    x = np.asarray(x0, dtype=np.float64).copy()
    n = x.shape[0]
    f, g = fg(x)
    g = np.asarray(g, dtype=np.float64)
    H = np.eye(n)
    evals = 1
    it = 0
    stop = 1
    while it < max_iter:
        if np.max(np.abs(g)) <= gtol:
            stop = 0
            break
        d = -H @ g
        slope = float(g @ d)
        if slope >= 0.0:            # not a descent direction: restart from steepest descent
            H = np.eye(n)
            d = -g
            slope = float(g @ d)
        a = 1.0
        accepted = False
        for _ in range(BFGS_MAX_HALVINGS + 1):
            xn = x + a * d
            fn, gn = fg(xn)
            evals += 1
            if fn <= f + c1 * a * slope:
                accepted = True
                break
            a *= 0.5
        if not accepted:
            stop = 2
            break
        gn = np.asarray(gn, dtype=np.float64)
        s_ = xn - x
        y_ = gn - g
        ys = float(y_ @ s_)
        if ys > 0.0:
            rho = 1.0 / ys
            I = np.eye(n)
            H = (I - rho * np.outer(s_, y_)) @ H @ (I - rho * np.outer(y_, s_)) + rho * np.outer(s_, s_)
        x, f, g = xn, fn, gn
        it += 1
    else:
        if np.max(np.abs(g)) <= gtol:
            stop = 0
    return x, f, it, evals, stop


def optimise(prob: Problem, gammas0, ts0, gtol: float = 1e-8, max_iter: int = 1000):
    """Minimise f(theta) = <theta|Q|theta> over theta = (gamma_1, t_1, ..., gamma_p, t_p) (the layer
    order of Example 1) with `bfgs_minimize` and the adjoint gradient. Returns
    (gammas, ts, f, iterations, evaluations, stop)."""
    p = len(gammas0)

    def fg(th):
        gs, ts = th[0::2], th[1::2]
        f, dg, dt = gradient(prob, gs, ts)
        out = np.empty(2 * p)
        out[0::2] = dg
        out[1::2] = dt
        return f, out

    th0 = np.empty(2 * p)
    th0[0::2] = gammas0
    th0[1::2] = ts0
    th, f, it, ev, stop = bfgs_minimize(fg, th0, gtol=gtol, max_iter=max_iter)
    return th[0::2], th[1::2], f, it, ev, stop


def benchmark(prob: Problem, d_min: int, d_max: int, repeats: int, init, gtol: float = 1e-8,
              max_iter: int = 1000):
    """Sec. 5, the Ansatz's benchmark method with param_persist = True: for each depth
    D = d_min..d_max, `repeats` optimisations (`optimise`). At D = d_min repeat r starts from
    init[r * 2 d_min:] (gamma_1..gamma_D, then t_1..t_D); at every later depth each repeat starts
    from the best optimum of depth D - 1 (lowest f, the first repeat on ties) for layers 1..D-1 and
    from its own next two init values (gamma_D, t_D) for layer D.
    Returns (f[depth][repeat], [(gammas, ts) of the best repeat at each depth])."""
    init = np.asarray(init, dtype=np.float64).reshape(-1)
    pos = 0
    fs, best = [], []
    for D in range(d_min, d_max + 1):
        row = []
        results = []
        for r in range(repeats):
            if D == d_min:
                g0 = init[pos + r * 2 * D: pos + r * 2 * D + D]
                t0 = init[pos + r * 2 * D + D: pos + (r + 1) * 2 * D]
            else:
                g0 = np.append(best[-1][0], init[pos + 2 * r])
                t0 = np.append(best[-1][1], init[pos + 2 * r + 1])
            gs, ts, f, _, _, _ = optimise(prob, g0, t0, gtol=gtol, max_iter=max_iter)
            row.append(f)
            results.append((np.asarray(gs), np.asarray(ts)))
        pos += repeats * 2 * D if D == d_min else repeats * 2
        fs.append(row)
        best.append(results[int(np.argmin(row))])
    return np.array(fs), best


# ============================================================== convenience builders


def maxcut_problem(n: int, eu, ev, w=None, q_dtype=None) -> Problem:
    """QAOA max-cut: hypercube mixer; q rounded to ``q_dtype`` (e.g. float32) and promoted back
    to fp64 when the simulated device path consumes that precision."""
    q = maxcut_quality(n, eu, ev, w)
    if q_dtype is not None:
        q = q.astype(q_dtype).astype(np.float64)
    return Problem(q=q, mixer="hypercube", n=n)


def qwoa_problem(log2n: int, weights, offsets, q_dtype=None) -> Problem:
    N = 1 << log2n
    q = subset_quality(log2n, weights)
    if q_dtype is not None:
        q = q.astype(q_dtype).astype(np.float64)
    lam = circulant_eigenvalues(circulant_first_row_from_offsets(N, offsets))
    return Problem(q=q, mixer="circulant", lam=lam)


def qaoaz_parity_problem(n: int, A: int, returns, cov, omega: float, q_dtype=None) -> Problem:
    """QAOAz with the paper's parity-ring mixer on the full 2^n register, portfolio qualities of
    every basis state, and the parity initial state with constraint value A."""
    q = portfolio_quality(n, np.arange(1 << n, dtype=np.int64), returns, cov, omega)
    if q_dtype is not None:
        q = q.astype(q_dtype).astype(np.float64)
    return Problem(q=q, mixer="parity", n=n, psi0=parity_state(n, A))


def qaoaz_problem(n: int, k: int, returns, cov, omega: float, q_dtype=None) -> Problem:
    states = subspace_states(n, k)
    q = portfolio_quality(n, states, returns, cov, omega)
    if q_dtype is not None:
        q = q.astype(q_dtype).astype(np.float64)
    return Problem(q=q, mixer="xy_ring", n=n, states=states)
