"""The oracle's pins catch planted mistakes (CPU only).

Each case takes the source of one oracle function, plants one plausible mistake in it by a textual
replacement (a flipped sign, a dropped term or qubit, a transposed operand, a wrong bit order, a
swapped parameter or factor order), rebuilds the function and puts it into the ``oracle`` module
in place of the original for the duration of the case. The pins of ``test_oracle_pins`` that
should notice are then run against the planted oracle: at least one of them must fail. A mutant
that no pin notices marks a gap in the pins.

The mistakes are planted in the oracle only, on the CPU; nothing here touches the CUDA library.
"""
import __future__
import inspect
import textwrap

import numpy as np
import pytest

import oracle as orc
from tests import test_oracle_pins as pins

PINS = {
    "ex1": pins.test_p1_example1_objective_matches_printed_value,
    "ex1_q": pins.test_p2_example1_optimal_quality_and_bit_order,
    "p1_closed": lambda: [pins.test_p3_p1_closed_form(*a) for a in ((8, False, 0), (9, True, 2))],
    "p1_amp": pins.test_p3_p1_amplitudes_explicit_sum,
    "hc_expm": pins.test_p4_hypercube_vs_expm,
    "circ_expm": pins.test_p4_circulant_vs_expm,
    "xy_expm": lambda: [pins.test_p4_xy_ring_vs_expm(*a) for a in ((6, 3), (7, 2))],
    "dense_forms": pins.test_dense_mixer_vs_independent_forms,
    "ansatz_dense": pins.test_p4_full_ansatz_vs_dense_qaoa,
    "complete": pins.test_p5_complete_graph_mixer,
    "circ_eigs": lambda: [pins.test_p7_circulant_eigenvalues(m) for m in (4, 9)],
    "givens": pins.test_p8_xy_pair_is_givens,
    "norm": pins.test_p9_norm_and_reversibility,
    "period": pins.test_p9_periodicities_and_symmetry,
    "parity_dense": lambda: pins.test_parity_mixer_vs_dense_factors(6),
    "parity_geom": pins.test_parity_mixer_ring_geometry_and_two_site_ring,
    "parity_state": pins.test_parity_state_and_conservation,
    "fd_hc": lambda: pins.test_p10_adjoint_vs_richardson_fd("hypercube"),
    "fd_circ": lambda: pins.test_p10_adjoint_vs_richardson_fd("circulant"),
    "fd_xy": lambda: pins.test_p10_adjoint_vs_richardson_fd("xy_ring"),
    "fd_dense": lambda: pins.test_p10_adjoint_vs_richardson_fd("dense"),
    "fd_parity": lambda: pins.test_p10_adjoint_vs_richardson_fd("parity"),
    "grad_closed": pins.test_p10_adjoint_vs_closed_form_derivative,
    "subset_port": pins.test_quality_subset_and_portfolio_small_cases,
    "port_hand": pins.test_portfolio_two_assets_hand_computed,
    "subspace": pins.test_subspace_count,
    "qubo_reduce": pins.test_qubo_reduces_to_maxcut_subset_and_portfolio,
    "qubo_bits": pins.test_qubo_reads_upper_triangle_and_bit_order,
    "qubo_fixed": pins.test_qubo_fixed_point_rule,
    "z_bits": pins.test_pauli_z_diag_bit_order,
    "ex_equal": pins.test_exqaoa_equal_gammas_is_qaoa,
    "ex_dense": pins.test_exqaoa_vs_dense_expm,
    "ex_fd": pins.test_exqaoa_gradient_vs_richardson_fd,
    "bfgs": pins.test_bfgs_quadratic_and_rosenbrock,
    "bfgs_stop": pins.test_bfgs_stops_on_precision_loss_at_the_best_point,
    "optimise": pins.test_optimise_qaoa_matches_scipy_bfgs_and_closed_form,
    "benchmark": pins.test_benchmark_depth_sweep_with_persisted_parameters,
}

# (function, text in its source, the planted replacement, pins expected to notice)
MUTANTS = {
    # qualities
    "maxcut counts cut edges": ("maxcut_quality", "same = (bu == bv)", "same = (bu != bv)", ["ex1", "ex1_q", "p1_closed"]),
    "maxcut least significant bit first": ("maxcut_quality", "(n - 1 - int(eu[e]))", "int(eu[e])", ["ex1_q", "qubo_reduce", "p1_amp"]),
    "maxcut drops the weights": ("maxcut_quality", "1.0 if w is None else float(w[e])", "1.0", ["p1_closed", "qubo_reduce"]),
    "subset least significant bit first": ("subset_quality", "(n - 1 - b)", "b", ["subset_port", "qubo_reduce"]),
    "qubit_bits least significant bit first": ("qubit_bits", "(n - 1 - u)", "u", ["port_hand", "qubo_bits", "z_bits"]),
    "portfolio long and short swapped": ("portfolio_quality", "x[2 * a] - x[2 * a + 1]", "x[2 * a + 1] - x[2 * a]", ["subset_port", "port_hand"]),
    "portfolio covariance index": ("portfolio_quality", "z[i] * z[j]", "z[i] * z[i]", ["port_hand", "qubo_reduce"]),
    "portfolio return sign": ("portfolio_quality", "q -= (1.0 - omega)", "q += (1.0 - omega)", ["subset_port", "port_hand"]),
    "subspace keeps other weights": ("subspace_states", "pc == k", "pc >= k", ["subspace", "xy_expm"]),
    "qubo reads J transposed": ("qubo_quality", "float(J[u][v])", "float(J[v][u])", ["qubo_bits", "qubo_reduce"]),
    "qubo drops the constant": ("qubo_quality", "np.full(N, float(c)", "np.full(N, 0.0", ["qubo_reduce", "qubo_bits"]),
    "qubo reads the diagonal": ("qubo_quality", "for v in range(u + 1, n):\n            q +=", "for v in range(u, n):\n            q +=", ["qubo_bits"]),
    "fixed point truncates": ("qubo_fixed_point", "math.floor(y + 0.5)", "math.floor(y)", ["qubo_fixed"]),
    "fixed point drops the margin": ("qubo_fixed_point", "S * 2.0 ** F + 1024.0 > 2.0 ** 30", "S * 2.0 ** F > 2.0 ** 30", ["qubo_fixed"]),
    "fixed point drops J": ("qubo_quality_fixed", "qi += Ji[u][v] * x[u] * x[v]", "pass", ["qubo_fixed"]),
    # unitaries
    "phase sign": ("phase", "- 1j * np.sin", "+ 1j * np.sin", ["ex1", "p1_closed", "ansatz_dense"]),
    "hypercube rotation sign": ("mix_hypercube", "c * a0 - 1j * s * a1", "c * a0 + 1j * s * a1", ["hc_expm", "ansatz_dense"]),
    "hypercube drops a qubit": ("mix_hypercube", "for b in range(n):", "for b in range(n - 1):", ["hc_expm", "ex1"]),
    "hypercube wrong partner": ("mix_hypercube", "c * a1 - 1j * s * a0", "c * a1 - 1j * s * a1", ["hc_expm", "norm"]),
    "hypercube W drops a qubit": ("apply_hypercube_W", "for b in range(n):", "for b in range(n - 1):", ["hc_expm", "fd_hc"]),
    "circulant offset off by one": ("circulant_first_row_from_offsets", "s = int(s) % N", "s = (int(s) + 1) % N", ["circ_eigs"]),
    "circulant eigenvalue index": ("circulant_eigenvalues", "((j * int(k)) % M)", "(((j + 1) * int(k)) % M)", ["circ_eigs", "circ_expm", "complete"]),
    "circulant printed +i t Lambda": ("mix_circulant", "np.exp(-1j * t * lam)", "np.exp(1j * t * lam)", ["circ_expm", "complete"]),
    "circulant transform unnormalised": ("mix_circulant", "np.fft.fft(psi))", "np.fft.fft(psi) / len(psi))", ["circ_expm", "norm"]),
    "circulant W eigenvalues reversed": ("apply_circulant_W", "lam * np.fft.fft(psi)", "lam[::-1] * np.fft.fft(psi)", ["circ_expm", "fd_circ"]),
    "xy ring without its closing pair": ("xy_ring_apply", "for a in range(n):", "for a in range(n - 1):", ["xy_expm"]),
    "xy ring pair factor 1": ("xy_ring_apply", "np.add.at(out, dst, 2.0 * psi[src])", "np.add.at(out, dst, psi[src])", ["xy_expm", "givens"]),
    "xy series sign": ("mix_xy_ring", "(-1j * tau / m)", "(1j * tau / m)", ["xy_expm", "givens"]),
    "xy series truncated": ("mix_xy_ring", "m > 60", "m > 2", ["xy_expm", "dense_forms"]),
    "dense mixer transposed eigenvectors": ("mix_dense", "(V.T @ np.asarray(psi", "(V @ np.asarray(psi", ["dense_forms"]),
    # parity-ring mixer
    "parity without closing pairs": ("parity_ring_rounds", "if N >= 2:", "if False:", ["parity_geom", "parity_state"]),
    "parity odd and even swapped": ("parity_ring_rounds", "rounds[0 if k % 2 == 1 else 1]", "rounds[1 if k % 2 == 1 else 0]", ["parity_geom"]),
    "parity pair factor 1": ("xy_pairs_apply", "2.0 * psi[", "psi[", ["parity_dense", "fd_parity"]),
    "parity Givens angle t": ("xy_pairs_exp", "math.cos(2.0 * t), math.sin(2.0 * t)", "math.cos(t), math.sin(t)", ["parity_dense", "parity_geom"]),
    "parity Givens sign": ("xy_pairs_exp", "out[hi] = c * b - 1j * s * a", "out[hi] = c * b + 1j * s * a", ["parity_dense", "norm"]),
    "parity factors reversed": ("mix_parity", "parity_ring_rounds(n):", "parity_ring_rounds(n)[::-1]:", ["parity_dense"]),
    "parity state last assets": ("parity_state", "if a < A:", "if a >= M - A:", ["parity_state"]),
    "parity state |10>": ("parity_state", "pair[0b01] = 1.0", "pair[0b10] = 1.0", ["parity_state"]),
    # ansatz and objective
    "layer mixes before the phase": ("evolve", "psi = phase(psi, prob.q, float(g))\n        psi = prob.mix(psi, float(t))",
                                     "psi = prob.mix(psi, float(t))\n        psi = phase(psi, prob.q, float(g))", ["ex1", "ansatz_dense"]),
    "gamma and t swapped": ("evolve", "zip(gammas, ts)", "zip(ts, gammas)", ["ex1", "p1_closed"]),
    "expectation drops the imaginary part": ("expectation", "psi.real ** 2 + psi.imag ** 2", "psi.real ** 2", ["ex1", "p1_closed"]),
    # adjoint gradient
    "dt from the layer input": ("gradient", "prob.apply_W(psis[k])", "prob.apply_W(phis[k])", ["fd_hc", "fd_circ", "fd_xy"]),
    "dgamma from the layer output": ("gradient", "prob.q * phis[k]).imag", "prob.q * psis[k]).imag", ["fd_hc", "fd_circ", "grad_closed"]),
    "lambda without Q": ("gradient", "lam = prob.q * psi\n", "lam = psi.copy()\n", ["fd_hc", "grad_closed"]),
    "dgamma sign": ("gradient", "dg[k] = 2.0 *", "dg[k] = -2.0 *", ["fd_hc", "grad_closed"]),
    "mixer adjoint not inverted": ("gradient", "lam = prob.mix(lam, -float(ts[k]))", "lam = prob.mix(lam, float(ts[k]))", ["fd_hc", "fd_circ", "fd_dense"]),
    "phase adjoint not inverted": ("gradient", "lam = phase(lam, prob.q, -float(gammas[k]))", "lam = phase(lam, prob.q, float(gammas[k]))", ["fd_hc", "fd_dense"]),
    "factored adjoint in forward order": ("_gradient_factored", "for fi in range(len(rounds) - 1, -1, -1):", "for fi in range(len(rounds)):", ["fd_parity"]),
    "factored dt at the layer input": ("_gradient_factored", "xy_pairs_apply(outs[k][fi]", "xy_pairs_apply(phis[k]", ["fd_parity"]),
    "finite differences without Richardson": ("central_fd", "(4 * d(True, k, h / 2) - d(True, k, h)) / 3", "d(True, k, h)", ["fd_hc", "fd_dense"]),
    "finite differences one-sided scale": ("central_fd", "/ (2 * hh)", "/ hh", ["fd_hc", "fd_dense"]),
    # ex-QAOA
    "Z is -1 on |0>": ("pauli_z_diag", "1.0 - 2.0 * x[u].astype(np.float64)", "2.0 * x[u].astype(np.float64) - 1.0", ["z_bits"]),
    "pair term reads u twice": ("exqaoa_term_diags", "int(tu[j]), int(tv[j])", "int(tu[j]), int(tu[j])", ["ex_equal", "ex_dense"]),
    "ex phase sign": ("exqaoa_phase", "np.exp(-1j * float(gam[j]) * S)", "np.exp(1j * float(gam[j]) * S)", ["ex_dense", "ex_equal"]),
    "ex first layer's gammas reused": ("exqaoa_evolve", "exqaoa_phase(psi, terms, G[k])", "exqaoa_phase(psi, terms, G[0])", ["ex_dense"]),
    "ex dgamma with Q": ("exqaoa_gradient", "terms[j] * phis[k]", "prob.q * phis[k]", ["ex_fd", "ex_equal"]),
    "ex phase adjoint not inverted": ("exqaoa_gradient", "exqaoa_phase(lam, terms, -np.asarray(G[k]", "exqaoa_phase(lam, terms, np.asarray(G[k]", ["ex_fd", "ex_equal"]),
    # optimiser and depth sweep
    "bfgs steepest descent": ("bfgs_minimize", "d = -H @ g\n", "d = -g\n", ["bfgs"]),
    "bfgs loose stop": ("bfgs_minimize", "if np.max(np.abs(g)) <= gtol:\n            stop = 0\n            break",
                        "if np.max(np.abs(g)) <= 1e3 * gtol:\n            stop = 0\n            break", ["bfgs"]),
    "bfgs takes the failed trial point": ("bfgs_minimize", "            stop = 2\n            break",
                                          "            stop = 2\n            x, f, g = xn, fn, np.asarray(gn, dtype=np.float64)\n            break",
                                          ["bfgs_stop"]),
    "optimise swaps gamma and t": ("optimise", "gs, ts = th[0::2], th[1::2]", "gs, ts = th[1::2], th[0::2]", ["optimise", "benchmark"]),
    "benchmark persists the first repeat": ("benchmark", "results[int(np.argmin(row))]", "results[0]", ["benchmark"]),
    "benchmark new layer gamma and t swapped": ("benchmark", "init[pos + 2 * r])", "init[pos + 2 * r + 1])", ["benchmark"]),
    "optimise packs the start swapped": ("optimise", "th0[0::2] = gammas0\n    th0[1::2] = ts0", "th0[0::2] = ts0\n    th0[1::2] = gammas0",
                                         ["optimise", "benchmark"]),
    # corners: the uniform state, signs, weights, problem builders
    "uniform state unnormalised": ("Problem.initial_state", "1.0 / math.sqrt(self.dim)", "1.0 / self.dim", ["norm", "ex1"]),
    "fixed point drops the sign": ("qubo_fixed_point", "return int(r) if x >= 0 else -int(r)", "return int(r)", ["qubo_fixed"]),
    "circulant eigenvalues drop the weights": ("circulant_eigenvalues", "lam += first_row[k] * np.cos", "lam += np.cos", ["circ_expm"]),
    "factored dgamma sign": ("_gradient_factored", "dg[k] = 2.0 *", "dg[k] = -2.0 *", ["fd_parity"]),
    "finite differences in t without Richardson": ("central_fd", "(4 * d(False, k, h / 2) - d(False, k, h)) / 3", "d(False, k, h)", ["fd_hc", "fd_dense"]),
    "parity Givens on reversed bits": ("xy_pairs_exp", "bu, bv = n - 1 - u, n - 1 - v", "bu, bv = u, v", ["parity_dense"]),
    "maxcut problem drops the weights": ("maxcut_problem", "maxcut_quality(n, eu, ev, w)", "maxcut_quality(n, eu, ev)", ["p1_closed"]),
    "qwoa problem drops an offset": ("qwoa_problem", "circulant_first_row_from_offsets(N, offsets)",
                                     "circulant_first_row_from_offsets(N, list(offsets)[1:])", ["circ_eigs"]),
    "parity problem starts uniform": ("qaoaz_parity_problem", "psi0=parity_state(n, A)", "psi0=None", ["parity_state"]),
    "qaoaz problem on the wrong weight": ("qaoaz_problem", "subspace_states(n, k)", "subspace_states(n, k - 1)", ["subspace"]),
}


def _owner(name):
    """(object holding the function, attribute name): the module, or a class of it ("Cls.meth")."""
    if "." in name:
        cls, attr = name.split(".")
        return getattr(orc, cls), attr
    return orc, name


def _planted(name, old=None, new=None):
    owner, attr = _owner(name)
    src = textwrap.dedent(inspect.getsource(getattr(owner, attr)))
    if old is not None:
        assert src.count(old) == 1, f"{name}: the text to replace must occur exactly once"
        src = src.replace(old, new)
    ns = dict(vars(orc))
    code = compile(src, f"<oracle.{name} with a planted mistake>", "exec",
                   flags=__future__.annotations.compiler_flag, dont_inherit=True)
    exec(code, ns)
    return ns[attr]


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_pins_catch_planted_mistake(mutant, monkeypatch):
    name, old, new, which = MUTANTS[mutant]
    monkeypatch.setattr(*_owner(name), _planted(name, old, new))
    caught = []
    for pin in which:
        try:
            with np.errstate(all="ignore"):
                PINS[pin]()
        except AssertionError:
            caught.append(pin)
    assert caught, f"no pin among {which} noticed: {mutant}"


def test_unplanted_rebuild_passes_every_pin(monkeypatch):
    """Rebuilding every mutated function from its unchanged source changes nothing: the pins used
    above all pass, so a failure above comes from the planted mistake alone."""
    for name in sorted({m[0] for m in MUTANTS.values()}):
        monkeypatch.setattr(*_owner(name), _planted(name))
    for pin in sorted({p for m in MUTANTS.values() for p in m[3]}):
        PINS[pin]()
