"""Host-side argument checks of the Python binding: the library receives bare pointers and reads or
writes a fixed number of elements, so a buffer that is too short, of another dtype, not contiguous
or on the wrong side is refused (QvsError, QVS_EINVAL) before any library call."""
import numpy as np
import pytest

import paper_2110_03963_gb300 as qvs


def _refused(fn, *args, **kw):
    with pytest.raises(qvs.QvsError) as e:
        fn(*args, **kw)
    assert e.value.status == qvs.QVS_EINVAL


def test_check_buffer_rules():
    x = np.zeros(16, np.float32)
    qvs._check_buffer(x, 16, {"float32"}, "x")
    qvs._check_buffer(x, 8, {"float32"}, "x")                      # at least 8
    _refused(qvs._check_buffer, x, 8, {"float32"}, "x", exact=True)  # exactly 8
    _refused(qvs._check_buffer, x, 17, {"float32"}, "x")
    _refused(qvs._check_buffer, x, 16, {"float64"}, "x")
    _refused(qvs._check_buffer, x, 16, {"float32"}, "x", device=True)
    _refused(qvs._check_buffer, np.zeros((4, 8), np.float32)[:, ::2], 16, {"float32"}, "x")
    _refused(qvs._check_buffer, [0.0] * 16, 16, {"float32"}, "x")


def test_generators_refuse_host_or_short_outputs():
    eu, ev = np.array([0, 1], np.int32), np.array([1, 2], np.int32)
    _refused(qvs.qvs_quality_maxcut, 3, eu, ev, None, np.zeros(8, np.int32), qvs.QVS_I32)     # host
    _refused(qvs.qvs_quality_subset, 3, np.ones(3), np.zeros(8, np.float32), qvs.QVS_F32)    # host
    _refused(qvs.qvs_state_parity, 4, 1, np.zeros(16, np.complex64))                         # host
    _refused(qvs.qvs_quality_qubo, 2, 0.0, np.zeros(2), np.zeros((2, 2)), np.zeros(4, np.float32),
             qvs.QVS_F32)
    _refused(qvs._quality_dtype, 99)


def test_csr_desc_checks_its_arrays():
    rowptr, colind = np.array([0, 1, 2], np.int64), np.array([1, 0], np.int32)
    d = qvs.csr_desc(rowptr, colind, None, 2.0)
    assert d.nnz == 2 and d.csr_on_device == 0
    _refused(qvs.csr_desc, rowptr.astype(np.int32), colind, None, 2.0)
    _refused(qvs.csr_desc, rowptr, colind.astype(np.int64), None, 2.0)
    _refused(qvs.csr_desc, rowptr, colind, np.ones(3, np.float32), 0.0)     # one value per nonzero


class _FakeLib:
    """Stands in for libqvs: records each call and returns QVS_OK; qvs_create and qvs_batch_create
    hand out distinct fake handles. A buffer check that let a bad buffer through would show up as a
    recorded call where the test expects none."""

    def __init__(self):
        self.calls = []
        self.next = 0x1000

    def __getattr__(self, name):
        if name == "qvs_strerror":
            return lambda status: b"fake status"
        def fn(*args):
            self.calls.append(name)
            if name in ("qvs_create", "qvs_batch_create"):
                args[0]._obj.value = self.next
                self.next += 0x100
            return 0
        return fn


@pytest.fixture
def fake(monkeypatch):
    lib = _FakeLib()
    monkeypatch.setattr(qvs, "_lib", lib)
    monkeypatch.setattr(qvs, "_HANDLES", {})
    monkeypatch.setattr(qvs, "_BATCHES", {})
    return lib


def _passes(lib, name, fn, *args, **kw):
    before = len(lib.calls)
    fn(*args, **kw)
    assert name in lib.calls[before:]


def _refused_before_library(lib, fn, *args, **kw):
    before = len(lib.calls)
    _refused(fn, *args, **kw)
    assert lib.calls[before:] == []


def test_handle_buffers_are_sized_by_the_handle(fake):
    h = qvs.qvs_create(16, qvs.QVS_C64)
    _passes(fake, "qvs_set_quality", qvs.qvs_set_quality, h, np.zeros(16, np.int32))
    _passes(fake, "qvs_set_quality", qvs.qvs_set_quality, h, np.zeros(16, np.float64), qvs.QVS_F64)
    _refused_before_library(fake, qvs.qvs_set_quality, h, np.zeros(8, np.float32))
    _refused_before_library(fake, qvs.qvs_set_quality, h, np.zeros(16, np.float32), qvs.QVS_F64)
    _refused_before_library(fake, qvs.qvs_set_quality, h, np.zeros(16, np.int64))
    _passes(fake, "qvs_set_initial_state", qvs.qvs_set_initial_state, h, np.zeros(16, np.complex64))
    _passes(fake, "qvs_set_initial_state", qvs.qvs_set_initial_state, h, None)
    _refused_before_library(fake, qvs.qvs_set_initial_state, h, np.zeros(16, np.complex128))
    _refused_before_library(fake, qvs.qvs_set_initial_state, h, np.zeros(15, np.complex64))
    _passes(fake, "qvs_get_state", qvs.qvs_get_state, h, np.zeros(16, np.complex64))
    _refused_before_library(fake, qvs.qvs_get_state, h, np.zeros(8, np.complex64))
    _refused_before_library(fake, qvs.qvs_get_state, h, np.zeros(16, np.complex128))
    h2 = qvs.qvs_create(16, qvs.QVS_C128)
    _passes(fake, "qvs_get_state", qvs.qvs_get_state, h2, np.zeros(16, np.complex128))
    _refused_before_library(fake, qvs.qvs_get_state, h2, np.zeros(16, np.complex64))
    qvs.qvs_destroy(h)
    _refused_before_library(fake, qvs.qvs_get_state, h, np.zeros(16, np.complex64))   # destroyed
    _refused_before_library(fake, qvs.qvs_get_state, None, np.zeros(16, np.complex64))


def test_ex_qaoa_parameters_match_the_terms(fake):
    h = qvs.qvs_create(1 << 13, qvs.QVS_C64)
    _passes(fake, "qvs_evolve_ex", qvs.qvs_evolve_ex, h, np.zeros((1, 1)), [0.1])   # no terms: library decides
    _refused_before_library(fake, qvs.qvs_set_phase_terms, h, [0, 1], [1], [1.0, 2.0])
    _passes(fake, "qvs_set_phase_terms", qvs.qvs_set_phase_terms, h, [0, 1, 2], [1, -1, 5], [1.0, 2.0, 0.5])
    _passes(fake, "qvs_gradient_ex", qvs.qvs_gradient_ex, h, np.zeros((2, 3)), [0.1, 0.2])
    _refused_before_library(fake, qvs.qvs_gradient_ex, h, np.zeros((2, 2)), [0.1, 0.2])
    _refused_before_library(fake, qvs.qvs_evolve_ex, h, np.zeros((1, 3)), [0.1, 0.2])


def test_edge_lists_have_one_length(fake):
    _refused_before_library(fake, qvs.qvs_qubo_from_maxcut, 4, [0, 1], [1], None)
    _refused_before_library(fake, qvs.qvs_qubo_from_maxcut, 4, [0, 1], [1, 2], [1.0])
    _passes(fake, "qvs_qubo_from_maxcut", qvs.qvs_qubo_from_maxcut, 4, [0, 1], [1, 2], [1.0, 0.5])


def test_batch_buffers_are_sized_by_the_batch(fake):
    b = qvs.qvs_batch_create([12, 13], [2, 3])
    _passes(fake, "qvs_batch_set_quality", qvs.qvs_batch_set_quality, b, np.zeros(4096 + 8192, np.float32))
    _refused_before_library(fake, qvs.qvs_batch_set_quality, b, np.zeros(4096 * 2, np.float32))
    _refused_before_library(fake, qvs.qvs_batch_set_quality, b, np.zeros(4096 + 8192, np.float64))
    _passes(fake, "qvs_batch_gradient", qvs.qvs_batch_gradient, b, np.zeros(5), np.zeros(5), 2)
    _refused_before_library(fake, qvs.qvs_batch_gradient, b, np.zeros(4), np.zeros(4), 2)
    _refused_before_library(fake, qvs.qvs_batch_gradient, b, np.zeros(5), np.zeros(5), 3)
    _passes(fake, "qvs_batch_optimise", qvs.qvs_batch_optimise, b, np.zeros(5), np.zeros(5), 2)
    _refused_before_library(fake, qvs.qvs_batch_optimise, b, np.zeros(6), np.zeros(6), 2)
    _refused_before_library(fake, qvs.qvs_batch_create, [12, 13], [2])
    bs = qvs.qvs_batch_create([12, 12, 12], [1, 2, 3])
    _passes(fake, "qvs_batch_set_quality_shared", qvs.qvs_batch_set_quality_shared, bs, np.zeros(4096, np.float32))
    _refused_before_library(fake, qvs.qvs_batch_set_quality_shared, bs, np.zeros(2048, np.float32))
    qvs.qvs_batch_destroy(b)
    _refused_before_library(fake, qvs.qvs_batch_gradient, b, np.zeros(5), np.zeros(5), 2)
    # the depth sweep reads 2^n fp32 qualities
    init = np.zeros(2 * 2 * 1 + 2 * 2)
    _passes(fake, "qvs_benchmark", qvs.qvs_benchmark, 12, np.zeros(4096, np.float32), 1, 2, 2, init)
    _refused_before_library(fake, qvs.qvs_benchmark, 12, np.zeros(2048, np.float32), 1, 2, 2, init)


def test_mixer_descriptions():
    d = qvs.circulant_desc([1, 2, 4], [0.5, 1.0, 2.0])
    assert d.n_offsets == 3 and [d.offsets[i] for i in range(3)] == [1, 2, 4]
    assert [d.offset_weights[i] for i in range(3)] == [0.5, 1.0, 2.0]
    assert not qvs.circulant_desc([1, 2]).offset_weights          # NULL: every weight 1
    _refused(qvs.circulant_desc, [1, 2, 4], [0.5, 1.0])            # one weight per offset
    d = qvs.xy_ring_desc(24, 12, (-31.0, 31.0), 1e-8)
    assert (d.n_qubits, d.hamming_weight, d.spec_lo, d.spec_hi, d.cheb_tol) == (24, 12, -31.0, 31.0, 1e-8)
    assert qvs.hypercube_desc(28).n_qubits == 28 and qvs.parity_desc(26).n_qubits == 26
    rowptr, colind = np.array([0, 1, 2], np.int64), np.array([1, 0], np.int32)
    d = qvs.csr_desc(rowptr, colind, np.full(2, 2.0, np.float32), 0.0, (-2.0, 2.0))
    assert (d.nnz, d.csr_on_device, d.spec_lo, d.spec_hi) == (2, 0, -2.0, 2.0) and d.values


def test_generator_inputs_have_the_sizes_the_library_reads(fake):
    def refused_for(what, fn, *args):
        before = len(fake.calls)
        with pytest.raises(qvs.QvsError) as e:
            fn(*args)
        assert e.value.status == qvs.QVS_EINVAL and what in str(e.value) and fake.calls[before:] == []
    refused_for("item weights", qvs.qvs_quality_subset, 4, np.ones(3), np.zeros(16, np.float32), qvs.QVS_F32)
    states = np.arange(16, dtype=np.int64)
    out = np.zeros(16, np.float32)
    refused_for("assets", qvs.qvs_quality_portfolio, 4, states, [1.0], np.eye(2), 0.5, out, qvs.QVS_F32)
    refused_for("assets", qvs.qvs_quality_portfolio, 4, states, [1.0, 2.0], np.eye(3), 0.5, out, qvs.QVS_F32)


def test_batch_parameters_per_instance(fake):
    b = qvs.Batch([12, 13], [2, 3])
    good_g, good_t = [np.zeros(2), np.zeros(3)], [np.zeros(2), np.zeros(3)]
    _passes(fake, "qvs_batch_gradient", b.gradient, good_g, good_t)
    # the right total (5) split 3 + 2 across the instances is refused, as is a missing instance
    _refused_before_library(fake, b.gradient, [np.zeros(3), np.zeros(2)], [np.zeros(3), np.zeros(2)])
    _refused_before_library(fake, b.optimise, [np.zeros(2)], [np.zeros(2)])
    _refused_before_library(fake, qvs.qvs_quality_qubo, 3, 0.0, np.zeros(3), np.zeros((2, 2)),
                            np.zeros(8, np.float32), qvs.QVS_F32)
    b.close()   # while the stand-in is in place: the fake handle must never reach the real library
