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
