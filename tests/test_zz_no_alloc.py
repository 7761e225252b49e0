"""Allocation-free field read (lbpm_read_field_noalloc) against lbpm_read_field.

Callers that cannot let the library allocate device memory after set-up use
the allocation-free entry point; it must return exactly what the regular
field read returns. Two calls in a row check that the shared static staging
buffer carries nothing over from one call to the next. This file is collected
last so that a stop-at-first-failure run has run every other test before it.
"""
import ctypes as ct

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

KW = dict(tau_a=0.7, tau_b=0.7, alpha=0.005, beta=0.95, force=(0.0, 0.0, 1e-5))


def _noalloc(lib, dom, code):
    out = np.empty(dom.shape, dtype=np.float32)
    st = lib.lbpm_read_field_noalloc(dom._h, code, out.ctypes.data)
    assert st == 0, lib.lbpm_last_error(dom._h).decode()
    return out


def _regular(lib, dom, code):
    out = np.empty(dom.shape, dtype=np.float32)
    assert lib.lbpm_read_field(dom._h, code, out.ctypes.data) == 0
    return out


def test_noalloc_field_read_matches_regular_on_two_calls():
    import paper_2007_12266_gb300 as lbm
    from paper_2007_12266_gb300 import _lib
    from synthetic import workload_parity32
    lib = _lib.load()
    w = workload_parity32()
    dom = lbm.Domain(w.labels, w.affinity, periodic=w.periodic, **KW)
    dom.init_fluids(w.phi0)
    dom.advance(5)
    # call 1: phase field
    a = _noalloc(lib, dom, lbm.FIELDS["phi"])
    b = _regular(lib, dom, lbm.FIELDS["phi"])
    np.testing.assert_array_equal(a, b)            # same kernels: identical, NaN at solids
    assert np.isfinite(a[w.labels == 0]).all() and np.isnan(a[w.labels != 0]).all()
    # call 2, right after (a different field, after more steps)
    dom.advance(3)
    c = _noalloc(lib, dom, lbm.FIELDS["uz"])
    d = _regular(lib, dom, lbm.FIELDS["uz"])
    np.testing.assert_array_equal(c, d)
    assert not np.array_equal(np.nan_to_num(a), np.nan_to_num(c))
    dom.close()


def test_noalloc_field_read_rejects_oversize_image():
    import paper_2007_12266_gb300 as lbm
    from paper_2007_12266_gb300 import _lib
    lib = _lib.load()
    n = 130                                          # 130^3 > 2^21 voxels
    lab = np.ones((n, n, n), np.uint16)
    lab[1:-1, 1:-1, 1:-1] = 0
    dom = lbm.Domain(lab, None, periodic=(0, 0, 0), **KW)
    dom.init_fluids(np.ones(lab.shape, np.float32))
    out = np.empty(lab.shape, dtype=np.float32)
    st = lib.lbpm_read_field_noalloc(dom._h, 0, out.ctypes.data)
    assert st == 1
    assert "at most" in lib.lbpm_last_error(dom._h).decode()
    dom.close()
