"""Allocation-free field read (lbpm_read_field_noalloc) against lbpm_read_field.

Some callers cannot let the library allocate device memory once their set-up
is done: a loop running under a fixed device-memory budget handed out at
start-up, or a host that must not enter the allocator while other work owns
it. They read fields through the allocation-free entry point, which must
return exactly what the regular field read returns. Two calls in a row check
that the shared static staging array carries nothing over from one call to
the next, a larger image read before a smaller one checks that no stale entry
of the larger read survives, and PyTorch's allocation counter (every device
allocation of a Domain goes through PyTorch's caching allocator) checks that
the call allocates nothing. This file is collected last so that a
stop-at-first-failure run has run every other test before it.
"""
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


def _allocations(torch):
    return torch.cuda.memory_stats(0).get("allocation.all.allocated", 0)


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_noalloc_field_read_matches_regular_on_two_calls(precision):
    import torch

    import paper_2007_12266_gb300 as lbm
    from paper_2007_12266_gb300 import _lib
    from synthetic import workload_parity32
    lib = _lib.load()
    w = workload_parity32()
    dom = lbm.Domain(w.labels, w.affinity, periodic=w.periodic, precision=precision, **KW)
    dom.init_fluids(w.phi0)
    dom.advance(5)
    torch.cuda.synchronize()
    # call 1: phase field; the library allocates nothing during it
    n0 = _allocations(torch)
    a = _noalloc(lib, dom, lbm.FIELDS["phi"])
    assert _allocations(torch) == n0
    b = _regular(lib, dom, lbm.FIELDS["phi"])
    assert _allocations(torch) > n0                # the regular read does allocate (the counter sees it)
    np.testing.assert_array_equal(a, b)            # same kernels: identical, NaN at solids
    assert np.isfinite(a[w.labels == 0]).all() and np.isnan(a[w.labels != 0]).all()
    # call 2, right after (a different field, after more steps)
    dom.advance(3)
    n1 = _allocations(torch)
    c = _noalloc(lib, dom, lbm.FIELDS["uz"])
    assert _allocations(torch) == n1
    d = _regular(lib, dom, lbm.FIELDS["uz"])
    np.testing.assert_array_equal(c, d)
    assert not np.array_equal(np.nan_to_num(a), np.nan_to_num(c))
    dom.close()


def test_noalloc_field_read_of_a_smaller_image_after_a_larger_one():
    import paper_2007_12266_gb300 as lbm
    from paper_2007_12266_gb300 import _lib
    from synthetic import phi0_iid, random_affinity, sphere_pack
    lib = _lib.load()
    reads = []
    for L, seed in ((48, 11), (20, 12)):             # both within the array's limit
        sp = sphere_pack(L, 0.4, 3.0, 1.0, seed)
        dom = lbm.Domain(sp.labels, random_affinity(sp.labels, -0.5, 0.5, seed + 1), periodic=(1, 1, 1), **KW)
        dom.init_fluids(phi0_iid(sp.labels, 0.5, seed + 2))
        dom.advance(4)
        a = _noalloc(lib, dom, lbm.FIELDS["pressure"])
        np.testing.assert_array_equal(a, _regular(lib, dom, lbm.FIELDS["pressure"]))
        assert np.isnan(a[sp.labels != 0]).all() and np.isfinite(a[sp.labels == 0]).all()
        reads.append(a)
        dom.close()
    assert reads[1].size < reads[0].size


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
