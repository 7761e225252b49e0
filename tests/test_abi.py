"""C-ABI checks that need no GPU.

* the library loads and exports every function include/lbpm.h declares, and
  each declaration carries its comment;
* the Python binding declares exactly those functions;
* the ctypes structures match the C layout (sizes and offsets from gcc);
* without a GPU, lbpm_create fails with a status code instead of crashing,
  and the binding refuses to run (no CPU fallback exists).
"""
import ctypes as ct
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbpm.h")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    from paper_2007_12266_gb300 import _build
    _build.build()
    from paper_2007_12266_gb300 import _lib
    return _lib.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(lbpm_[a-z_0-9]+)\s*\(", src)
    return sorted(set(n for n in names if not n.endswith("_fn")))


def test_header_declares_expected_calls():
    names = declared_functions()
    for must in ("lbpm_create", "lbpm_load_image", "lbpm_set_affinity_table", "lbpm_set_affinity_map",
                 "lbpm_set_params", "lbpm_init_fluids", "lbpm_advance", "lbpm_measure",
                 "lbpm_read_field", "lbpm_read_distributions", "lbpm_get_index"):
        assert must in names


def test_every_declared_call_is_documented():
    """Each declaration (or group of adjacent declarations) follows a comment
    that states what the call does and how it fails."""
    lines = open(HEADER).read().split("\n")
    decl = re.compile(r"^(lbpm_status|const char\*|int|void|double|long long)\s+\**(lbpm_\w+)\(")
    undocumented = []
    for i, line in enumerate(lines):
        m = decl.match(line)
        if not m:
            continue
        j = i - 1
        while j >= 0 and decl.match(lines[j]):
            j -= 1
        prev = lines[j].strip()
        if not (prev.endswith("*/") or prev.startswith("*") or prev.startswith("/*")):
            undocumented.append(m.group(2))
    assert not undocumented, undocumented


def test_every_declared_symbol_is_exported(lib):
    from paper_2007_12266_gb300 import _lib
    names = declared_functions()
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(_lib.SIGNATURES) == names


def test_version_string(lib):
    assert lib.lbpm_version().decode().startswith("lbpm-gb300")


def _c_layout():
    prog = r"""
#include <stdio.h>
#include <stddef.h>
#include "lbpm.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(lbpm_params), offsetof(lbpm_params, precision),
         offsetof(lbpm_params, periodic), offsetof(lbpm_params, reservoir_z), offsetof(lbpm_params, rho_in));
  printf("%zu %zu %zu %zu %zu\n", sizeof(lbpm_measures), offsetof(lbpm_measures, mom_a),
         offsetof(lbpm_measures, ca), offsetof(lbpm_measures, n_sites), offsetof(lbpm_measures, status));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(prog)
        subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        out = subprocess.check_output([exe]).decode().split("\n")
    return [list(map(int, out[0].split())), list(map(int, out[1].split()))]


def test_struct_layout_matches_c():
    from paper_2007_12266_gb300._lib import Measures, Params
    p, m = _c_layout()
    assert p == [ct.sizeof(Params), Params.precision.offset, Params.periodic.offset,
                 Params.reservoir_z.offset, Params.rho_in.offset]
    assert m == [ct.sizeof(Measures), Measures.mom_a.offset, Measures.ca.offset,
                 Measures.n_sites.offset, Measures.status.offset]


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ct.c_void_p()
    st = lib.lbpm_create(ct.byref(h), 0, None)
    assert st in (1, 3)
    assert not h.value
    assert lib.lbpm_last_error(None).decode()


def test_null_arguments_are_rejected(lib):
    assert lib.lbpm_create(None, 0, None) == 1
    assert lib.lbpm_destroy(None) == 0
    assert lib.lbpm_advance(None, 1) == 1
    assert lib.lbpm_num_sites(None, None) == 1


def test_binding_refuses_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import numpy as np
    import paper_2007_12266_gb300 as lbm
    with pytest.raises(RuntimeError):
        lbm.Domain(np.zeros((4, 4, 4), np.uint16))


def test_server_struct_layout_matches_c():
    from paper_2007_12266_gb300._lib import JobSpec, JobStatus
    prog = r"""
#include <stdio.h>
#include <stddef.h>
#include "lbpm.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(lbpm_job_spec), offsetof(lbpm_job_spec, params),
         offsetof(lbpm_job_spec, kind), offsetof(lbpm_job_spec, max_steps), offsetof(lbpm_job_spec, force_cap));
  printf("%zu %zu %zu %zu\n", sizeof(lbpm_job_status), offsetof(lbpm_job_status, footprint),
         offsetof(lbpm_job_status, force_raises), offsetof(lbpm_job_status, last));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(prog)
        subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        out = subprocess.check_output([exe]).decode().split("\n")
    a = list(map(int, out[0].split()))
    b = list(map(int, out[1].split()))
    assert a == [ct.sizeof(JobSpec), JobSpec.params.offset, JobSpec.kind.offset, JobSpec.max_steps.offset,
                 JobSpec.force_cap.offset]
    assert b == [ct.sizeof(JobStatus), JobStatus.footprint.offset, JobStatus.force_raises.offset,
                 JobStatus.last.offset]
