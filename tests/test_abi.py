"""The C ABI without a GPU: librbffd builds for sm_103a, loads, exports every
entry point that include/rbffd.h declares, and rejects bad arguments before
touching the device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1509_02615_gb300 import _build, rbffd
    _build.build()
    return rbffd.lib()


def _declared():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(rbf_\w+)\s*\(", src)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "rbf_build_weights" in names and "rbf_rk4_step" in names and "rbf_run" in names
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    from paper_1509_02615_gb300 import rbffd
    bound = {s[0] for s in rbffd.SIGNATURES}
    assert set(_declared()) <= bound


def test_argument_errors_need_no_gpu(lib):
    from paper_1509_02615_gb300 import rbffd
    # n = 0 is rejected by the argument checks before any CUDA call
    rc = lib.rbf_build_stencils(None, None, 10, 10, 0, 0.0, None, None)
    assert rc == rbffd.RBF_E_ARG
    assert b"stencil size" in lib.rbf_last_error()
    rc = lib.rbf_build_weights(None, None, 10, None, 5, 37, 0.0, 4, 4, 0, None, 1, None, None)
    assert rc == rbffd.RBF_E_ARG
    rc = lib.rbf_rk4_step(None, 0.0, 1.0, None)
    assert rc == rbffd.RBF_E_ARG
    # an ensemble's lanes per node: 0 (autotune), 1, 2 or 4
    common = rbffd.NSParams(n_sten=37, phs_p=7, poly_l=4, hv_k=3, hv_p=7, precision=32, threads_per_node=3)
    mem = (rbffd.EnsMember * 1)(rbffd.EnsMember(n_prog=4, n_all=8, n_sten=37, poly_l=4, dt=1.0, n_steps=1))
    buf = (C.c_double * 8)()
    ibuf = (C.c_int32 * 8)()
    h = C.c_void_p()
    rc = lib.rbf_ens_create(C.byref(h), C.byref(common), 1, mem, buf, buf, ibuf, ibuf, None)
    assert rc == rbffd.RBF_E_ARG and not h.value
    assert b"threads per node" in lib.rbf_last_error()


def test_struct_layouts_match_header():
    from paper_1509_02615_gb300 import rbffd
    # 8 int32 + 8 doubles; 6 int32 + 2 doubles; see include/rbffd.h
    assert C.sizeof(rbffd.NSParams) == 8 * 4 + 8 * 8
    assert C.sizeof(rbffd.AdvParams) == 6 * 4 + 2 * 8
    assert C.sizeof(rbffd.Info) == 3 * 8 + 10 * 4 + 4 * 8 + 6 * 4
