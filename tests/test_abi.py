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


def _c_layouts(tmp_path, structs):
    """sizeof and every field's offsetof of the header's structs, printed by a
    C program compiled against include/rbffd.h (gcc)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "rbffd.h"', "int main(void) {"]
    for cname, fields in structs.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f in fields:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    c = tmp_path / "layout.c"
    c.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {(a, b): int(v) for a, b, v in (ln.split() for ln in out.strip().splitlines())}


def test_struct_layouts_match_header(tmp_path):
    from paper_1509_02615_gb300 import rbffd
    pairs = {"rbf_ns_params": rbffd.NSParams, "rbf_adv_params": rbffd.AdvParams,
             "rbf_ens_member": rbffd.EnsMember, "rbf_info": rbffd.Info}
    got = _c_layouts(tmp_path, {c: [f for f, _ in py._fields_] for c, py in pairs.items()})
    for cname, py in pairs.items():
        assert got[(cname, "sizeof")] == C.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_hyperviscosity_gamma_needs_no_gpu(lib):
    from paper_1509_02615_gb300 import rbffd
    assert rbffd.hyperviscosity_gamma(2.0 ** -6, 100.0, 3) == pytest.approx(2.0 ** -6 * 100.0 ** 5, rel=1e-15)
    v = C.c_double()
    assert lib.rbf_hyperviscosity_gamma(1.0, 0.0, 3, C.byref(v)) == rbffd.RBF_E_ARG
    assert lib.rbf_hyperviscosity_gamma(-1.0, 1.0, 3, C.byref(v)) == rbffd.RBF_E_ARG
