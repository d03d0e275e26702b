"""The allocation-free stencil builder (rbf_build_stencils_static).

It serves callers that must not allocate device memory: a framework whose
memory pool owns the GPU, a fixed device-memory budget, or a loop that cannot
take cudaMalloc's implicit device synchronisation.  Its scratch lives in one
static device array.  This test calls it through the C ABI twice in a row, on
two different node sets, and requires the same index lists as the
allocating entry point rbf_build_stencils (stencils are integer output:
bit-exact, as in the other stencil tests).  The file name makes pytest
collect it last.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1509_02615_gb300 import inputs as inp  # noqa: E402
from paper_1509_02615_gb300 import rbffd  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    from paper_1509_02615_gb300 import _build
    _build.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return rbffd.lib()


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _static(lib, nodes, n):
    x, z = _dev(nodes.x), _dev(nodes.z)
    idx = torch.full((nodes.n_prog, n), -7, dtype=torch.int32, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.rbf_build_stencils_static(C.c_void_p(x.data_ptr()), C.c_void_p(z.data_ptr()), nodes.n_all,
                                       nodes.n_prog, n, float(nodes.period_x), C.c_void_p(idx.data_ptr()), stream)
    assert rc == rbffd.RBF_OK, lib.rbf_last_error()
    return idx


def test_static_stencils_match_allocating_entry_point_twice(lib):
    cases = [(inp.density_current_nodes(200.0), 37),
             (inp.poisson_disk_nodes(0.0, 20.0, 0.0, 10.0, 0.4, seed=11), 56)]
    for nodes, n in cases:   # two calls in a row, different sizes and layouts
        ref = rbffd.build_stencils(_dev(nodes.x), _dev(nodes.z), nodes.n_prog, n, nodes.period_x)
        got = _static(lib, nodes, n)
        torch.cuda.synchronize()
        assert torch.equal(got, ref)


def test_static_stencils_reject_oversize_input(lib):
    n_all = 262144 + 1
    rc = lib.rbf_build_stencils_static(None, None, n_all, 10, 37, 0.0, None, None)
    assert rc == rbffd.RBF_E_ARG
    assert b"static scratch limit" in lib.rbf_last_error()
