"""Full-size parity of the advection (64^2, 1000 RK4 steps to t = T) and
warm-bubble workloads (walled box, scattered nodes, n = 56, r^9 + deg 5:
lateral-wall and corner ghost systems).

Tolerances: FP64 GPU vs FP64 oracle 1e-10 relative l2 after the stated steps
(the per-step parity of 1e-11 with RK4's mild growth); FP32 vs FP64 per-field
bounds stated in each test (eps32 ~ 6e-8 amplified by the run).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle.advection import AdvectionOracle  # noqa: E402
from oracle.ns import NSOracle  # noqa: E402
from paper_1509_02615_gb300 import configs  # noqa: E402
from paper_1509_02615_gb300 import rbffd  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1509_02615_gb300 import _build
    _build.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_advection_full_period_fp64_and_fp32():
    wl = configs.advection(64)
    o = AdvectionOracle(wl.nodes, **wl.params)
    ref = o.run(wl.U0, 0.0, wl.dt, wl.n_steps)[0]
    pb = rbffd.advection_problem(wl.nodes, precision=64, **wl.params)
    P = rbffd.state_tensor(wl.U0, 64)
    pb.run(0.0, wl.dt, wl.n_steps, P)
    got = rbffd.fields(P)[0]
    e = rel(got, ref)
    ret_gpu, ret_ref = rel(got, wl.U0), rel(ref, wl.U0)
    print(f"advection 64^2, t = T: GPU vs oracle {e:.2e}; return error GPU {ret_gpu:.6f} oracle {ret_ref:.6f}")
    assert e < 1e-10
    pb32 = rbffd.advection_problem(wl.nodes, precision=32, **wl.params)
    Q = rbffd.state_tensor(wl.U0, 32)
    pb32.run(0.0, wl.dt, wl.n_steps, Q)
    e32 = rel(rbffd.fields(Q)[0], ref)
    print(f"advection FP32 vs FP64 oracle at t = T: {e32:.2e}")
    assert e32 < 1e-4


def test_bubble_small_fp64_matches_oracle():
    wl = configs.bubble(h=500.0, seed=1, t_end=60.0)
    o = NSOracle(wl.nodes, **wl.params)
    ref = o.run(wl.U0, 0.0, wl.dt, wl.n_steps)
    pb = rbffd.ns_problem(wl.nodes, precision=64, **wl.params)
    U = rbffd.state_tensor(wl.U0, 64)
    r0 = rbffd.fields(pb.rhs(0.0, U.clone()))
    rref = o.rhs(0.0, wl.U0)
    for f in range(4):
        if np.abs(rref[f]).max() < 1e-20:
            # a field at rest: both sides give rounding noise around zero
            assert np.abs(r0[f]).max() < 1e-20
        else:
            assert rel(r0[f], rref[f]) < 1e-11, (f, rel(r0[f], rref[f]))
    pb.run(0.0, wl.dt, wl.n_steps, U)
    got = rbffd.fields(U)
    P = wl.nodes.n_prog
    errs = [rel(got[f, :P], ref[f, :P]) for f in range(4)]
    print("bubble 500 m, 48 steps: GPU vs oracle", errs)
    assert max(errs) < 1e-10


def test_bubble_full_size_fp32_vs_fp64():
    """The bubble workload at 25 m (~320k scattered nodes) to 1000 s in FP64
    and in FP32 (FP64-built weights stored in FP32): per-field relative l2 of
    the FP32 run against the FP64 run."""
    wl = configs.bubble(h=25.0, seed=1, t_end=1000.0)
    res = {}
    for prec in (64, 32):
        pb = rbffd.ns_problem(wl.nodes, precision=prec, **wl.params)
        U = rbffd.state_tensor(wl.U0, prec)
        pb.run(0.0, wl.dt, wl.n_steps, U)
        pb.sync()
        res[prec] = rbffd.fields(U)[:, :wl.nodes.n_prog]
        mm = pb.minmax(U)
        print(f"FP{prec} bubble 25 m ({wl.nodes.n_prog} nodes) at 1000 s: theta' [{mm[2, 0]:.3f}, {mm[2, 1]:.3f}] "
              f"w [{mm[1, 0]:.3f}, {mm[1, 1]:.3f}]")
        pb.close()
    errs = [rel(res[32][f], res[64][f]) for f in range(4)]
    print("FP32 vs FP64 per-field relative l2 at 1000 s [u, w, theta', pi']:", errs)
    assert np.all(np.isfinite(res[32])) and np.all(np.isfinite(res[64]))
    assert max(errs) < 1e-2
