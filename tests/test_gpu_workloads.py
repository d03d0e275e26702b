"""Full-size parity of the advection (64^2, 1000 RK4 steps to t = T) and
warm-bubble workloads (walled box, scattered nodes, n = 56, r^9 + deg 5:
lateral-wall and corner ghost systems).

Tolerances: FP64 GPU vs FP64 oracle 1e-10 relative l2 after the stated steps
(the per-step parity of 1e-11 with RK4's mild growth); the bubble's FP64
right-hand side within 0.05 kappa_max eps64 of the term scale (the weight
parity bound); FP32 vs FP64 per-field bounds stated in each test (eps32 ~
6e-8 amplified by the run).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import stencils as ost  # noqa: E402
from oracle import weights as owt  # noqa: E402
from oracle.advection import AdvectionOracle  # noqa: E402
from oracle.ns import NSOracle  # noqa: E402
from paper_1509_02615_gb300 import configs  # noqa: E402
from paper_1509_02615_gb300 import inputs as inp  # noqa: E402
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


def term_scale(o, U):
    """Per field, per node: the sum of the magnitudes of the terms of
    Eqs. (uEq)-(piEq) (each stencil sum taken with |w_ij| |f_j|).  Two FP64
    evaluations that differ only by rounding in the weights and the sums
    differ by about eps * kappa * this scale; where the terms cancel (a
    smooth field's dissipation), it is far above |tendency|."""
    V = np.array(U, dtype=np.float64, copy=True)
    o.fill_ghosts(V)
    A = {k: abs(M) for k, M in o.D.items()}
    P = o.n_prog
    au, aw, at, ap = np.abs(V)
    up, wp, tp, pp = np.abs(V[:, :P])
    cpth = np.abs(inp.CP * (o.theta_bar + V[2, :P]))
    diss = lambda f: o.mu * (A["lap"] @ f) + abs(o.hv_coef) * (A["hv"] @ f)
    su = up * (A["dx"] @ au) + wp * (A["dz"] @ au) + cpth * (A["dx"] @ ap) + diss(au)
    sw = up * (A["dx"] @ aw) + wp * (A["dz"] @ aw) + cpth * (A["dz"] @ ap) + inp.G * tp / o.theta_bar + diss(aw)
    st = up * (A["dx"] @ at) + wp * (A["dz"] @ at) + diss(at)
    sp = (up * (A["dx"] @ ap) + wp * (abs(o.dpibar) + A["dz"] @ ap)
          + (inp.RD / inp.CV) * np.abs(o.pibar + V[3, :P]) * ((A["dx"] @ au) + (A["dz"] @ aw))
          + abs(o.hv_coef) * (A["hv"] @ ap))
    return np.stack([su, sw, st, sp])


def test_bubble_small_fp64_matches_oracle():
    """RHS parity in FP64 measured against the term scale (the bubble's r^9 +
    deg-5, n = 56 weights are less well conditioned than the density
    current's, and its theta' tendency at rest is a strongly cancelling
    dissipation sum), then 48 RK4 steps against the oracle."""
    wl = configs.bubble(h=500.0, seed=1, t_end=60.0)
    o = NSOracle(wl.nodes, **wl.params)
    ref = o.run(wl.U0, 0.0, wl.dt, wl.n_steps)
    pb = rbffd.ns_problem(wl.nodes, precision=64, **wl.params)
    U = rbffd.state_tensor(wl.U0, 64)
    r0 = rbffd.fields(pb.rhs(0.0, U.clone()))
    rref = o.rhs(0.0, wl.U0)
    scale = term_scale(o, wl.U0)
    # the weight parity bound: two partial-pivoting LU codes give weights
    # that agree to O(kappa eps), kappa the augmented systems' condition
    nd = wl.nodes
    idx = ost.knn(nd.x, nd.z, np.arange(nd.n_prog), 56, nd.period_x)
    kappa = max(owt.condition_number(nd.x, nd.z, idx[i], 9, 5, nd.period_x) for i in range(0, nd.n_prog, 8))
    tol = max(1e-12, 0.05 * kappa * np.finfo(np.float64).eps)
    print(f"kappa_max {kappa:.2e}, bound {tol:.2e}")
    for f in range(4):
        if np.abs(rref[f]).max() < 1e-20:
            # a field at rest: both sides give rounding noise around zero
            assert np.abs(r0[f]).max() < 1e-20
        else:
            e = np.linalg.norm(r0[f] - rref[f]) / np.linalg.norm(scale[f])
            print(f"field {f}: |d| / |terms| = {e:.2e}, |d| / |rhs| = {rel(r0[f], rref[f]):.2e}")
            assert e < tol, (f, e)
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
