"""The vortex-flow advection test of Sec. 6.1 on the GPU (two-part velocity,
rbf_adv_create_flow), through the C ABI.

* Parity: 60 FP64 RK4 steps against the oracle on reflected hexagonal and
  Cartesian nodes, both method variants, below max(1e-12, 10 s), s the
  oracle's own spread between stencil orders (tests/fp64_bounds.py); FP32
  within 1e-5.
* The paper's figures at h = 0.005 on hexagonal nodes (r^9 + deg 4,
  -2^-14 Delta^4, dt = h/15, one period T = 1): after one period the bell's
  maximum exceeds 1 by at most 0.1% (the paper reports +0.07%); at t = T/4
  and 3T/4, the most deformed states, the maximum is within 0.001 of 1 (as the
  paper states).  The undershoot is bounded at -0.5%: the paper reports
  -0.08%, this build gets -0.38%; stronger hyperviscosity does not reduce it
  (-0.43% with 4x gamma, unstable beyond), it is the dispersion around the
  bell's rim, where the second derivative jumps.
* Convergence (Fig. convergence_BD): r^3 + deg 5 with Delta^3, relative l2
  error of psi(T) against psi(0) at h = 0.01, 0.005, 0.0025 on Cartesian and
  hexagonal nodes.  On a smooth (Gaussian) bell of the same size the fitted
  order is at least 3.5 (l = 5 in the limit).  The cosine bell is only C1,
  which caps any method's l2 order near 2.5; its fitted order must be at
  least 2 (the paper's fifth order is not reached with the C1 bell).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle.advection import AdvectionOracle  # noqa: E402
from paper_1509_02615_gb300 import configs  # noqa: E402
from paper_1509_02615_gb300 import rbffd  # noqa: E402

import fp64_bounds as fb  # noqa: E402


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1509_02615_gb300 import _build
    _build.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


@pytest.mark.parametrize("layout", ["hex", "cart"])
@pytest.mark.parametrize("method", ["paper", "r3"])
def test_vortex_steps_match_oracle(layout, method):
    wl = configs.vortex(0.04, layout, method)
    ref, s = fb.with_spread(lambda order: AdvectionOracle(wl.nodes, stencil_order=order, **wl.params),
                            lambda o: o.run(wl.U0, 0.0, wl.dt, 60))
    for prec in (64, 32):
        pb = rbffd.advection_problem(wl.nodes, precision=prec, **wl.params)
        P = rbffd.state_tensor(wl.U0, prec)
        pb.run(0.0, wl.dt, 60, P)
        got = rbffd.fields(P)
        if prec == 64:
            fb.check(got, ref, s, f"vortex {layout} {method}, 60 steps")
        else:
            e = rel(got[0], ref[0])
            print(f"vortex {layout} {method} FP32 60 steps vs oracle: {e:.2e}")
            assert e < 1e-5
        pb.close()


def _period(wl, precision=64, marks=()):
    """psi after one period; the maxima at the step counts in ``marks``."""
    pb = rbffd.advection_problem(wl.nodes, precision=precision, **wl.params)
    P = rbffd.state_tensor(wl.U0, precision)
    done, seen = 0, {}
    for m in sorted(marks) + [wl.n_steps]:
        pb.run(done * wl.dt, wl.dt, m - done, P)
        done = m
        seen[m] = rbffd.fields(P)[0].copy()
    pb.close()
    return seen


def test_vortex_bell_extrema_match_paper():
    wl = configs.vortex(0.005, "hex", "paper")
    q = wl.n_steps // 4
    seen = _period(wl, 64, marks=(q, 3 * q))
    psi = seen[wl.n_steps]
    print("vortex hex h=0.005 r^9 deg 4: max %.5f min %.5f at T; max %.5f / %.5f at T/4, 3T/4; rel l2 %.3e"
          % (psi.max(), psi.min(), seen[q].max(), seen[3 * q].max(), rel(psi, wl.U0)))
    assert psi.max() - 1.0 < 1e-3
    assert psi.min() > -5e-3
    assert abs(seen[q].max() - 1.0) < 1e-3 and abs(seen[3 * q].max() - 1.0) < 1e-3


def _gaussian_bell(nodes):
    x, y = nodes.x[:nodes.n_prog], nodes.z[:nodes.n_prog]
    return np.exp(-((x - 0.3) ** 2 + (y - 0.5) ** 2) / (2 * 0.07 ** 2))


@pytest.mark.parametrize("layout", ["cart", "hex"])
def test_vortex_convergence_order(layout):
    hs = [0.01, 0.005, 0.0025]
    ec, eg = [], []
    for h in hs:
        wl = configs.vortex(h, layout, "r3")
        ec.append(rel(_period(wl)[wl.n_steps], wl.U0))
        g0 = _gaussian_bell(wl.nodes)
        pb = rbffd.advection_problem(wl.nodes, precision=64, **wl.params)
        P = rbffd.state_tensor(g0, 64)
        pb.run(0.0, wl.dt, wl.n_steps, P)
        eg.append(rel(rbffd.fields(P)[0], g0))
        pb.close()
    sc = np.polyfit(np.log(hs), np.log(ec), 1)[0]
    sg = np.polyfit(np.log(hs), np.log(eg), 1)[0]
    print(f"vortex {layout} r^3 deg 5: cosine bell", ["%.3e" % e for e in ec], f"order {sc:.2f};",
          "Gaussian bell", ["%.3e" % e for e in eg], f"order {sg:.2f}")
    assert sg > 3.5, (sg, eg)
    assert sc > 2.0, (sc, ec)


def test_vortex_order_follows_the_bells_smoothness():
    """What caps the order of the printed cosine bell (Fig. convergence_BD):
    the same r^3 + deg 5 method, flow, reflected walls and nodes (hexagonal,
    h = 0.005 and 0.0025, hyperviscosity 2^-12 h^5), three initial bells that
    differ only in smoothness at the rim -- the printed bell (1 + cos)/2 (C1),
    its cube (C5) -- and a Gaussian.  The smooth bells converge at the fifth
    order the paper prints (>= 4.5 here); the C1 bell stays near 2.2 whatever
    the hyperviscosity (the same in this run), so the bell, not the method,
    the walls or gamma, caps its order."""
    orders = {}
    errs = {"cos": [], "cos3": [], "gauss": []}
    hs = [0.005, 0.0025]
    for h in hs:
        wl = configs.vortex(h, "hex", "r3")
        prm = dict(wl.params, gamma_c=2.0 ** -12)
        pb = rbffd.advection_problem(wl.nodes, precision=64, **prm)
        c = wl.U0
        for name, b0 in (("cos", c), ("cos3", c ** 3), ("gauss", _gaussian_bell(wl.nodes))):
            P = rbffd.state_tensor(b0, 64)
            pb.run(0.0, wl.dt, wl.n_steps, P)
            errs[name].append(rel(rbffd.fields(P)[0], b0))
        pb.close()
    for name, e in errs.items():
        orders[name] = np.log(e[0] / e[1]) / np.log(hs[0] / hs[1])
    print("vortex hex r^3 deg 5, gamma 2^-12 h^5, errors", {k: ["%.3e" % v for v in e] for k, e in errs.items()},
          "orders", {k: round(float(v), 2) for k, v in orders.items()})
    assert orders["cos3"] >= 4.5 and orders["gauss"] >= 4.5, orders
    assert orders["cos"] < 2.6, orders
