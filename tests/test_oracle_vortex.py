"""Pins of the vortex-flow advection case of Sec. 6.1 (no GPU).

* The time-separable split of the velocity that the CUDA path is fed
  (inputs.vortex_flow_parts) sums to the oracle's own closed form of the
  paper's u_theta, sin(theta), cos(theta) at every time, including the centre
  r = 0 and all four quadrants.
* The flow is divergence-free, so a constant scalar keeps a zero tendency
  up to the truncation error of -(Dx u + Dy v), which falls at the polynomial
  order; a smooth field that is even about every wall has a tendency error
  falling at order >= l - 1/2 (Sec. 4) on the reflected hexagonal lattice.
* Reflection on the hexagonal lattice: each reflected node sits at the mirror
  image of its source across the nearest walls.
* Stability at dt = h/15 (the paper's step).  The vortex flow crosses the
  walls (it is a rotation about the centre, so near the corners it enters and
  leaves the square), and the reflected nodes then act as inflow boundaries:
  the frozen-time operator has modes at the walls whose RK4 amplification
  exceeds 1 slightly.  What matters is their growth per unit time,
  log max|R| / dt, which must stay bounded as h shrinks (a grid-scale
  instability grows like 1/h): below 15 per period for the paper's variant
  and below 2 for the r^3 variant, at h = 0.04 and 0.02, at t = 0 (fastest
  flow) and t = T/4.
"""
import numpy as np
import pytest

from oracle.advection import AdvectionOracle, vortex_velocity
from paper_1509_02615_gb300 import configs
from paper_1509_02615_gb300 import inputs as inp


def test_separable_parts_sum_to_the_closed_form():
    rng = np.random.default_rng(3)
    x = np.concatenate([[0.5, 0.0, 1.0, 0.5, 0.2], rng.uniform(-0.1, 1.1, 200)])
    y = np.concatenate([[0.5, 0.0, 1.0, 0.9, 0.5], rng.uniform(-0.1, 1.1, 200)])
    for T in (1.0, 2.5):
        parts, coef = inp.vortex_flow_parts(x, y, T)
        for t in (0.0, 0.13, 0.25, 0.5, 0.77, 1.0):
            u = sum((a + b * np.cos(m * np.pi * t / T)) * pu for (pu, _), (a, b, m) in zip(parts, coef))
            v = sum((a + b * np.cos(m * np.pi * t / T)) * pv for (_, pv), (a, b, m) in zip(parts, coef))
            ue, ve = vortex_velocity(x, y, t, T)
            assert np.abs(u - ue).max() < 1e-12 * (1 + np.abs(ue).max())
            assert np.abs(v - ve).max() < 1e-12 * (1 + np.abs(ve).max())


def test_hex_reflections_are_mirror_images():
    nodes = inp.unit_square_hex_mirrored(0.05, layers=5)
    for j in range(nodes.n_prog, nodes.n_all):
        s = nodes.src[j]
        x, y = nodes.x[j], nodes.z[j]
        rx = x if 0.0 <= x <= 1.0 else (-x if x < 0 else 2.0 - x)
        ry = y if 0.0 <= y <= 1.0 else (-y if y < 0 else 2.0 - y)
        assert abs(rx - nodes.x[s]) < 1e-12 and abs(ry - nodes.z[s]) < 1e-12
    # every prognostic node's stencil stays inside the reflected layers: the
    # 37 nearest nodes of a corner node lie within 3.1 spacings
    o = AdvectionOracle(nodes, n=37, p=9, l=4, T=1.0, flow="vortex")
    d = np.hypot(nodes.x[o.idx] - nodes.x[:nodes.n_prog, None], nodes.z[o.idx] - nodes.z[:nodes.n_prog, None])
    assert d.max() < 3.1 * 0.05


@pytest.mark.parametrize("method", ["paper", "r3"])
def test_divergence_free_and_smooth_field_converge(method):
    hs = [0.08, 0.04, 0.02]
    e1, e2 = [], []
    prm = dict(configs.VORTEX_METHODS[method], T=1.0, flow="vortex")
    l = prm["l"]
    t = 0.3
    for h in hs:
        nodes = inp.unit_square_hex_mirrored(h)
        o = AdvectionOracle(nodes, **dict(prm, gamma=0.0))
        x, y = nodes.x[:nodes.n_prog], nodes.z[:nodes.n_prog]
        e1.append(np.abs(o.rhs(t, np.ones(nodes.n_prog))).max())
        psi = np.cos(np.pi * x) * np.cos(np.pi * y)
        u, v = vortex_velocity(x, y, t, 1.0)
        exact = -(u * (-np.pi * np.sin(np.pi * x) * np.cos(np.pi * y)) + v * (-np.pi * np.cos(np.pi * x) * np.sin(np.pi * y)))
        e2.append(np.abs(o.rhs(t, psi)[0] - exact).max())
    s1 = np.polyfit(np.log(hs), np.log(e1), 1)[0]
    s2 = np.polyfit(np.log(hs), np.log(e2), 1)[0]
    print(method, "divergence slope %.2f smooth-field slope %.2f" % (s1, s2), e1, e2)
    assert s1 > l - 0.5 and s2 > l - 0.5, (s1, s2, e1, e2)


@pytest.mark.slow
@pytest.mark.parametrize("method,limit", [("paper", 15.0), ("r3", 2.0)])
def test_growth_per_unit_time_is_bounded(method, limit):
    for h in (0.04, 0.02):
        wl = configs.vortex(h, "hex", method)
        o = AdvectionOracle(wl.nodes, **wl.params)
        N = wl.nodes.n_prog
        rows = np.repeat(np.arange(N), o.cols.shape[1])
        for t in (0.0, 0.25):
            A = np.zeros((N, N))
            np.add.at(A, (rows, o.cols.ravel()), (o.advection_weights(t) + o.Whv).ravel())
            z = np.linalg.eigvals(A * wl.dt)
            R = np.abs(1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24)
            rate = np.log(R.max()) / wl.dt
            print(method, h, t, "max |R| %.6f, growth %.2f per unit time" % (R.max(), rate))
            assert rate < limit, (h, t, rate)
