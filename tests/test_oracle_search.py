"""Pins of the oracle's large-set infrastructure (no GPU).

* The k-d tree stencil search (used above a few thousand nodes) returns the
  brute-force stencils exactly: the same nodes in the same (squared distance,
  index) order, on lattices with many equidistant ties, scattered walled
  sets, reflected sets and periodic strips.
* The pooled weight solve (worker processes) equals the serial one bit for
  bit: every stencil is solved on its own.
* The stencil orders behind the FP64 spread are permutations of the same
  stencils, whose weights differ only by rounding: on a well-conditioned
  system the spread is at rounding level, and on the density current it is
  far below a planted mistake (the viscous term dropped from one node).
"""
import numpy as np
import pytest

from oracle import stencils as st
from oracle import weights as wt
from oracle.ns import NSOracle
from oracle.operators import stencil_permutation
from paper_1509_02615_gb300 import configs
from paper_1509_02615_gb300 import inputs as inp

from fp64_bounds import bound, rel, with_spread


@pytest.mark.parametrize("case", ["dc800", "dc400cart", "square32", "scattered", "bubble200", "hexsquare"])
def test_tree_search_equals_brute_force(case):
    nodes, n = {
        "dc800": lambda: (inp.density_current_nodes(800.0), 37),
        "dc400cart": lambda: (inp.density_current_nodes(400.0, layout="cart"), 37),
        "square32": lambda: (inp.unit_square_mirrored(32), 37),
        "scattered": lambda: (inp.poisson_disk_nodes(0.0, 20.0, 0.0, 10.0, 0.5, seed=3), 56),
        "bubble200": lambda: (configs.bubble(h=200.0).nodes, 56),
        "hexsquare": lambda: (inp.unit_square_hex_mirrored(0.02), 37),
    }[case]()
    centers = np.arange(nodes.n_prog)
    a = st.knn(nodes.x, nodes.z, centers, n, nodes.period_x)
    b = st.knn_tree(nodes.x, nodes.z, centers, n, nodes.period_x)
    assert np.array_equal(a, b)


def test_tree_search_on_a_narrow_periodic_strip():
    # a strip so narrow that a node and its periodic copy are both proposed
    nodes = inp.lattice_nodes("hex", -1500.0, 1500.0, 0.0, 6400.0, 400.0, True)
    c = np.arange(nodes.n_prog)
    assert np.array_equal(st.knn(nodes.x, nodes.z, c, 37, nodes.period_x),
                          st.knn_tree(nodes.x, nodes.z, c, 37, nodes.period_x))


def test_pooled_weights_equal_serial_bit_for_bit():
    nodes = inp.density_current_nodes(400.0)
    idx = st.knn(nodes.x, nodes.z, np.arange(nodes.n_prog), 37, nodes.period_x)
    ops = ["dx", "dz", "lap"]
    a = wt.all_weights(nodes.x, nodes.z, idx, 7, 4, ops, 0, nodes.period_x)
    b = wt.all_weights_pool(nodes.x, nodes.z, idx, 7, 4, ops, 0, nodes.period_x, workers=2)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("order", ["reversed", "shuffled"])
def test_stencil_orders_are_permutations(order):
    perm = stencil_permutation(order, 37)
    assert perm[0] == 0 and sorted(perm) == list(range(37)) and not np.array_equal(perm, np.arange(37))


def test_spread_is_rounding_level_on_a_well_conditioned_system():
    nodes = inp.density_current_nodes(400.0)
    idx = st.knn(nodes.x, nodes.z, np.arange(nodes.n_prog), 37, nodes.period_x)
    ref = wt.all_weights(nodes.x, nodes.z, idx, 3, 2, ["dx", "lap"], 0, nodes.period_x)
    for order in ("reversed", "shuffled"):
        perm = stencil_permutation(order, 37)
        w = wt.all_weights(nodes.x, nodes.z, idx[:, perm], 3, 2, ["dx", "lap"], 0, nodes.period_x)
        w = w[:, :, np.argsort(perm)]
        assert max(rel(w[o], ref[o]) for o in range(2)) < 1e-13


def test_spread_bound_is_far_below_a_planted_mistake():
    nodes = inp.density_current_nodes(800.0)
    U = NSOracle(nodes).run(inp.density_current_state(nodes), 0.0, 2.0, 20)
    ref, s = with_spread(lambda o: NSOracle(nodes, stencil_order=o), lambda o: o.rhs(0.0, U))
    print("density current 800 m RHS spread", s)
    assert np.all(bound(s) < 1e-10)
    # planted in the oracle: one node's viscous term dropped
    o = NSOracle(nodes)
    D = o.D["lap"].tolil()
    D[nodes.n_prog // 2, :] = 0.0
    o.D["lap"] = D.tocsr()
    bad = o.rhs(0.0, U)
    errs = np.array([rel(bad[f], ref[f]) for f in range(4)])
    assert np.any(errs > 1e3 * bound(s)), errs
