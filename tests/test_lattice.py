"""Lattice operator storage, host side (no GPU): rbf_lattice_classes.

* Every member of a class has a stencil that is a translate of its first
  member's: the same relative index offsets and the same relative positions
  (minimum image in periodic x) to 1e-9 h.  Against a brute-force grouping
  of the nodes by those exact tuples.
* On the periodic hexagonal density-current lattice every node of a row
  away from the seam falls in its row's class; on scattered nodes no class
  reaches 32 members.
* Bad arguments are rejected before any work.
"""
import numpy as np
import pytest

from oracle import stencils as ost
from paper_1509_02615_gb300 import inputs as inp


@pytest.fixture(scope="module")
def rbffd():
    from paper_1509_02615_gb300 import _build, rbffd
    _build.build()
    return rbffd


def _rel(nodes, idx):
    n = nodes.n_prog
    dx = nodes.x[idx] - nodes.x[:n, None]
    if nodes.period_x > 0:
        P = nodes.period_x
        dx = np.where(dx > 0.5 * P, dx - P, np.where(dx < -0.5 * P, dx + P, dx))
    return dx, nodes.z[idx] - nodes.z[:n, None]


@pytest.mark.parametrize("case", ["dc400", "bubble400", "translating800"])
def test_classes_are_translates_and_match_brute_force(rbffd, case):
    nodes = {"dc400": lambda: inp.density_current_nodes(400.0),
             "bubble400": lambda: inp.rising_bubble_nodes(400.0, "cart"),
             "translating800": lambda: inp.translating_current_nodes(800.0, "hex")}[case]()
    n = 37
    idx = ost.knn(nodes.x, nodes.z, np.arange(nodes.n_prog), n, nodes.period_x)
    cls, nc = rbffd.lattice_classes(idx, nodes.x, nodes.z, nodes.n_prog, nodes.period_x, nodes.h, min_members=8)
    dx, dz = _rel(nodes, idx)
    off = idx - np.arange(nodes.n_prog)[:, None]
    # brute force: group by exact offsets and positions rounded to h / 2^20
    q = 2.0 ** 20 / nodes.h
    groups = {}
    for i in range(nodes.n_prog):
        key = (tuple(off[i]), tuple(np.round(dx[i] * q).astype(np.int64)), tuple(np.round(dz[i] * q).astype(np.int64)))
        groups.setdefault(key, []).append(i)
    big = [g for g in groups.values() if len(g) >= 8]
    assert nc == len(big)
    for g in big:
        c = cls[g[0]]
        assert c >= 0 and np.all(cls[g] == c)
        r = g[0]
        assert np.array_equal(off[g], np.broadcast_to(off[r], (len(g), n)))
        assert np.abs(dx[g] - dx[r]).max() < 1e-9 * nodes.h and np.abs(dz[g] - dz[r]).max() < 1e-9 * nodes.h
    assert np.sum(cls >= 0) == sum(len(g) for g in big)
    # classes are numbered in the order of their first members
    firsts = [np.nonzero(cls == c)[0][0] for c in range(nc)]
    assert firsts == sorted(firsts)


def test_hex_lattice_rows_form_classes(rbffd):
    """Every row of the periodic hexagonal lattice is one class apart from
    its seam nodes.  (Rows do not all share one class: equidistant neighbours
    are ordered by their FP64 squared distances, and that rounding differs
    from row to row, so the ordered offsets differ.)"""
    nodes = inp.density_current_nodes(200.0)          # 256 columns, 37 row intervals
    idx = ost.knn(nodes.x, nodes.z, np.arange(nodes.n_prog), 37, nodes.period_x)
    cls, nc = rbffd.lattice_classes(idx, nodes.x, nodes.z, nodes.n_prog, nodes.period_x, nodes.h)
    z = nodes.z[:nodes.n_prog]
    rows = np.unique(z)
    row_of = np.searchsorted(rows, z)
    for r in range(len(rows)):
        vals, counts = np.unique(cls[row_of == r], return_counts=True)
        assert vals[np.argmax(counts)] >= 0 and counts.max() >= 0.95 * counts.sum(), (r, vals, counts)
    frac = np.mean(cls >= 0)
    print(f"200 m hex: {nc} classes hold {frac:.3f} of the nodes")
    assert frac > 0.95 and nc <= len(rows)


def test_scattered_nodes_have_no_classes(rbffd):
    nodes = inp.poisson_disk_nodes(0.0, 20.0, 0.0, 10.0, 0.5, seed=3)
    idx = ost.knn(nodes.x, nodes.z, np.arange(nodes.n_prog), 37, nodes.period_x)
    cls, nc = rbffd.lattice_classes(idx, nodes.x, nodes.z, nodes.n_prog, nodes.period_x, nodes.h)
    assert nc == 0 and np.all(cls == -1)


def test_bad_arguments_are_rejected(rbffd):
    nodes = inp.density_current_nodes(800.0)
    idx = ost.knn(nodes.x, nodes.z, np.arange(nodes.n_prog), 37, nodes.period_x)
    bad = idx.copy()
    bad[3, 5] = nodes.n_all
    with pytest.raises(rbffd.RBFError):
        rbffd.lattice_classes(bad, nodes.x, nodes.z, nodes.n_prog, nodes.period_x, nodes.h)
    with pytest.raises(rbffd.RBFError):
        rbffd.lattice_classes(idx, nodes.x, nodes.z, nodes.n_prog, nodes.period_x, 0.0)
