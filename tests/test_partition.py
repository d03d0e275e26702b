"""Host logic of the persistent run mode without a GPU: the node blocks
(recursive coordinate bisection, rbf_partition_blocks) on the density-current
and scattered node sets."""
import numpy as np
import pytest

from paper_1509_02615_gb300 import inputs as inp


@pytest.fixture(scope="module")
def rbffd():
    from paper_1509_02615_gb300 import _build, rbffd
    _build.build()
    return rbffd


@pytest.mark.parametrize("case,parts", [("hex100", 152), ("hex400", 38), ("scattered", 152), ("hex400", 1)])
def test_blocks_are_balanced_compact_and_cover_every_node(rbffd, case, parts):
    if case == "hex100":
        nodes = inp.density_current_nodes(100.0)
    elif case == "hex400":
        nodes = inp.density_current_nodes(400.0)
    else:
        nodes = inp.poisson_disk_nodes(0.0, 20.0, 0.0, 10.0, 0.25, seed=2)
    P = nodes.n_prog
    x, z = nodes.x[:P], nodes.z[:P]
    b = rbffd.partition_blocks(x, z, parts)
    counts = np.bincount(b, minlength=parts)
    # every node in exactly one block, blocks of equal size +-1
    assert b.min() == 0 and b.max() == parts - 1
    assert counts.sum() == P and counts.max() - counts.min() <= 1
    # compact: each block's bounding box holds few nodes of other blocks
    # (a random assignment of this size would be ~parts times worse)
    foreign = 0
    for k in range(parts):
        m = b == k
        inside = (x >= x[m].min()) & (x <= x[m].max()) & (z >= z[m].min()) & (z <= z[m].max())
        foreign += int(np.count_nonzero(inside & ~m))
    print(f"{case}, {parts} blocks: sizes {counts.min()}-{counts.max()}, foreign nodes in boxes {foreign / P:.3f} per node")
    assert foreign <= 0.6 * P


def test_blocks_are_deterministic_and_reject_bad_arguments(rbffd):
    nodes = inp.density_current_nodes(800.0)
    P = nodes.n_prog
    a = rbffd.partition_blocks(nodes.x[:P], nodes.z[:P], 17)
    b = rbffd.partition_blocks(nodes.x[:P], nodes.z[:P], 17)
    assert np.array_equal(a, b)
    with pytest.raises(rbffd.RBFError) as e:
        rbffd.partition_blocks(nodes.x[:P], nodes.z[:P], P + 1)
    assert e.value.code == rbffd.RBF_E_ARG
    x = nodes.x[:P].copy()
    x[3] = np.nan
    with pytest.raises(rbffd.RBFError):
        rbffd.partition_blocks(x, nodes.z[:P], 4)
