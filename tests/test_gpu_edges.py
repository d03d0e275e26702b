"""Edge cases of the stencil and weight entry points (a1, a2; Sec. 3,
Eq. (weights), App. A): empty inputs, node counts that fill no warp, block or
tile evenly, the largest stencil and augmented system the kernels accept, the
sizes just past those limits, and the method's degenerate stencils.

Stencils are compared bit for bit with the oracle's brute-force ranking;
weights per operator within max(1e-12, 10 s), s the oracle's own spread over
stencil orders (tests/fp64_bounds.py)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import stencils as ost  # noqa: E402
from oracle import weights as owt  # noqa: E402
from oracle.operators import stencil_permutation  # noqa: E402
from paper_1509_02615_gb300 import inputs as inp  # noqa: E402
from paper_1509_02615_gb300 import rbffd  # noqa: E402

import fp64_bounds as fb  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1509_02615_gb300 import _build
    _build.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def _t(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _check_weights(x, z, idx, p, l, k, label):
    """GPU weights of d/dx, d/dz, Lap, d2/dx2, d2/dz2 and Delta^k of the
    stencils idx against the oracle's, within the spread bound."""
    ops = ["dx", "dz", "lap", "dxx", "dzz"]
    n = idx.shape[1]
    w = rbffd.build_weights(_t(x), _t(z), _t(idx, torch.int32), p, l, ops, 0, 0.0).cpu().numpy()
    hv = rbffd.build_weights(_t(x), _t(z), _t(idx, torch.int32), p, l, ["hv"], k, 0.0).cpu().numpy()

    def oracle_weights(order):
        perm = stencil_permutation(order, n)
        a = owt.all_weights(x, z, idx[:, perm], p, l, ops, 0, 0.0)
        b = owt.all_weights(x, z, idx[:, perm], p, l, ["hv"], k, 0.0)
        return np.concatenate([a, b])[:, :, np.argsort(perm)]

    ref, s = fb.with_spread(lambda order: order, oracle_weights)
    fb.check(np.concatenate([w, hv]), ref, s, label)


def test_empty_inputs():
    nodes = inp.density_current_nodes(800.0)
    idx = rbffd.build_stencils(_t(nodes.x), _t(nodes.z), 0, 37, nodes.period_x)
    assert tuple(idx.shape) == (0, 37)
    w = rbffd.build_weights(_t(nodes.x), _t(nodes.z), torch.zeros((0, 37), dtype=torch.int32, device="cuda"),
                            7, 4, ["dx", "dz"], 0, nodes.period_x)
    assert tuple(w.shape) == (2, 0, 37)


@pytest.mark.parametrize("h,seed", [(0.61, 11), (0.43, 12), (0.29, 13)])
def test_ragged_node_counts(h, seed):
    """Scattered node sets whose sizes are no multiple of a warp, a block or
    a binning tile; every centre's stencil and weights."""
    nodes = inp.poisson_disk_nodes(0.0, 13.0, 0.0, 7.0, h, seed=seed)
    assert nodes.n_prog % 32 != 0
    n = 37
    idx = rbffd.build_stencils(_t(nodes.x), _t(nodes.z), nodes.n_prog, n, 0.0).cpu().numpy()
    ref = ost.knn(nodes.x, nodes.z, np.arange(nodes.n_prog), n, 0.0)
    assert np.array_equal(idx, ref)
    _check_weights(nodes.x, nodes.z, ref[:257], 7, 4, 3, f"ragged {nodes.n_prog} nodes")


def test_largest_stencil_and_system():
    """n = 128 (the largest stencil) with degree 6: S = 128 + 28 = 156 unknowns
    and six right-hand sides, about 206 KB of shared memory for one system."""
    nodes = inp.poisson_disk_nodes(0.0, 20.0, 0.0, 10.0, 0.5, seed=5)
    n = 128
    idx = rbffd.build_stencils(_t(nodes.x), _t(nodes.z), nodes.n_prog, n, 0.0).cpu().numpy()
    centres = np.arange(0, nodes.n_prog, max(1, nodes.n_prog // 40))
    ref = ost.knn(nodes.x, nodes.z, centres, n, 0.0)
    assert np.array_equal(idx[centres], ref)
    # the weights of the first centres (the kernel's centre c is node c)
    _check_weights(nodes.x, nodes.z, idx[:40], 7, 6, 3, "n = 128, l = 6 (S = 156)")


def test_sizes_past_the_limits_are_rejected():
    nodes = inp.poisson_disk_nodes(0.0, 20.0, 0.0, 10.0, 0.5, seed=5)
    with pytest.raises(rbffd.RBFError) as e:
        rbffd.build_stencils(_t(nodes.x), _t(nodes.z), 8, 129, 0.0)
    assert e.value.code == rbffd.RBF_E_ARG
    idx = torch.zeros((4, 128), dtype=torch.int32, device="cuda")
    with pytest.raises(rbffd.RBFError) as e:   # degree 7: S = 128 + 36 = 164 > 160
        rbffd.build_weights(_t(nodes.x), _t(nodes.z), idx, 9, 7, ["dx"], 0, 0.0)
    assert e.value.code == rbffd.RBF_E_ARG
    small = torch.zeros((4, 6), dtype=torch.int32, device="cuda")
    with pytest.raises(rbffd.RBFError) as e:   # 6 stencil nodes, 10 monomials of degree 3
        rbffd.build_weights(_t(nodes.x), _t(nodes.z), small, 7, 3, ["dx"], 0, 0.0)
    assert e.value.code == rbffd.RBF_E_ARG


def test_collinear_stencil_is_singular():
    """Nodes on one line cannot fix the degree-1 polynomial in the other
    direction: the augmented system is singular and the node is reported."""
    t = np.linspace(0.0, 1.0, 12)
    x, z = t.copy(), 2.0 * t + 0.5
    idx = np.arange(12, dtype=np.int32)[None, :]
    with pytest.raises(rbffd.RBFError) as e:
        rbffd.build_weights(_t(x), _t(z), _t(idx, torch.int32), 3, 1, ["dx"], 0, 0.0)
    assert e.value.code == rbffd.RBF_E_SINGULAR
    # one node off the line makes the same stencil solvable
    z2 = z.copy()
    z2[5] += 0.3
    w = rbffd.build_weights(_t(x), _t(z2), _t(idx, torch.int32), 3, 1, ["dx"], 0, 0.0).cpu().numpy()
    assert np.all(np.isfinite(w))
    # d/dx of a linear function is reproduced exactly (polynomial constraints)
    assert abs(float(w[0, 0] @ (3.0 * x + 2.0 * z2)) - 3.0) < 1e-10
