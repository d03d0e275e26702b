"""GPU parity of librbffd against the FP64 oracle (through the C ABI).

Tolerances (relative l2 unless stated):
  * stencils: identical index lists (bit-exact: both sides order by the same
    FP64 squared distance, then index);
  * FP64 weights, right-hand sides, ghost values and RK4 steps: per output
    max(1e-12, 10 s), s the oracle's own spread between stencil orders
    (tests/fp64_bounds.py); the largest 2-norm condition number of the
    scaled augmented systems is printed beside the weights;
  * FP32: per-field bounds stated in each test (FP32 weights and arithmetic,
    eps32 = 6e-8, difference form).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import stencils as ost  # noqa: E402
from oracle import weights as owt  # noqa: E402
from oracle.advection import AdvectionOracle  # noqa: E402
from oracle.ns import NSOracle, front_location  # noqa: E402
from oracle.operators import stencil_permutation  # noqa: E402
from paper_1509_02615_gb300 import inputs as inp  # noqa: E402
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


def _t(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


@pytest.mark.parametrize("case", ["dc800", "dc400", "square32", "scattered"])
def test_stencils_bit_exact(case):
    if case == "dc800":
        nodes, n = inp.density_current_nodes(800.0), 37
    elif case == "dc400":
        nodes, n = inp.density_current_nodes(400.0), 37
    elif case == "square32":
        nodes, n = inp.unit_square_mirrored(32), 37
    else:
        nodes, n = inp.poisson_disk_nodes(0.0, 20.0, 0.0, 10.0, 0.5, seed=3), 56
    idx = rbffd.build_stencils(_t(nodes.x), _t(nodes.z), nodes.n_prog, n, nodes.period_x).cpu().numpy()
    ref = ost.knn(nodes.x, nodes.z, np.arange(nodes.n_prog), n, nodes.period_x)
    assert np.array_equal(idx, ref)


def test_stencils_full_density_current_sampled():
    nodes = inp.density_current_nodes(100.0)
    idx = rbffd.build_stencils(_t(nodes.x), _t(nodes.z), nodes.n_prog, 37, nodes.period_x).cpu().numpy()
    rng = np.random.default_rng(0)
    sample = np.concatenate([rng.choice(nodes.n_prog, 400, replace=False), np.arange(600), np.arange(nodes.n_prog - 600, nodes.n_prog)])
    ref = ost.knn(nodes.x, nodes.z, sample, 37, nodes.period_x)
    assert np.array_equal(idx[sample], ref)


@pytest.mark.parametrize("p,l,k", [(7, 4, 3), (9, 5, 3), (3, 2, 1)])
def test_weights_fp64(p, l, k):
    nodes = inp.density_current_nodes(400.0)
    n = 37
    idx = ost.knn(nodes.x, nodes.z, np.arange(nodes.n_prog), n, nodes.period_x)
    ops = ["dx", "dz", "lap", "dxx", "dzz"]
    w = rbffd.build_weights(_t(nodes.x), _t(nodes.z), _t(idx, torch.int32), p, l, ops, 0, nodes.period_x).cpu().numpy()
    hv = rbffd.build_weights(_t(nodes.x), _t(nodes.z), _t(idx, torch.int32), p, l, ["hv"], k, nodes.period_x).cpu().numpy()

    def oracle_weights(order):
        # weights of the same stencils listed in another order, put back in
        # the ranked order
        perm = stencil_permutation(order, n)
        a = owt.all_weights(nodes.x, nodes.z, idx[:, perm], p, l, ops, 0, nodes.period_x)
        b = owt.all_weights(nodes.x, nodes.z, idx[:, perm], p, l, ["hv"], k, nodes.period_x)
        return np.concatenate([a, b])[:, :, np.argsort(perm)]

    ref, s = fb.with_spread(lambda order: order, oracle_weights)
    kappa = max(owt.condition_number(nodes.x, nodes.z, idx[i], p, l, nodes.period_x)
                for i in range(0, nodes.n_prog, 37))
    print(f"p={p} l={l} kappa_max={kappa:.3e} (0.05 kappa eps = {0.05 * kappa * np.finfo(np.float64).eps:.1e})")
    fb.check(np.concatenate([w, hv]), ref, s, f"weights p={p} l={l}")


def test_weights_singular_stencil_is_reported():
    # two nodes at the same position make the augmented system singular
    x = np.array([0.0, 1.0, 0.0, 1.0, 0.5, 0.5, 2.0, 0.0])
    z = np.array([0.0, 0.0, 1.0, 1.0, 0.5, 0.5, 2.0, 2.0])
    idx = np.array([[4, 5, 0, 1, 2, 3]], np.int32)
    with pytest.raises(rbffd.RBFError) as e:
        rbffd.build_weights(_t(x), _t(z), _t(idx, torch.int32), 3, 1, ["dx"], 0, 0.0)
    assert e.value.code == rbffd.RBF_E_SINGULAR


def _dc_state(nodes, oracle, steps):
    U = inp.density_current_state(nodes)
    return oracle.run(U, 0.0, nodes.h / 400.0, steps)


@pytest.fixture(scope="module")
def dc800():
    nodes = inp.density_current_nodes(800.0)
    o = NSOracle(nodes)
    U = _dc_state(nodes, o, 60)
    return nodes, o, U


@pytest.fixture(scope="module")
def dc800_fp64_ref(dc800):
    """The oracle's right-hand side and ghost values at the 60-step state,
    with their spreads over stencil orders."""
    nodes, o, U = dc800

    def outputs(orc):
        V = U.copy()
        orc.fill_ghosts(V)
        return orc.rhs(0.0, U), V[:, nodes.n_prog:]

    res = {order: outputs(o if order == "nearest" else NSOracle(nodes, stencil_order=order))
           for order in ("nearest",) + fb.ORDERS}
    rhs, s_rhs = fb.with_spread(lambda order: order, lambda order: res[order][0])
    gh, s_gh = fb.with_spread(lambda order: order, lambda order: res[order][1])
    return rhs, s_rhs, gh, s_gh


def test_ns_rhs_fp64(dc800, dc800_fp64_ref):
    nodes, o, U = dc800
    ref, s, gref, gs = dc800_fp64_ref
    pb = rbffd.ns_problem(nodes, precision=64, threads_per_node=4)
    Ud = rbffd.state_tensor(U, 64)
    got = rbffd.fields(pb.rhs(0.0, Ud))
    fb.check(got, ref, s, "density current 800 m RHS")
    # the ghost entries written into U solve the ghost systems
    fb.check(rbffd.fields(Ud)[:, nodes.n_prog:], gref, gs, "density current 800 m ghost values")


@pytest.mark.parametrize("G", [1, 2, 4, 8])
def test_ns_rhs_fp64_every_lane_split(dc800, dc800_fp64_ref, G):
    nodes, o, U = dc800
    ref, s, _, _ = dc800_fp64_ref
    pb = rbffd.ns_problem(nodes, precision=64, threads_per_node=G)
    got = rbffd.fields(pb.rhs(0.0, rbffd.state_tensor(U, 64)))
    fb.check(got, ref, s, f"RHS G={G}")


def test_ns_rk4_fp64_steps():
    nodes = inp.density_current_nodes(400.0)
    U0 = inp.density_current_state(nodes)
    P = nodes.n_prog
    ref, s = fb.with_spread(lambda order: NSOracle(nodes, stencil_order=order),
                            lambda o: o.run(U0, 0.0, 1.0, 10)[:, :P])
    pb = rbffd.ns_problem(nodes, precision=64)
    Ud = rbffd.state_tensor(U0, 64)
    for step in range(10):
        pb.rk4_step(step * 1.0, 1.0, Ud)
    fb.check(rbffd.fields(Ud)[:, :P], ref, s, "density current 400 m, 10 steps")


def test_run_graph_equals_steps_bitwise():
    nodes = inp.density_current_nodes(800.0)
    U0 = inp.density_current_state(nodes)
    for prec in (64, 32):
        pb = rbffd.ns_problem(nodes, precision=prec, threads_per_node=4)
        A = rbffd.state_tensor(U0, prec)
        B = A.clone()
        for s in range(21):
            pb.rk4_step(2.0 * s, 2.0, A)
        pb.run(0.0, 2.0, 21, B)
        pb.sync()
        assert torch.equal(A[:nodes.n_prog], B[:nodes.n_prog])
        # end-to-end form on a host tensor
        C = rbffd.state_tensor(U0, prec, device="cpu").pin_memory()
        pb.run_host(0.0, 2.0, 21, C)
        assert torch.equal(C[:nodes.n_prog], B.cpu()[:nodes.n_prog])


def test_ns_fp32_rhs(dc800):
    nodes, o, U = dc800
    pb = rbffd.ns_problem(nodes, precision=32)
    got = rbffd.fields(pb.rhs(0.0, rbffd.state_tensor(U, 32)))
    ref = o.rhs(0.0, U)
    print("fp32 rhs rel l2 per field", [f"{rel(got[f], ref[f]):.2e}" for f in range(4)])
    for f, tol in zip(range(4), (2e-4, 2e-4, 2e-4, 2e-3)):
        assert rel(got[f], ref[f]) < tol, (f, rel(got[f], ref[f]))


@pytest.mark.parametrize("G", [1, 2, 4, 8])
def test_ns_rhs_fp32_every_lane_split(dc800, G):
    nodes, o, U = dc800
    pb = rbffd.ns_problem(nodes, precision=32, threads_per_node=G)
    got = rbffd.fields(pb.rhs(0.0, rbffd.state_tensor(U, 32)))
    ref = o.rhs(0.0, U)
    for f, tol in zip(range(4), (2e-4, 2e-4, 2e-4, 2e-3)):
        assert rel(got[f], ref[f]) < tol


def test_ns_fp32_run_400m_to_300s():
    nodes = inp.density_current_nodes(400.0)
    o = NSOracle(nodes)
    U0 = inp.density_current_state(nodes)
    ref = o.run(U0, 0.0, 1.0, 300)
    pb = rbffd.ns_problem(nodes, precision=32)
    Ud = rbffd.state_tensor(U0, 32)
    pb.run(0.0, 1.0, 300, Ud)
    got = rbffd.fields(Ud)
    print("fp32 300-step rel l2 per field", [f"{rel(got[f, :nodes.n_prog], ref[f, :nodes.n_prog]):.2e}" for f in range(4)])
    for f in range(4):
        assert rel(got[f, :nodes.n_prog], ref[f, :nodes.n_prog]) < 1e-3, (f, rel(got[f, :nodes.n_prog], ref[f, :nodes.n_prog]))


def test_minmax_and_nonfinite(dc800):
    nodes, o, U = dc800
    pb = rbffd.ns_problem(nodes, precision=64)
    Ud = rbffd.state_tensor(U, 64)
    mm = pb.minmax(Ud)
    P = U[:, :nodes.n_prog]
    assert np.allclose(mm[:, 0], P.min(axis=1)) and np.allclose(mm[:, 1], P.max(axis=1))
    Ud[5, 2] = float("nan")
    with pytest.raises(rbffd.RBFError) as e:
        pb.minmax(Ud)
    assert e.value.code == rbffd.RBF_E_NONFINITE


def test_advection_fp64():
    nodes = inp.unit_square_mirrored(32)
    psi0 = inp.cosine_bell(nodes.x[:nodes.n_prog], nodes.z[:nodes.n_prog])
    orc = {order: AdvectionOracle(nodes, stencil_order=order) for order in ("nearest",) + fb.ORDERS}
    pb = rbffd.advection_problem(nodes, precision=64)
    P = rbffd.state_tensor(psi0, 64)
    got = rbffd.fields(pb.rhs(0.7, P))
    ref, s = fb.with_spread(lambda order: orc[order], lambda o: o.rhs(0.7, psi0))
    fb.check(got, ref, s, "advection 32^2 RHS")
    pb.run(0.0, 0.005, 50, P)
    ref, s = fb.with_spread(lambda order: orc[order], lambda o: o.run(psi0, 0.0, 0.005, 50))
    fb.check(rbffd.fields(P), ref, s, "advection 32^2, 50 steps")


def test_density_current_100m_matches_paper_table():
    """Table straka, hexagonal 100 m: min/max theta', min/max w, front at
    t = 900 s (the GPU runs the full 3600 RK4 steps in FP64)."""
    nodes = inp.density_current_nodes(100.0)
    pb = rbffd.ns_problem(nodes, precision=64)
    U = rbffd.state_tensor(inp.density_current_state(nodes), 64)
    pb.run(0.0, 0.25, 3600, U)
    mm = pb.minmax(U)
    th = rbffd.fields(U)[2]
    front = front_location(nodes, th)
    print("100 m hex FP64 at 900 s: theta' [%.3f, %.3f] w [%.3f, %.3f] front %.1f m" % (mm[2, 0], mm[2, 1], mm[1, 0], mm[1, 1], front))
    assert abs(mm[2, 0] - (-9.70)) < 0.15
    assert abs(mm[2, 1] - 0.20) < 0.05
    assert abs(mm[1, 0] - (-15.90)) < 0.3
    assert abs(mm[1, 1] - 12.96) < 0.3
    assert abs(front - 15444.0) < 60.0
