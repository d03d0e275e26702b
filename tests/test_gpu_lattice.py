"""Lattice operator storage on the GPU (rbf_set_operator_storage), through
the C ABI.

* The right-hand side with lattice storage equals the per-node one up to the
  rounding of the weights (a class member's augmented system is its first
  member's, translated).  FP64: both storages against the oracle, per field
  below max(1e-12, 10 s), s the oracle's own spread between stencil orders
  (tests/fp64_bounds.py); FP32: lattice against per-node < 1e-5; for every
  lane count.
* FP64 RK4 steps with lattice storage against the oracle (the same bound)
  after 20 steps, on the periodic hexagonal density current and the walled
  Cartesian rising bubble.
* Scattered nodes form no class: the storage falls back to per-node rows and
  the result is bit-identical.
* On the 100 m hexagonal density current more than 95% of the nodes are in
  classes.
* The switch rejects advection problems and leaves a persistent run (which
  keeps its own operators) bit-identical.
* A batched ensemble created with lattice storage matches the same ensemble
  with per-node storage member by member (FP32 < 1e-5; FP64 within the
  member's oracle spread bound), and FP64 members match the oracle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle.ns import NSOracle  # noqa: E402
from paper_1509_02615_gb300 import configs  # noqa: E402
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


@pytest.fixture(scope="module")
def dc400_rhs_ref():
    nodes = inp.density_current_nodes(400.0)
    U0 = inp.density_current_state(nodes)
    ref, s = fb.with_spread(lambda order: NSOracle(nodes, stencil_order=order), lambda o: o.rhs(0.0, U0))
    return nodes, U0, ref, s


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("G", [1, 2, 4, 8])
def test_lattice_rhs_equals_per_node(dc400_rhs_ref, prec, G):
    nodes, U0, oref, s = dc400_rhs_ref
    pb = rbffd.ns_problem(nodes, precision=prec, threads_per_node=G)
    U = rbffd.state_tensor(U0, prec)
    ref = rbffd.fields(pb.rhs(0.0, U.clone()))
    cn, nc = pb.set_operator_storage("lattice", threads_per_node=G)
    assert pb.info()["threads_per_node"] == G and nc > 0
    got = rbffd.fields(pb.rhs(0.0, U.clone()))
    errs = [rel(got[f], ref[f]) for f in range(4)]
    print(f"FP{prec} G={G}: {nc} classes, {cn}/{nodes.n_prog} nodes; lattice vs per-node RHS", ["%.1e" % e for e in errs])
    if prec == 64:
        fb.check(ref, oref, s, f"per-node G={G}")
        fb.check(got, oref, s, f"lattice G={G}")
    else:
        assert max(errs) < 1e-5
    pb.close()


@pytest.mark.parametrize("case", ["density_current", "rising_bubble"])
def test_lattice_steps_match_oracle(case):
    if case == "density_current":
        nodes = inp.density_current_nodes(400.0)
        params = dict(mu=75.0)
        U0 = inp.density_current_state(nodes)
        dt = 1.0
    else:
        wl = configs.rising_bubble(400.0, "cart")
        nodes, params, U0, dt = wl.nodes, dict(wl.params), wl.U0, wl.dt
    P = nodes.n_prog
    ref, s = fb.with_spread(lambda order: NSOracle(nodes, stencil_order=order, **params),
                            lambda o: o.run(U0, 0.0, dt, 20)[:, :P])
    pb = rbffd.ns_problem(nodes, precision=64, **params)
    pb.set_run_mode("graph")
    cn, nc = pb.set_operator_storage("lattice")
    U = rbffd.state_tensor(U0, 64)
    pb.run(0.0, dt, 20, U)
    pb.sync()
    got = rbffd.fields(U)
    fb.check(got[:, :P], ref, s, f"{case}: {nc} classes, {cn}/{P} nodes; 20 steps")
    pb.close()


def test_scattered_nodes_fall_back_bitwise():
    wl = configs.bubble(h=500.0, seed=1, t_end=10.0)
    for prec in (64, 32):
        pb = rbffd.ns_problem(wl.nodes, precision=prec, threads_per_node=2, **wl.params)
        pb.set_run_mode("graph")
        A = rbffd.state_tensor(wl.U0, prec)
        B = A.clone()
        pb.run(0.0, wl.dt, 10, A)
        cn, nc = pb.set_operator_storage("lattice", threads_per_node=2)
        assert cn == 0 and nc == 0
        pb.run(0.0, wl.dt, 10, B)
        pb.sync()
        assert torch.equal(A, B)
        pb.close()


def test_hex_100m_is_mostly_classes():
    nodes = inp.density_current_nodes(100.0)
    pb = rbffd.ns_problem(nodes, precision=32, threads_per_node=1)
    cn, nc = pb.set_operator_storage("lattice", threads_per_node=1)
    info = pb.info()
    print(f"100 m hex: {nc} classes hold {cn}/{nodes.n_prog} nodes; {info['rhs_bytes_per_node']:.1f} B per node-RHS")
    assert cn > 0.95 * nodes.n_prog
    assert info["rhs_bytes_per_node"] < 150.0
    pb.close()


def _members():
    spec = [(800.0, "hex", 37, 4, 30.0), (400.0, "cart", 31, 3, 12.0), (800.0, "scattered", 45, 4, 20.0),
            (400.0, "hex", 56, 5, 8.0), (800.0, "cart", 75, 5, 16.0)]
    return [inp.density_current_member(h, lay, n, l, seed=17 + i, t_end=t)
            for i, (h, lay, n, l, t) in enumerate(spec)]


@pytest.mark.parametrize("prec", [64, 32])
def test_ensemble_lattice_matches_per_node(prec):
    """An ensemble created with lattice storage (each member with its own
    class table; the scattered member keeps per-node rows) against the same
    ensemble with per-node storage, every member after its own step count;
    FP64 also against the oracle."""
    mem = _members()
    out = {}
    for storage in ("per-node", "lattice"):
        ens = rbffd.ensemble_problem(mem, precision=prec, storage=storage)
        U = ens.state()
        ens.run(-1, U)
        ens.sync()
        out[storage] = [ens.member_fields(U, r)[:, :m.nodes.n_prog] for r, m in enumerate(mem)]
        info = ens.info()
        print(f"FP{prec} {storage}: {info['rhs_bytes_per_node']:.1f} B per node-RHS")
        ens.close()
    for r, m in enumerate(mem):
        errs = [rel(out["lattice"][r][f], out["per-node"][r][f]) for f in range(4)]
        print(f"member {r} ({m.nodes.layout}, h={m.nodes.h:g}, n={m.n}) lattice vs per-node", ["%.1e" % e for e in errs])
        if prec == 32:
            assert max(errs) < 1e-5, (r, errs)
            continue
        P = m.nodes.n_prog
        ref, s = fb.with_spread(lambda order: NSOracle(m.nodes, n=m.n, l=m.l, gamma_c=m.gamma_c, stencil_order=order),
                                lambda o: o.run(m.U0, 0.0, m.dt, m.n_steps)[:, :P])
        # the two storages differ by the rounding of translated stencils' weights
        assert np.all(np.array(errs) < fb.bound(s)), (r, errs, s)
        fb.check(out["lattice"][r], ref, s, f"member {r} lattice")


def test_storage_switch_rules():
    """The switch applies to Navier-Stokes problems only, and a persistent run
    (which keeps its own operators) is unchanged by it, bit for bit."""
    adv = rbffd.advection_problem(inp.unit_square_mirrored(16), precision=64)
    with pytest.raises(rbffd.RBFError):
        adv.set_operator_storage("lattice")
    adv.close()
    nodes = inp.density_current_nodes(800.0)
    U0 = inp.density_current_state(nodes)
    pb = rbffd.ns_problem(nodes, precision=32, threads_per_node=1)
    pb.set_run_mode("persistent", lanes=1)
    A = rbffd.state_tensor(U0, 32)
    B = A.clone()
    pb.run(0.0, 2.0, 10, A)
    pb.set_operator_storage("lattice", threads_per_node=1)
    pb.run(0.0, 2.0, 10, B)
    pb.sync()
    assert pb.info()["run_mode"] == 2
    assert torch.equal(A, B)
    pb.close()


def test_lattice_tables_survive_run_mode_autotuning():
    """A lattice problem with autotuned lanes and run mode (the persistent
    plans tried at creation pack operators for their own lane counts) keeps
    graph-mode tables that match its lanes: its graph-mode right-hand side
    equals the per-node problem's to FP32 rounding."""
    nodes = inp.density_current_nodes(400.0)
    U0 = inp.density_current_state(nodes)
    out = {}
    for storage in ("per-node", "lattice"):
        pb = rbffd.ns_problem(nodes, precision=32, storage=storage)
        pb.set_run_mode("persistent", lanes=2)    # plans for another lane count, then back
        pb.set_run_mode("graph")
        U = rbffd.state_tensor(U0, 32)
        out[storage] = rbffd.fields(pb.rhs(0.0, U))
        pb.close()
    errs = [rel(out["lattice"][f], out["per-node"][f]) for f in range(4)]
    print("lattice after run-mode planning vs per-node RHS", ["%.1e" % e for e in errs])
    assert max(errs) < 1e-5
