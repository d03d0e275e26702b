"""a8: batched ensembles of uneven runs (GPU, through the C ABI).

* FP64: every member after its own number of RK4 steps (of its own dt)
  matches the oracle run of that member, per field below max(1e-12, 10 s),
  s the oracle's own spread between stencil orders for that member
  (tests/fp64_bounds.py).  One member is a 50 m hexagonal density current
  (about 150k nodes), the finest spacing of the batched draw.
* FP32: every member is bitwise equal to the same member stepped alone as a
  single problem with the same lanes per node (same operand order, same
  ghost solve), so batching changes nothing but the launch geometry.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle.ns import NSOracle  # noqa: E402
from paper_1509_02615_gb300 import inputs as inp  # noqa: E402
from paper_1509_02615_gb300 import rbffd  # noqa: E402

import fp64_bounds as fb  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1509_02615_gb300 import _build
    _build.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def _members(t_scale=1.0):
    spec = [(800.0, "hex", 37, 4, 30.0), (400.0, "cart", 31, 3, 12.0), (800.0, "scattered", 45, 4, 20.0),
            (400.0, "hex", 56, 5, 8.0), (800.0, "cart", 75, 5, 16.0)]
    return [inp.density_current_member(h, lay, n, l, seed=17 + i, t_end=t * t_scale)
            for i, (h, lay, n, l, t) in enumerate(spec)]


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


WORKERS = min(16, os.cpu_count() or 1)


def test_ensemble_fp64_matches_oracle_per_member():
    mem = _members() + [inp.density_current_member(50.0, "hex", 37, 4, seed=23, t_end=0.5)]
    ens = rbffd.ensemble_problem(mem, precision=64)
    U = ens.state()
    ens.run(-1, U)
    ens.sync()
    assert ens.node_updates() == sum(m.nodes.n_prog * m.n_steps for m in mem)
    for r, m in enumerate(mem):
        P = m.nodes.n_prog
        ref, s = fb.with_spread(lambda order: NSOracle(m.nodes, n=m.n, l=m.l, gamma_c=m.gamma_c, stencil_order=order,
                                                                workers=WORKERS),
                                lambda o: o.run(m.U0, 0.0, m.dt, m.n_steps)[:, :P])
        got = ens.member_fields(U, r)
        fb.check(got[:, :P], ref, s, f"member {r} ({m.nodes.layout}, h={m.nodes.h:g}, n={m.n}, steps={m.n_steps})")


def test_ensemble_fp32_equals_members_stepped_alone():
    mem = _members()
    ens = rbffd.ensemble_problem(mem, precision=32)
    G = ens.info()["threads_per_node"]
    U = ens.state()
    ens.run(-1, U)
    ens.sync()
    for r, m in enumerate(mem):
        pb = rbffd.ns_problem(m.nodes, precision=32, n=m.n, l=m.l, gamma_c=m.gamma_c, threads_per_node=G)
        V = rbffd.state_tensor(m.U0, 32)
        pb.run(0.0, m.dt, m.n_steps, V)
        pb.sync()
        a = U[ens.rec0[r]:ens.rec0[r] + m.nodes.n_prog]
        assert torch.equal(a, V[:m.nodes.n_prog]), r


def test_ensemble_partial_run_counts():
    mem = _members(t_scale=0.5)
    ens = rbffd.ensemble_problem(mem, precision=32)
    assert ens.node_updates(3) == sum(m.nodes.n_prog * min(3, m.n_steps) for m in mem)
    U = ens.state()
    ens.run(3, U)
    mm = ens.minmax(U)
    assert np.all(np.isfinite(mm))


@pytest.mark.parametrize("precision", [32, 64])
def test_blown_up_member_leaves_the_others_untouched(precision):
    """A non-finite value on a wall node of the first member in run order
    (the owner of ghost position 0 in the merged ghost systems) must not reach
    any other member: the others end bitwise equal to the same ensemble run
    without it."""
    mem = [inp.density_current_member(800.0, lay, n, l, seed=5 + i, t_end=8.0)
           for i, (lay, n, l) in enumerate([("hex", 37, 4), ("cart", 45, 4), ("scattered", 37, 4)])]
    ens = rbffd.ensemble_problem(mem, precision=precision)
    clean = ens.state()
    ens.run(-1, clean)
    bad = ens.state()
    wall = int(np.flatnonzero(np.isin(mem[0].nodes.kind, (1, 2)))[0])
    bad[wall, :] = float("nan")
    ens.run(-1, bad)
    ens.sync()
    assert not torch.all(torch.isfinite(bad[:mem[0].nodes.n_prog]))
    for r, m in enumerate(mem[1:], start=1):
        sl = slice(ens.rec0[r], ens.rec0[r] + m.nodes.n_prog)
        assert torch.equal(bad[sl], clean[sl]), r


def test_coarse_draw_runs_to_900s_finite():
    """Every member of a seeded draw at 200 and 400 m stays finite to 900 s
    (the draw skips the Cartesian stencil choices that blow up)."""
    mem = inp.ensemble_members(48, seed=1, spacings=(200.0, 400.0))
    ens = rbffd.ensemble_problem(mem, precision=32)
    U = ens.state()
    ens.run(-1, U)
    ens.sync()
    bad = [r for r, m in enumerate(mem) if not np.all(np.isfinite(ens.member_fields(U, r)[:, :m.nodes.n_prog]))]
    assert not bad, [(r, mem[r].nodes.h, mem[r].nodes.layout, mem[r].n, mem[r].l) for r in bad]


def test_cartesian_31_3_member_runs_to_900s_with_its_constant():
    """The Cartesian n = 31, l = 3 member at 50 m (the finest spacing of the
    draw), batched with a hexagonal member: with its own hyperviscosity
    constant 2^-5 (inputs.ENSEMBLE_GAMMA_C) both run to 900 s finite in FP32;
    with the common 2^-6 it goes non-finite near 630 s."""
    mem = [inp.density_current_member(50.0, "cart", 31, 3, seed=31),
           inp.density_current_member(400.0, "hex", 37, 4, seed=32)]
    assert mem[0].gamma_c == 2.0 ** -5 and mem[1].gamma_c == 2.0 ** -6
    ens = rbffd.ensemble_problem(mem, precision=32)
    U = ens.state()
    ens.run(-1, U)
    ens.sync()
    mm = ens.minmax(U)
    print("Cartesian (31,3) 50 m + hex 400 m to 900 s: theta' [%.3f, %.3f], w [%.2f, %.2f]"
          % (mm[2, 0], mm[2, 1], mm[1, 0], mm[1, 1]))
    assert np.all(np.isfinite(mm))


@pytest.mark.parametrize("precision", [32, 64])
def test_whole_run_is_one_graph_launch_equal_to_phase_replay(precision):
    """rbf_ens_run without stage timing runs the whole ensemble as one CUDA
    graph launch (a device-side WHILE loop per phase of constant active
    prefix, leftover steps after it); with stage timing it replays one-step
    graphs per phase.  Members of uneven step counts (20, 40 and 45 steps,
    so the phases have leftover steps) end bitwise equal on both paths."""
    mem = [inp.density_current_member(800.0, "hex", 37, 4, seed=41, t_end=40.0),
           inp.density_current_member(400.0, "cart", 45, 4, seed=42, t_end=40.0),
           inp.density_current_member(400.0, "scattered", 37, 4, seed=43, t_end=45.0)]
    assert sorted(m.n_steps for m in mem) == [20, 40, 45]
    ens = rbffd.ensemble_problem(mem, precision=precision)
    A = ens.state()
    ens.run(-1, A)
    B = ens.state()
    ens.set_stage_timing(True)
    ens.run(-1, B)
    ens.set_stage_timing(False)
    ens.sync()
    assert torch.equal(A, B)
    assert torch.all(torch.isfinite(A))

