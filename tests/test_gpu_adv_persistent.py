"""Persistent run mode of scalar advection problems (Sec. 6.1 flux form and
RK4 in one cooperative launch), through the C ABI.

* Bitwise equality with the launch-per-stage graph replay at the same lanes
  per node (2, 4 and 8), FP64 and FP32: the deformational flow (one velocity
  part) on 64 x 64 nodes and the vortex flow (two parts) on reflected
  hexagonal nodes at h = 0.02.  Runs start at t0 != 0 and mix whole graph
  chunks with leftover steps, so the stage times of both forms are compared
  too.
* A problem created with autotuning keeps the faster form; either way the
  full period matches the launch-per-stage form bit for bit.
* A barrier wait that runs out (spin limit 0) reports RBF_E_TIMEOUT through
  rbf_sync, and the same problem runs correctly afterwards.
* rbf_set_run_mode's rules for advection problems: lanes 0, 2, 4 or 8 and no
  CTA count.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1509_02615_gb300 import configs  # noqa: E402
from paper_1509_02615_gb300 import rbffd  # noqa: E402


def _run_both(pb, U0, prec, t0, dt, n, lanes):
    pb.set_run_mode("persistent", lanes=lanes)
    info = pb.info()
    assert info["run_mode"] == 2 and info["persist_lanes"] == lanes and info["threads_per_node"] == lanes
    U = rbffd.state_tensor(U0, prec)
    V = U.clone()
    pb.run(t0, dt, n, U)
    pb.sync()
    pb.set_run_mode("graph")
    assert pb.info()["run_mode"] == 1 and pb.info()["threads_per_node"] == lanes
    pb.run(t0, dt, n, V)
    pb.sync()
    return U, V


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("lanes", [2, 4, 8])
def test_persistent_equals_graph_bitwise_deformational(prec, lanes):
    wl = configs.advection(64)
    pb = rbffd.advection_problem(wl.nodes, precision=prec, **wl.params)
    # 37 steps: two graph chunks of 16 and five leftover steps
    U, V = _run_both(pb, wl.U0, prec, 0.37 * wl.dt, wl.dt, 37, lanes)
    assert torch.isfinite(U).all()
    assert not torch.equal(U, rbffd.state_tensor(wl.U0, prec))
    assert torch.equal(U, V)
    pb.close()


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("lanes", [2, 4, 8])
def test_persistent_equals_graph_bitwise_vortex(prec, lanes):
    wl = configs.vortex(h=0.02, layout="hex")
    pb = rbffd.advection_problem(wl.nodes, precision=prec, **wl.params)
    U, V = _run_both(pb, wl.U0, prec, 0.1, wl.dt, 21, lanes)
    assert torch.isfinite(U).all()
    assert torch.equal(U, V)
    pb.close()


def test_autotuned_problem_matches_graph_over_a_period():
    wl = configs.advection(64)
    pb = rbffd.advection_problem(wl.nodes, precision=64, **wl.params)
    info = pb.info()
    print(f"autotuned: run mode {info['run_mode']}, lanes {info['threads_per_node']}, "
          f"CTAs {info['persist_ctas']}")
    U = rbffd.state_tensor(wl.U0, 64)
    V = U.clone()
    pb.run(0.0, wl.dt, wl.n_steps, U)
    pb.sync()
    pb.set_run_mode("graph")
    pb.run(0.0, wl.dt, wl.n_steps, V)
    pb.sync()
    assert torch.equal(U, V)
    pb.close()


def test_persistent_timeout_reports_and_recovers():
    wl = configs.advection(64)
    pb = rbffd.advection_problem(wl.nodes, precision=64, **wl.params)
    pb.set_run_mode("persistent", lanes=8)
    assert pb.info()["persist_ctas"] > 1
    U = rbffd.state_tensor(wl.U0, 64)
    pb.set_spin_limit(0)
    pb.run(0.0, wl.dt, 5, U)
    with pytest.raises(rbffd.RBFError) as e:
        pb.sync()
    assert e.value.code == rbffd.RBF_E_TIMEOUT
    pb.sync()   # the flag is cleared once reported
    pb.set_spin_limit(1 << 21)
    U = rbffd.state_tensor(wl.U0, 64)
    V = U.clone()
    pb.run(0.0, wl.dt, 5, U)
    pb.sync()
    pb.set_run_mode("graph")
    pb.run(0.0, wl.dt, 5, V)
    pb.sync()
    assert torch.equal(U, V)
    pb.close()


def test_run_mode_arguments_for_advection():
    wl = configs.advection(64)
    pb = rbffd.advection_problem(wl.nodes, precision=32, **wl.params)
    for lanes, ctas in ((1, 0), (3, 0), (4, 7)):
        with pytest.raises(rbffd.RBFError) as e:
            pb.set_run_mode("persistent", lanes=lanes, ctas=ctas)
        assert e.value.code == rbffd.RBF_E_ARG
    pb.set_run_mode("persistent", lanes=4)
    assert pb.info()["run_mode"] == 2
    pb.close()
