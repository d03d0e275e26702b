"""Split stage launches (rbf_set_stage_split; Sec. 5.2, Eq. (bcEqn) and
Sec. 6.2).  Each stage runs as a launch of the wall set (the nodes whose
records the ghost residual reads and the nodes whose stencils read a ghost)
after the stage's ghost fill, and a launch of the other nodes on a second
stream, which overlaps the next stage's ghost fill.  No node's arithmetic
changes, so the states must be bitwise equal to the unsplit path: in graph
mode (runs of several graph replays plus leftover steps), in rbf_rk4_step,
for every lane count and both precisions, on a walled box (lateral and
corner ghosts) and on the periodic density current (top and bottom walls).
"""
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1509_02615_gb300 import configs  # noqa: E402
from paper_1509_02615_gb300 import rbffd  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1509_02615_gb300 import _build
    _build.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


CASES = {"bubble_500m": lambda: configs.bubble(h=500.0, seed=1, t_end=60.0),
         "density_current_400m": lambda: configs.density_current(400.0)}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("lanes", [1, 2, 4])
def test_split_is_bitwise_the_unsplit_path(case, precision, lanes):
    wl = CASES[case]()
    pb = rbffd.ns_problem(wl.nodes, precision=precision, threads_per_node=lanes, **wl.params)
    pb.set_run_mode("graph")
    out = {}
    for split in (True, False, True):
        pb.set_stage_split(split)
        A = rbffd.state_tensor(wl.U0, precision)
        pb.run(0.0, wl.dt, 37, A)      # two replays of the 16-step graph, then 5 leftover steps
        B = rbffd.state_tensor(wl.U0, precision)
        for k in range(3):
            pb.rk4_step(k * wl.dt, wl.dt, B)
        pb.sync()
        assert torch.all(torch.isfinite(A)) and torch.all(torch.isfinite(B))
        if split in out:
            # split runs are reproducible from run to run
            assert torch.equal(A, out[split][0]) and torch.equal(B, out[split][1])
        out[split] = (A, B)
    assert torch.equal(out[True][0], out[False][0]), f"{case} FP{precision} G={lanes}: graph runs differ"
    assert torch.equal(out[True][1], out[False][1]), f"{case} FP{precision} G={lanes}: rk4_step differs"
    # the run moved the state (the comparison is not of two untouched copies)
    assert not torch.equal(out[True][0], rbffd.state_tensor(wl.U0, precision))


def test_split_needs_a_wall_set():
    wl = configs.advection(16)
    pb = rbffd.advection_problem(wl.nodes, precision=64, **wl.params)
    with pytest.raises(rbffd.RBFError):
        pb.set_stage_split(True)


@pytest.mark.parametrize("precision", [64, 32])
def test_split_with_lattice_storage(precision):
    """The split's two node lists with lattice operator storage (class nodes
    read the class table, the others their own rows): bitwise the unsplit
    lattice run, on the hexagonal density current."""
    wl = configs.density_current(400.0)
    pb = rbffd.ns_problem(wl.nodes, precision=precision, threads_per_node=1, storage="lattice", **wl.params)
    pb.set_run_mode("graph")
    out = {}
    for split in (True, False):
        pb.set_stage_split(split)
        A = rbffd.state_tensor(wl.U0, precision)
        pb.run(0.0, wl.dt, 21, A)
        pb.sync()
        assert torch.all(torch.isfinite(A))
        out[split] = A
    assert pb.info()["stage_split"] == 0
    assert torch.equal(out[True], out[False])
