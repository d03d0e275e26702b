"""a9: learned coarse-grid correction (GPU, through the C ABI).

* Gradients: the training kernel's loss and gradient on a fixed batch match
  the FP64 oracle (oracle/mlp.py, hand-written backprop pinned by central
  differences) evaluated with the same BF16-rounded weights and the same
  FP32 states: relative l2 < 1e-3 (FP32 accumulation, FP32 tanh).
* Forward: the fused gather + MLP kernel matches the oracle forward pass.
* Gain: trained on fine runs restricted to the coarse nodes, the corrected
  coarse runs of held-out seeds end closer to the fine reference than the
  uncorrected coarse runs.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import mlp as omlp  # noqa: E402
from oracle import stencils as ost  # noqa: E402
from oracle.ns import NSOracle  # noqa: E402
from paper_1509_02615_gb300 import inputs as inp  # noqa: E402
from paper_1509_02615_gb300 import learned  # noqa: E402
from paper_1509_02615_gb300 import rbffd  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1509_02615_gb300 import _build
    _build.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def small_data():
    """Seeded synthetic data set on the 800 m lattice: states with ghosts
    filled by the oracle's ghost solve, random targets."""
    nodes = inp.density_current_nodes(800.0)
    o = NSOracle(nodes)
    rng = np.random.default_rng(4)
    R, n_snap = 2, 3
    S = np.zeros((R, n_snap, nodes.n_all, 4))
    for r in range(R):
        for k in range(n_snap):
            U = inp.perturbed_density_current(nodes, 10 * r + k)
            U[:, :nodes.n_prog] += 0.3 * rng.normal(size=(4, nodes.n_prog)) * np.array([[5.0], [3.0], [1.0], [1e-3]])
            o.fill_ghosts(U)
            S[r, k] = U.T
    T = rng.normal(size=(R, n_snap - 1, nodes.n_prog, 4)) * np.array([0.1, 0.05, 0.02, 1e-5])
    idx = ost.knn(nodes.x, nodes.z, np.arange(nodes.n_prog), 37, nodes.period_x)
    return nodes, S.astype(np.float32), T.astype(np.float32), idx, R, n_snap


def test_training_gradient_matches_oracle(small_data):
    nodes, S, T, idx, R, n_snap = small_data
    coarse = rbffd.ns_problem(nodes, precision=32)
    mlp = rbffd.Mlp(coarse)
    n_in = 4 * 36 + 4
    params = learned.init_params(n_in, seed=3)
    params[-4:] = [0.05, -0.02, 0.01, 0.03]
    mlp.set_params(params)
    scales = np.array([2.0, 1.5, 0.5, 2e-4, 0.1, 0.05, 0.02, 1e-5, 4.0, 3.0, 6.0, 1e-3], np.float32)
    mlp.set_scales(scales)
    rng = np.random.default_rng(9)
    B = 300   # three training blocks, the last one partly filled
    ks = rng.integers(0, R * (n_snap - 1), B)
    iis = rng.integers(0, nodes.n_prog, B)
    samples = torch.as_tensor(np.stack([ks, iis], 1), dtype=torch.int64, device="cuda").contiguous()
    St = torch.as_tensor(S, device="cuda").contiguous()
    Tt = torch.as_tensor(T, device="cuda").contiguous()
    loss, g = mlp.grad(St, Tt, R, n_snap, samples)
    # oracle: same FP32 states, BF16-rounded weights, FP64 arithmetic
    w = omlp.bf16_round(params)
    off = n_in * 64
    for o, cnt in ((off, 64), (off + 64 + 64 * 64, 64), (len(params) - 4, 4)):   # biases stay FP32
        w[o:o + cnt] = params[o:o + cnt]
    X = np.zeros((B, n_in))
    Tg = np.zeros((B, 4))
    for b in range(B):
        k = ks[b]
        st = (k // (n_snap - 1)) * n_snap + k % (n_snap - 1)
        U = S.reshape(R * n_snap, nodes.n_all, 4)[st].astype(np.float64).T
        X[b] = omlp.features(U, idx, np.array([iis[b]]), scales[:4].astype(np.float64),
                             scales[8:].astype(np.float64))[0]
        Tg[b] = T.reshape(-1, nodes.n_prog, 4)[k, iis[b]] / scales[4:8].astype(np.float64)
    L, gref = omlp.loss_and_grad(X, Tg, w, n_in, 64)
    print("loss gpu %.6e oracle %.6e; grad rel l2 %.3e" % (loss, L, rel(g, gref)))
    assert abs(loss - L) <= 1e-4 * abs(L)
    assert rel(g, gref) < 1e-3


def test_forward_matches_oracle(small_data):
    nodes, S, T, idx, R, n_snap = small_data
    coarse = rbffd.ns_problem(nodes, precision=32)
    mlp = rbffd.Mlp(coarse)
    params = learned.init_params(4 * 36 + 4, seed=5)
    mlp.set_params(params)
    scales = np.array([2.0, 1.5, 0.5, 2e-4, 0.1, 0.05, 0.02, 1e-5, 4.0, 3.0, 6.0, 1e-3], np.float32)
    mlp.set_scales(scales)
    U = torch.as_tensor(S[0, 1], device="cuda").contiguous()
    d = mlp.forward(U).cpu().numpy().astype(np.float64)
    w = omlp.bf16_round(params)
    n_in = 4 * 36 + 4
    off = n_in * 64
    for o, cnt in ((off, 64), (off + 64 + 64 * 64, 64), (len(params) - 4, 4)):
        w[o:o + cnt] = params[o:o + cnt]
    X = omlp.features(S[0, 1].astype(np.float64).T, idx, np.arange(nodes.n_prog), scales[:4].astype(np.float64),
                      scales[8:].astype(np.float64))
    y = np.clip(omlp.forward(X, w, n_in, 64)[2], -4.0, 4.0) * scales[4:8].astype(np.float64)
    y[nodes.kind == inp.KIND_BOTTOM, 1] = 0.0
    y[nodes.kind == inp.KIND_TOP, 1] = 0.0
    assert rel(d, y) < 1e-4, rel(d, y)


def test_correction_on_held_out_seeds():
    """400 m coarse runs corrected by an MLP trained on 100 m FP64 runs
    restricted to the coarse nodes (10 training seeds, 30k iterations: the
    bench's setting); the per-field strength is chosen on 3 validation seeds
    among candidates that include the uncorrected solver; 3 held-out seeds are
    scored at 900 s against the restricted 100 m reference.  The selected
    strength must be non-zero and the corrected mean error at least 15% below
    the uncorrected one (the bench measures about 30%)."""
    seeds = inp.learned_correction_seeds(16, seed=1)
    ds = learned.build_dataset(400.0, 4, seeds, 900.0)
    mlp, loss = learned.train(ds, 10, iters=30000, batch=4096, lr=2e-3)
    assert loss[-50:].mean() < 0.2 * loss[:50].mean()
    alpha, scores = learned.select_alpha(ds, mlp, range(10, 13))
    test = range(13, 16)
    ep = learned.run_errors(ds, mlp, test, (0.0, 0.0, 0.0, 0.0))
    el = learned.run_errors(ds, mlp, test, alpha)
    skill = learned.prediction_skill(ds, mlp, range(10, 13))
    print("validation scores", scores)
    print("selected alpha", alpha, "held-out relative l2 [u, w, theta', pi']: uncorrected", ep, "corrected", el,
          f"gain {1.0 - np.mean(el) / np.mean(ep):.3f}; validation skill per field", skill)
    assert np.all(np.isfinite(el))
    assert any(a > 0.0 for a in alpha), alpha
    assert np.mean(el) < 0.85 * np.mean(ep), (np.mean(el), np.mean(ep))


def test_training_is_deterministic(small_data):
    """Per-block gradient partials summed in block order, and the scale sums
    added per warp in warp order: two trainings from the same data and seed
    give the same scales, losses and parameters, bit for bit."""
    nodes, S, T, idx, R, n_snap = small_data
    pb = rbffd.ns_problem(nodes, precision=32, threads_per_node=1)
    St = torch.as_tensor(S, device="cuda")
    Tt = torch.as_tensor(T, device="cuda")
    out = []
    for _ in range(2):
        mlp = rbffd.Mlp(pb)
        mlp.set_params(learned.init_params(4 * 36 + 4, seed=3))
        mlp.fit_scales(St, Tt, R, n_snap)
        loss = mlp.train(St, Tt, R, n_snap, 300, batch=512, lr=2e-3, seed=5)
        out.append((mlp.scales(), loss, mlp.params()))
        mlp.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    assert np.array_equal(out[0][2], out[1][2])
    assert np.all(np.isfinite(out[0][1])) and out[0][1][-1] < out[0][1][0]
