"""Pins of the MLP oracle (no GPU): hand-written backpropagation against
central differences of the loss; BF16 rounding against the bit-level
definition; features against their definition on a lattice."""
import numpy as np

from oracle import mlp
from oracle import stencils as st
from paper_1509_02615_gb300 import inputs as inp


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    n_in, width, B = 12, 7, 9
    params = rng.normal(scale=0.4, size=mlp.n_params(n_in, width))
    X = rng.normal(size=(B, n_in))
    T = rng.normal(size=(B, 4))
    L, g = mlp.loss_and_grad(X, T, params, n_in, width)
    eps = 1e-6
    num = np.empty_like(params)
    for k in range(params.size):
        e = np.zeros_like(params)
        e[k] = eps
        num[k] = (mlp.loss_and_grad(X, T, params + e, n_in, width)[0] -
                  mlp.loss_and_grad(X, T, params - e, n_in, width)[0]) / (2 * eps)
    assert np.abs(num - g).max() <= 1e-7 * max(1.0, np.abs(g).max())


def test_bf16_round_definition():
    vals = np.array([1.0, 1.00390625, 1.005859375, -3.14159, 65504.0, 1e-3], np.float32)
    got = mlp.bf16_round(vals)
    for v, r in zip(vals, got):
        # the result is representable in bfloat16 (low 16 bits zero) and is the
        # nearest such value
        b = np.float32(r).view(np.uint32)
        assert b & 0xFFFF == 0
        down = np.uint32(np.float32(v).view(np.uint32) & 0xFFFF0000).view(np.float32)
        up = np.uint32((np.float32(v).view(np.uint32) & 0xFFFF0000) + 0x10000).view(np.float32)
        assert abs(r - v) <= min(abs(float(down) - v), abs(float(up) - v)) + 1e-30
    # ties go to even: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7
    assert mlp.bf16_round(np.array([1.00390625]))[0] == 1.0


def test_features_are_scaled_stencil_differences_and_values():
    nodes = inp.density_current_nodes(800.0)
    idx = st.knn(nodes.x, nodes.z, np.arange(nodes.n_prog), 37, nodes.period_x)
    U = np.random.default_rng(2).normal(size=(4, nodes.n_all))
    s_in = np.array([2.0, 3.0, 0.5, 1e-3])
    s_own = np.array([4.0, 5.0, 6.0, 7e-3])
    X = mlp.features(U, idx, np.array([5, 100]), s_in, s_own)
    assert X.shape == (2, 4 * 36 + 4)
    for r, i in enumerate((5, 100)):
        for f in range(4):
            for k in range(36):
                assert X[r, f * 36 + k] == (U[f, idx[i, k + 1]] - U[f, i]) / s_in[f]
            assert X[r, 4 * 36 + f] == U[f, i] / s_own[f]
