"""CPU pin of the FP64 reference network used to check the tensor-core
kernels: its analytic gradient equals central finite differences of its loss."""
import numpy as np

from oracle import mlp_ref


def test_reference_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = rng.normal(0, 0.2, mlp_ref.NPARAM)
    X = rng.normal(size=(7, 16))
    T = rng.normal(size=(7, 4))
    w = np.array([1.0, 0.5, 2.0, 0.1])
    _, g = mlp_ref.loss_and_grad(p, X, T, w)
    idx = rng.choice(mlp_ref.NPARAM, 60, replace=False)
    d = 1e-6
    for i in idx:
        e = np.zeros_like(p); e[i] = d
        lp, _ = mlp_ref.loss_and_grad(p + e, X, T, w)
        lm, _ = mlp_ref.loss_and_grad(p - e, X, T, w)
        assert abs((lp - lm) / (2 * d) - g[i]) < 1e-6 * max(1.0, abs(g[i]))


def test_reference_layout_is_the_abi_layout():
    # W1[128][16], b1[128], W2[128][128], b2, W3[128][128], b3, W4[4][128], b4[4]
    assert mlp_ref.NPARAM == 128 * 16 + 128 + 2 * (128 * 128 + 128) + 4 * 128 + 4
    p = np.arange(mlp_ref.NPARAM, dtype=np.float64)
    P = mlp_ref.unpack(p)
    assert P["W1"][1, 0] == 16 and P["b1"][0] == 128 * 16
    np.testing.assert_array_equal(mlp_ref.pack(P), p)
