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


def test_bf16_rounding():
    """round_bf16 against values whose BF16 rounding is known: exact BF16
    values stay, a value just above a midpoint rounds up, a tie rounds to the
    even mantissa, and the result always has 8 significant bits."""
    one = 1.0
    ulp = 2.0 ** -7                                  # BF16 spacing in [1, 2)
    assert mlp_ref.round_bf16(np.array([one]))[0] == one
    assert mlp_ref.round_bf16(np.array([one + ulp]))[0] == one + ulp
    assert mlp_ref.round_bf16(np.array([one + 0.5 * ulp]))[0] == one          # tie: even (1.0)
    assert mlp_ref.round_bf16(np.array([one + 1.5 * ulp]))[0] == one + 2 * ulp  # tie: even (1 + 2 ulp)
    assert mlp_ref.round_bf16(np.array([one + 0.51 * ulp]))[0] == one + ulp
    assert mlp_ref.round_bf16(np.array([-(one + 0.49 * ulp)]))[0] == -one
    x = np.random.default_rng(0).normal(size=1000)
    r = mlp_ref.round_bf16(x)
    m, e = np.frexp(r)
    assert np.all(m * 2 ** 8 == np.round(m * 2 ** 8))
    assert np.all(np.abs(r - x) <= 2.0 ** -8 * np.abs(x) * 1.0001)


def test_bf16_reference_stays_within_bf16_rounding_of_fp64():
    """The BF16-rounded network differs from the FP64 one by the BF16 unit
    (2^-8 relative per rounding, a few roundings deep), neither more nor
    (as a check that the rounding is applied at all) much less."""
    rng = np.random.default_rng(3)
    p = np.concatenate([rng.normal(0, 0.3, s).ravel() for _, s in mlp_ref.SHAPES])
    X = rng.normal(size=(40, mlp_ref.NIN)); T = rng.normal(size=(40, mlp_ref.NOUT)); w = np.array([1, 1, 1, 0.1])
    y64, _ = mlp_ref.forward(p, X)
    y16, _ = mlp_ref.forward_bf16(p, X)
    e = np.linalg.norm(y16 - y64) / np.linalg.norm(y64)
    assert 1e-4 < e < 3e-2
    l64, g64 = mlp_ref.loss_and_grad(p, X, T, w)
    l16, g16 = mlp_ref.loss_and_grad_bf16(p, X, T, w)
    assert abs(l16 - l64) < 3e-2 * l64
    assert np.linalg.norm(g16 - g64) < 5e-2 * np.linalg.norm(g64)
