"""Learned warm start on the GPU: tensor-core forward/backward against the
FP64 reference network, training, and the warm-start modes of nsn_step."""
import numpy as np
import pytest

from oracle import mlp_ref
from paper_1907_04587_gb300 import learn, nsn, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    return torch


def bf16(a):
    import torch
    return torch.tensor(np.asarray(a, np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


def rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b)


def test_forward_and_gradients_match_fp64_reference(torch_cuda):
    torch = torch_cuda
    rng = np.random.default_rng(1)
    p = bf16(learn.init_params(3))                 # BF16-representable weights on both sides
    n = 200                                       # not a multiple of the 64-row tile
    X = bf16(rng.normal(size=(n, 16)))
    T = rng.normal(size=(n, 4)).astype(np.float32).astype(np.float64)
    w = np.array([1.0, 1.0, 1.0, 0.1], np.float32)
    tr = learn.Trainer(params=p.astype(np.float32))
    Xd = torch.tensor(X, dtype=torch.float32, device="cuda")
    Yd = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    nsn.nsn_mlp_forward(tr.host.ctx, Xd.data_ptr(), n, Yd.data_ptr())
    torch.cuda.synchronize()
    y_ref, _ = mlp_ref.forward(p, X)
    assert rel(Yd.cpu().numpy(), y_ref) < 2e-2
    Td = torch.tensor(T, dtype=torch.float32, device="cuda")
    wd = torch.tensor(w, device="cuda")
    loss = nsn.nsn_mlp_train_step(tr.host.ctx, Xd.data_ptr(), Td.data_ptr(), wd.data_ptr(), n, 0.0)
    l_ref, g_ref = mlp_ref.loss_and_grad(p, X, T, w.astype(np.float64))
    assert abs(loss - l_ref) < 2e-2 * l_ref
    _, g = nsn.nsn_mlp_get_params(tr.host.ctx)
    G, Gr = mlp_ref.unpack(g), mlp_ref.unpack(g_ref)
    for name in ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4"):
        assert rel(G[name], Gr[name]) < 5e-2, name


def test_forward_and_gradients_match_bf16_rounding_reference(torch_cuda):
    """Against the FP64 reference rounded to BF16 where the kernels round
    (inputs, weights, hidden activations, dY and dz for the GEMM operands):
    forward (the tensor-core inference kernel) and every gradient within 1e-3."""
    torch = torch_cuda
    rng = np.random.default_rng(5)
    p = learn.init_params(7)
    n = 333                                       # ragged against the 16- and 64-row tiles
    X = rng.normal(size=(n, 16)).astype(np.float32).astype(np.float64)
    T = rng.normal(size=(n, 4)).astype(np.float32).astype(np.float64)
    w = np.array([1.0, 1.0, 1.0, 0.1], np.float32)
    tr = learn.Trainer(params=p.astype(np.float32))
    Xd = torch.tensor(X, dtype=torch.float32, device="cuda")
    Yd = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    nsn.nsn_mlp_forward(tr.host.ctx, Xd.data_ptr(), n, Yd.data_ptr())
    torch.cuda.synchronize()
    y_ref, _ = mlp_ref.forward_bf16(p, X)
    e = rel(Yd.cpu().numpy(), y_ref)
    print(f"forward {e:.2e}")
    assert e < 1e-3
    Td = torch.tensor(T, dtype=torch.float32, device="cuda")
    wd = torch.tensor(w, device="cuda")
    loss = nsn.nsn_mlp_train_step(tr.host.ctx, Xd.data_ptr(), Td.data_ptr(), wd.data_ptr(), n, 0.0)
    l_ref, g_ref = mlp_ref.loss_and_grad_bf16(p, X, T, w.astype(np.float64))
    assert abs(loss - l_ref) < 1e-3 * l_ref
    _, g = nsn.nsn_mlp_get_params(tr.host.ctx)
    G, Gr = mlp_ref.unpack(g), mlp_ref.unpack(g_ref)
    for name in ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4"):
        e = rel(G[name], Gr[name])
        print(f"{name} {e:.2e}")
        assert e < 1e-3, name


@pytest.mark.parametrize("n", [1, 127, 128, 129, 50000])
@pytest.mark.parametrize("offset", [0, 1])
def test_tensor_core_inference_against_bf16_reference(torch_cuda, n, offset):
    """The inference kernel (tcgen05 MMAs, FP32 accumulators in tensor memory,
    128 rows per tile, persistent over tiles: 50,000 rows are 391 tiles on at
    most two CTAs per SM) against the FP64 network rounded to BF16 where the
    kernel rounds: one row, a tile less one, one tile, one more, many tiles;
    X at a 16-byte boundary and one float past it (scalar loads).  Norm-wise
    within 1e-3.  Element-wise, against each output's RMS: all but four rows'
    outputs and 0.1% of the rest within 2e-3, and all within 5e-2 -- an FP32
    sum order that differs from the reference's moves an activation that lies
    near a BF16 rounding boundary to the neighbouring BF16 value (2^-8 of it),
    and a few such flips in one row move that row's outputs by up to about 1%
    of the RMS."""
    torch = torch_cuda
    rng = np.random.default_rng(11 + n)
    p = learn.init_params(5)
    X = rng.normal(size=(n, 16)).astype(np.float32)
    tr = learn.Trainer(params=p.astype(np.float32))
    buf = torch.zeros(n * 16 + 4, dtype=torch.float32, device="cuda")
    buf[offset:offset + n * 16] = torch.from_numpy(X.ravel()).cuda()
    Xd = buf[offset:offset + n * 16]
    Yd = torch.full((n, 4), float("nan"), dtype=torch.float32, device="cuda")
    nsn.nsn_mlp_forward(tr.host.ctx, Xd.data_ptr(), n, Yd.data_ptr())
    torch.cuda.synchronize()
    y = Yd.cpu().numpy().astype(np.float64)
    y_ref, _ = mlp_ref.forward_bf16(p, X.astype(np.float64))
    assert np.isfinite(y).all()
    e = rel(y, y_ref) if n > 1 else np.abs(y - y_ref).max() / max(np.abs(y_ref).max(), 1e-30)
    scale = np.sqrt(np.mean(y_ref ** 2, axis=0)) + 1e-30
    d = np.abs(y - y_ref) / scale
    rows_off = int((d.max(axis=1) > 2e-3).sum())
    print(f"n {n} offset {offset}: norm-wise {e:.2e}, rows beyond 2e-3 of the RMS {rows_off}, "
          f"max {d.max():.2e}")
    assert e < 1e-3
    assert rows_off <= 4 + 0.001 * n
    assert d.max() < 5e-2
    # the timed entry point repeats the same call: bit-identical outputs
    ms = nsn.nsn_mlp_time_forward(tr.host.ctx, Xd.data_ptr(), n, Yd.data_ptr(), 3)
    assert ms > 0.0
    np.testing.assert_array_equal(Yd.cpu().numpy(), y.astype(np.float32))


def test_training_reduces_loss(torch_cuda):
    torch = torch_cuda
    rng = np.random.default_rng(2)
    teacher = learn.init_params(11) * 0.5
    X = rng.normal(size=(8192, 16)).astype(np.float32)
    T, _ = mlp_ref.forward(teacher.astype(np.float64), X.astype(np.float64))
    tr = learn.Trainer(seed=4)
    Xd = torch.tensor(X, device="cuda")
    Td = torch.tensor(T.astype(np.float32), device="cuda")
    hist = tr.train(Xd, Td, epochs=6, batch=1024, lr=3e-3)
    assert np.mean(hist[-4:]) < 0.3 * np.mean(hist[:4])


def test_warm_start_modes_and_fallback(torch_cuda):
    s = scenes.batched_envs(seed=9, n_envs=16)
    base = nsn.Solver(s, newton_iters=4, cr_iters=20)
    base.step()
    st = base.get_state()
    ref = nsn.Solver(s, newton_iters=4, cr_iters=20)
    ref.step(); ref.set_state(**st); r0 = ref.step()
    h0 = ref.merit_history()
    # previous-step warm start: accepted or rejected, never worse at the start
    g = nsn.Solver(s, newton_iters=4, cr_iters=20)
    g.step(); g.set_state(**st); g.set_warm_start(nsn.NSN_WARM_PREV)
    r = g.step()
    ws = g.warm_stats()
    assert ws["merit_warm"] <= ws["merit_zero"] or ws["rejected"]
    assert abs(r["merit0"] - r0["merit0"]) <= 1e-6 * r0["merit0"]
    # a network with huge outputs: its candidate must lose to the previous-step
    # fallback, and the step must then equal the previous-step warm start
    bad = learn.init_params(0)
    bad[-4:] = 1e4
    b = nsn.Solver(s, newton_iters=4, cr_iters=20)
    nsn.nsn_mlp_set_params(b.ctx, bad)
    b.step(); b.set_state(**st); b.set_warm_start(nsn.NSN_WARM_LEARNED)
    b.step()
    assert b.warm_stats()["rejected"]
    np.testing.assert_allclose(b.merit_history(), g.merit_history(), rtol=1e-5)


def test_learned_warm_start_after_training(torch_cuda):
    """Train on the solver's converged pairs (two seeds), evaluate on a held-out
    seed over an advancing trajectory: the learned start (the network's
    correction of the previous-step multipliers, with the previous-step
    fallback) converges at least as many islands as the zero start and as the
    previous-step start, in fewer Newton iterations than either (measured:
    islands 0.910 against 0.904, mean Newton iterations 11.7 against 12.4)."""
    params, hist, n = learn.train_warm_start(seeds=(100, 101), n_envs=64, steps=2, epochs=10, batch=1024)
    assert n > 1000 and np.mean(hist[-5:]) < np.mean(hist[:5])
    res = learn.compare_warm_starts(params, seed=5000, n_envs=64, steps=3)
    for k, v in res.items():
        print(k, "islands converged", round(v["island_fraction"], 4), "mean Newton to 1e-6", v["mean_newton"],
              "CR iterations", v["cr_total"])
    assert res["learned"]["island_fraction"] >= res["zero"]["island_fraction"] - 0.02
    assert res["learned"]["mean_newton"] < res["zero"]["mean_newton"]
    assert res["learned"]["island_fraction"] >= res["prev"]["island_fraction"]
    assert res["learned"]["mean_newton"] < res["prev"]["mean_newton"]
    # the learned preconditioner scale changes the CR iterates, not what the
    # islands converge to: as many islands reach the tolerance
    assert res["learned_precond"]["island_fraction"] >= res["learned"]["island_fraction"] - 0.03


def _probe_dense(g):
    """Dense A of the kept system, one operator apply per row (small scenes)."""
    import torch
    R = g.R
    A = np.zeros((R, R))
    x = torch.zeros(R, dtype=torch.float32, device="cuda")
    y = torch.zeros(R, dtype=torch.float32, device="cuda")
    for j in range(R):
        x.zero_(); x[j] = 1.0
        torch.cuda.synchronize()
        nsn.nsn_apply_operator_noalloc(g.ctx, x.data_ptr(), y.data_ptr())
        torch.cuda.synchronize()
        A[:, j] = y.double().cpu().numpy()
    return A


def test_precond_targets_equal_the_dense_inverse(torch_cuda):
    """The block-probing target (all islands' columns from one apply each)
    equals A_ii (A^-1)_ii of the contacts' normal rows from the dense A of the
    whole scene, and is >= 1 (Cauchy-Schwarz on an SPD matrix)."""
    s = scenes.batched_envs(seed=7, n_envs=3, links=(3, 4), boxes=(2, 8))
    g = nsn.Solver(s, **learn.SOLVE)
    g.step()
    sc = learn.precond_targets(g, s)
    A = _probe_dense(g)
    A = 0.5 * (A + A.T)
    inv = np.linalg.inv(A)
    nc = len(s["c_body"])
    ref = np.diag(A)[0:3 * nc:3] * np.diag(inv)[0:3 * nc:3]
    print("scales", np.round(sc[:8], 3), "min", sc.min(), "max", sc.max())
    np.testing.assert_allclose(sc, ref, rtol=1e-3)
    assert np.all(sc >= 1.0 - 1e-4)


def test_precond_scale_one_is_the_jacobi_preconditioner(torch_cuda):
    """A network whose fourth output is zero scales every contact by exp(0) = 1:
    the step is the one without the scale, to FP32 rounding of the CR
    iterations (the two launch configurations sum in different orders)."""
    s = scenes.batched_envs(seed=8, n_envs=4)
    p = learn.init_params(3)
    p[-4 * 128 - 4 + 3 * 128:-4 * 128 - 4 + 4 * 128] = 0.0   # fourth row of the last layer
    p[-1] = 0.0                                              # its bias
    out = []
    for mode in (nsn.NSN_WARM_LEARNED, nsn.NSN_WARM_LEARNED | nsn.NSN_WARM_PRECOND):
        g = nsn.Solver(s, **learn.SOLVE)
        nsn.nsn_mlp_set_params(g.ctx, p)
        g.set_warm_start(mode)
        g.step(); g.step()
        out.append(g.get_state())
    for k in ("pos", "vel", "omega"):
        np.testing.assert_allclose(out[0][k], out[1][k], rtol=0, atol=1e-6 * max(1.0, np.abs(out[0][k]).max()))
