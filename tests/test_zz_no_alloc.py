"""Allocation-free operator apply (nsn_apply_operator_noalloc).

Callers that cannot allocate device memory where they need an operator
product -- a host application that owns the device's memory and leaves the
library no budget for it, a real-time loop that must not block in the device
allocator -- use this entry point; its scratch is a static device array in
the library.  The tests call it through the C ABI and compare it with the
allocating apply (nsn_apply_operator) and with the FP64 oracle's operator.
This file is collected last so that a failure here comes after every other
test has run; it also passes when run alone in a fresh process.
"""
import numpy as np
import pytest

from paper_1907_04587_gb300 import nsn, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    return torch


def _rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b)


def test_noalloc_apply_matches_allocating_apply_twice(torch_cuda):
    torch = torch_cuda
    s = scenes.chain_block(seed=7, hexes=3, links=5)   # rigid and particle entries, tets, joints
    g = nsn.Solver(s, precision=nsn.NSN_FP32, newton_iters=3, cr_iters=10)
    g.linearize(1)
    rng = np.random.default_rng(21)
    for call in range(2):
        x = rng.normal(size=g.R).astype(np.float32).astype(np.float64)
        y_ref = g.apply(x)                                   # existing entry point
        xd = torch.tensor(x, dtype=torch.float32, device="cuda")
        yd = torch.full_like(xd, float("nan"))
        nsn.nsn_apply_operator_noalloc(g.ctx, xd.data_ptr(), yd.data_ptr())
        torch.cuda.synchronize()
        assert _rel(yd.cpu().numpy(), y_ref) < 1e-5, call


def test_noalloc_after_step_and_on_batched_scene(torch_cuda):
    torch = torch_cuda
    s = scenes.batched_envs(seed=4, n_envs=20)
    g = nsn.Solver(s, precision=nsn.NSN_FP32, newton_iters=2, cr_iters=5)
    g.step()
    g.linearize(0)
    x = np.random.default_rng(3).normal(size=g.R)
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    y_ref = g.apply(xd.cpu().numpy().astype(np.float64))
    for _ in range(2):
        yd = torch.empty_like(xd)
        nsn.nsn_apply_operator_noalloc(g.ctx, xd.data_ptr(), yd.data_ptr())
        torch.cuda.synchronize()
        assert _rel(yd.cpu().numpy(), y_ref) < 1e-5


def test_noalloc_rejects_too_many_entries(torch_cuda):
    torch = torch_cuda
    s = scenes.batched_envs(seed=5, n_envs=6000)
    g = nsn.Solver(s, precision=nsn.NSN_FP32, newton_iters=1, cr_iters=1)
    sz = g.sizes()
    assert 2 * sz["pair_rows"] + 12 * sz["tets"] > 4 * 1024 * 1024
    g.linearize(0)
    xd = torch.zeros(g.R, dtype=torch.float32, device="cuda")
    yd = torch.zeros_like(xd)
    with pytest.raises(nsn.NSNError, match="exceed the static scratch"):
        nsn.nsn_apply_operator_noalloc(g.ctx, xd.data_ptr(), yd.data_ptr())


def test_noalloc_apply_matches_oracle_operator(torch_cuda, orc):
    """At the zero iterate of a step (u = 0, lambda = 0: identical inputs on
    both sides) the allocation-free product equals the FP64 oracle's
    y = (J H~^-1 J^T + C + eps I) x (Eq. schur_system, Sec. 8.4) within the
    FP32 tolerance of the linear-system parity tests, on two calls in a row."""
    torch = torch_cuda
    s = scenes.chain_block(seed=5, hexes=3, links=4)   # contacts, joints, tets
    p = dict(newton_iters=3, cr_iters=10)
    o = orc.Oracle(s, **p)
    o.linearize(n_before=0)
    g = nsn.Solver(s, precision=nsn.NSN_FP32, **p)
    g.linearize(0)
    rng = np.random.default_rng(8)
    for call in range(2):
        x = rng.normal(size=g.R).astype(np.float32).astype(np.float64)
        xd = torch.tensor(x, dtype=torch.float32, device="cuda")
        yd = torch.full_like(xd, float("nan"))
        nsn.nsn_apply_operator_noalloc(g.ctx, xd.data_ptr(), yd.data_ptr())
        torch.cuda.synchronize()
        assert _rel(yd.cpu().numpy(), o.apply_A(x)) < 1e-5, call
