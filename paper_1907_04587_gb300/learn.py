"""Learned warm start: data generation from the solver, training, evaluation.

Every numerical step runs in libnsn's kernels (features, targets, BF16
tensor-core forward/backward, Adam); this module only drives them and moves
batches of device pointers around.
"""
from __future__ import annotations

import numpy as np

from . import nsn, scenes

NPARAM = nsn.NSN_MLP_NPARAM


def init_params(seed=0):
    """He-normal weights, zero biases (FP32, the layout of include/nsn.h)."""
    rng = np.random.default_rng(seed)
    out = []
    for fan_in, fan_out in ((16, 128), (128, 128), (128, 128), (128, 4)):
        out.append(rng.normal(0.0, np.sqrt(2.0 / fan_in), (fan_out, fan_in)).ravel())
        out.append(np.zeros(fan_out))
    p = np.concatenate(out).astype(np.float32)
    assert len(p) == NPARAM
    return p


def generate(seeds, n_envs=256, newton=5, cr=25, target_newton=12, target_cr=60):
    """(features, targets) on the device for every contact of batched scenes.

    For each seed: one plain step (so that each contact has a previous-step
    multiplier), then the features at the committed state, then one step with
    a larger budget whose final multipliers are the targets."""
    import torch
    Xs, Ts = [], []
    for seed in seeds:
        s = scenes.batched_envs(seed=seed, n_envs=n_envs)
        g = nsn.Solver(s, newton_iters=newton, cr_iters=cr)
        g.step()
        nc = len(s["c_body"])
        X = torch.empty((nc, 16), dtype=torch.float32, device="cuda")
        T = torch.empty((nc, 4), dtype=torch.float32, device="cuda")
        nsn.nsn_contact_features(g.ctx, X.data_ptr())
        st = g.get_state()
        lam_prev = g.get_lambda()
        g2 = nsn.Solver(s, newton_iters=target_newton, cr_iters=target_cr)
        g2.set_state(**st)
        g2.step()
        nsn.nsn_contact_features(g2.ctx, 0, T.data_ptr())
        torch.cuda.synchronize()
        Xs.append(X); Ts.append(T)
        del lam_prev
        g.close(); g2.close()
    return torch.cat(Xs), torch.cat(Ts)


class Trainer:
    """Owns a small solver context that hosts the network and its Adam state."""

    def __init__(self, params=None, seed=0):
        s = scenes.cube_stack(seed=0)
        self.host = nsn.Solver(s)
        nsn.nsn_mlp_set_params(self.host.ctx, init_params(seed) if params is None else params)

    def params(self):
        return nsn.nsn_mlp_get_params(self.host.ctx)[0]

    def train(self, X, T, epochs=2, batch=4096, lr=1e-3, weights=(1.0, 1.0, 1.0, 0.1), seed=0):
        import torch
        w = torch.tensor(weights, dtype=torch.float32, device="cuda")
        gen = torch.Generator(device="cuda").manual_seed(seed)
        n = len(X)
        hist = []
        for _ in range(epochs):
            perm = torch.randperm(n, device="cuda", generator=gen)
            for i in range(0, n - batch + 1, batch):
                idx = perm[i:i + batch]
                xb = X[idx].contiguous(); tb = T[idx].contiguous()
                hist.append(nsn.nsn_mlp_train_step(self.host.ctx, xb.data_ptr(), tb.data_ptr(), w.data_ptr(),
                                                   batch, lr))
        return hist


def compare_warm_starts(params, seed, n_envs=256, newton=5, cr=25):
    """Merit history of one step from the same state with the zero, previous
    step and learned warm starts (the relative merit is always against the
    zero start's merit)."""
    s = scenes.batched_envs(seed=seed, n_envs=n_envs)
    g = nsn.Solver(s, newton_iters=newton, cr_iters=cr)
    nsn.nsn_mlp_set_params(g.ctx, params)
    g.step()
    st = g.get_state()
    lam_prev_state = None
    out = {}
    modes = (("zero", nsn.NSN_WARM_ZERO), ("prev", nsn.NSN_WARM_PREV), ("learned", nsn.NSN_WARM_LEARNED),
             ("prev+friction", nsn.NSN_WARM_PREV | nsn.NSN_WARM_FRICTION),
             ("learned+friction", nsn.NSN_WARM_LEARNED | nsn.NSN_WARM_FRICTION))
    for name, mode in modes:
        h = nsn.Solver(s, newton_iters=newton, cr_iters=cr)
        nsn.nsn_mlp_set_params(h.ctx, params)
        h.step()                      # same first step: identical previous multipliers
        h.set_state(**st)
        h.set_warm_start(mode)
        r = h.step()
        mh = h.merit_history()
        out[name] = dict(rel=mh / r["merit0"], final_rel=r["merit_final"] / r["merit0"], warm=h.warm_stats())
        h.close()
    g.close()
    del lam_prev_state
    return out
