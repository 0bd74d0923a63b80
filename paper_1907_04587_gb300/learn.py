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


SOLVE = dict(newton_iters=30, cr_iters=50, tol_rel=1e-6, island_stop=1, cone_project=1)


def contact_islands(g, s):
    """Island of every contact (that of its first non-world body)."""
    _, bi = g.islands()
    cb = np.asarray(s["c_body"])
    return bi[np.where(cb[:, 0] >= 0, cb[:, 0], cb[:, 1])]


def generate(seeds, n_envs=512, steps=3, solve=None):
    """(features, targets) on the device from the solver's own trajectories.

    For each seed, a batched scene is advanced `steps` steps by the island
    solver to a relative residual of 1e-6.  Before each step the contact
    features are taken at the committed state (the previous-step multipliers
    among them); after it, the converged multipliers are the targets.  Only
    contacts of islands that reached the tolerance are kept, so every target
    is a converged solution."""
    import torch
    Xs, Ts = [], []
    for seed in seeds:
        s = scenes.batched_envs(seed=seed, n_envs=n_envs)
        g = nsn.Solver(s, **(solve or SOLVE))
        cisl = contact_islands(g, s)
        nc = len(s["c_body"])
        for _ in range(steps):
            X = torch.empty((nc, 16), dtype=torch.float32, device="cuda")
            T = torch.empty((nc, 4), dtype=torch.float32, device="cuda")
            nsn.nsn_contact_features(g.ctx, X.data_ptr())
            g.step()
            nsn.nsn_contact_features(g.ctx, 0, T.data_ptr())
            ok = g.island_stats()["stopped_at"][cisl] >= 0
            keep = torch.from_numpy(np.nonzero(ok)[0]).to("cuda")
            torch.cuda.synchronize()
            Xs.append(X[keep]); Ts.append(T[keep])
        g.close()
    return torch.cat(Xs), torch.cat(Ts)


def standardization(X):
    """Per-feature mean and scale (scale 1 where a feature does not vary)."""
    mu = X.mean(0)
    sd = X.std(0)
    sd = sd.where(sd > 1e-6, sd.new_ones(()))
    return mu, sd


def fold_standardization(params, mu, sd):
    """A network trained on (x - mu) / sd as one acting on x: W1 / sd, and
    b1 - (W1 / sd) mu."""
    p = np.array(params, dtype=np.float64)
    mu = np.asarray(mu, np.float64); sd = np.asarray(sd, np.float64)
    W1 = p[:128 * 16].reshape(128, 16) / sd[None, :]
    b1 = p[128 * 16:128 * 16 + 128] - W1 @ mu
    p[:128 * 16] = W1.ravel()
    p[128 * 16:128 * 16 + 128] = b1
    return p.astype(np.float32)


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


def train_warm_start(seeds=(100, 101, 102, 103), n_envs=512, steps=3, epochs=20, batch=4096, lr=1e-3,
                     weights=(1.0, 0.1, 0.1, 0.0), seed=1):
    """Data from the solver, standardised inputs, training on the tensor
    cores; returns (params acting on raw features, loss history, pairs)."""
    X, T = generate(list(seeds), n_envs=n_envs, steps=steps)
    mu, sd = standardization(X)
    tr = Trainer(seed=seed)
    hist = tr.train(((X - mu) / sd).contiguous(), T, epochs=epochs, batch=batch, lr=lr, weights=weights, seed=seed)
    params = fold_standardization(tr.params(), mu.cpu().numpy(), sd.cpu().numpy())
    tr.host.close()
    return params, hist, len(X)


def compare_warm_starts(params, seed, n_envs=256, steps=3, solve=None):
    """Per warm-start mode, over `steps` advancing steps from the same start:
    the share of islands that reached the tolerance and their mean Newton
    iterations to it."""
    s = scenes.batched_envs(seed=seed, n_envs=n_envs)
    out = {}
    for name, mode in (("zero", nsn.NSN_WARM_ZERO), ("prev", nsn.NSN_WARM_PREV), ("learned", nsn.NSN_WARM_LEARNED)):
        g = nsn.Solver(s, **(solve or SOLVE))
        nsn.nsn_mlp_set_params(g.ctx, params)
        g.set_warm_start(mode)
        stops, warm = [], []
        for _ in range(steps):
            g.step()
            stops.append(g.island_stats()["stopped_at"].copy())
            warm.append(g.warm_stats())
        g.close()
        st = np.concatenate(stops)
        ok = st >= 0
        out[name] = dict(island_fraction=float(ok.mean()), mean_newton=float(st[ok].mean()) if ok.any() else None,
                         warm=warm)
    return out
