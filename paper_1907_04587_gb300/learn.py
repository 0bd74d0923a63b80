"""Learned warm start: data generation from the solver, training, evaluation.

Every numerical step of the solver and the network runs in libnsn's kernels
(features, targets, operator applies, BF16 tensor-core forward/backward,
Adam); this module drives them and moves batches of device pointers around.
The one host computation is the preconditioner-scale target: dense inverses
of the islands' Schur blocks (precond_targets).
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


def island_rows(g, s):
    """Rows (ABI order) of every island that has rows: contact rows 3c..3c+2,
    then joint rows 3 nc + 5j..5j+4, each island's rows ascending."""
    _, bi = g.islands()
    nc = len(s["c_body"])
    cb = np.asarray(s["c_body"]); jb = np.asarray(s["j_body"]).reshape(-1, 2) if len(s["j_body"]) else np.zeros((0, 2), int)
    ci = bi[np.where(cb[:, 0] >= 0, cb[:, 0], cb[:, 1])]
    ji = bi[np.where(jb[:, 0] >= 0, jb[:, 0], jb[:, 1])] if len(jb) else np.zeros(0, int)
    row_isl = np.concatenate([np.repeat(ci, 3), np.repeat(ji, 5)])
    order = np.argsort(row_isl, kind="stable")
    isl_sorted = row_isl[order]
    starts = np.searchsorted(isl_sorted, np.unique(isl_sorted))
    return np.split(order, starts[1:]), row_isl


def precond_targets(g, s):
    """Per contact, A_ii (A^-1)_ii of its normal row for the system kept by
    the last step (its final evaluation): the diagonal of the inverse over the
    Jacobi diagonal, the scale that turns Jacobi into the exact diagonal of
    A^-1.  A (Eq. schur_system) is block diagonal by island, so one operator
    apply (libnsn's CR kernels, nsn_apply_operator_noalloc) on the sum of every
    island's j-th unit row vector gives column j of every island's block at
    once: as many applies as the largest island has rows.  The blocks are then
    inverted on the host in FP64 (training-data preparation, not the solver)."""
    import torch
    blocks, _ = island_rows(g, s)
    R = g.R
    nc = len(s["c_body"])
    sizes = np.array([len(b) for b in blocks])
    classes = {int(n): torch.from_numpy(np.stack([blocks[i] for i in np.nonzero(sizes == n)[0]])).cuda()
               for n in np.unique(sizes)}
    A = {n: torch.zeros((len(ri), n, n), dtype=torch.float32, device="cuda") for n, ri in classes.items()}
    x = torch.zeros(R, dtype=torch.float32, device="cuda")
    y = torch.zeros(R, dtype=torch.float32, device="cuda")
    for j in range(int(sizes.max())):
        x.zero_()
        for n, ri in classes.items():
            if n > j:
                x[ri[:, j]] = 1.0
        torch.cuda.synchronize()
        nsn.nsn_apply_operator_noalloc(g.ctx, x.data_ptr(), y.data_ptr())
        torch.cuda.synchronize()
        for n, ri in classes.items():
            if n > j:
                A[n][:, :, j] = y[ri]
    out = np.ones(nc)
    for n, ri in classes.items():
        An = A[n].double().cpu().numpy()
        An = 0.5 * (An + An.transpose(0, 2, 1))
        inv = np.linalg.inv(An)
        sc = np.einsum("kii->ki", An) * np.einsum("kii->ki", inv)
        rows = ri.cpu().numpy()
        normal = (rows < 3 * nc) & (rows % 3 == 0)
        out[rows[normal] // 3] = sc[normal]
    return out


def generate(seeds, n_envs=512, steps=3, solve=None, precond=True):
    """(features, targets) on the device from the solver's own trajectories.

    For each seed, a batched scene is advanced `steps` steps by the island
    solver to a relative residual of 1e-6.  Before each step the contact
    features are taken at the committed state (the previous-step multipliers
    among them); after it, the change from those to the converged multipliers
    is the target (the difference taken on the device by torch).  Only
    contacts of islands that reached the tolerance are kept, so every target
    is a converged solution.  The fourth target is the logarithm of the
    contact's preconditioner scale (precond_targets) at the converged state."""
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
            # the network predicts the change from the previous-step multipliers
            # (features 9..11, over the same lambda_s)
            T[:, :3] -= X[:, 9:12]
            if precond:
                # log scale, clamped to the range the solver applies ([1, 4]:
                # nearly singular blocks of redundant contacts give ratios of 1e7)
                sc = precond_targets(g, s)
                T[:, 3] = torch.from_numpy(np.log(np.clip(sc, 1.0, 4.0))).to(T)
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
                     weights=(1.0, 0.1, 0.1, 0.1), seed=1):
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
    """Per warm-start mode (zero, previous step, learned, learned with the
    preconditioner scale), over `steps` advancing steps from the same start:
    the share of islands that reached the tolerance, their mean Newton
    iterations to it and the CR iterations of the steps."""
    s = scenes.batched_envs(seed=seed, n_envs=n_envs)
    out = {}
    for name, mode in (("zero", nsn.NSN_WARM_ZERO), ("prev", nsn.NSN_WARM_PREV), ("learned", nsn.NSN_WARM_LEARNED),
                       ("learned_precond", nsn.NSN_WARM_LEARNED | nsn.NSN_WARM_PRECOND)):
        g = nsn.Solver(s, **(solve or SOLVE))
        nsn.nsn_mlp_set_params(g.ctx, params)
        g.set_warm_start(mode)
        stops, warm, cr = [], [], 0
        for _ in range(steps):
            r = g.step()
            cr += r["cr_total"]
            stops.append(g.island_stats()["stopped_at"].copy())
            warm.append(g.warm_stats())
        g.close()
        st = np.concatenate(stops)
        ok = st >= 0
        out[name] = dict(island_fraction=float(ok.mean()), mean_newton=float(st[ok].mean()) if ok.any() else None,
                         cr_total=int(cr), warm=warm)
    return out
