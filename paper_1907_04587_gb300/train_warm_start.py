"""Trains the learned warm start on the solver's own converged solutions and
writes the network (raw-feature input) to weights/warm_start_mlp.npy.

    python -m paper_1907_04587_gb300.train_warm_start [--envs 512] [--epochs 20]

Needs a CUDA device; the solver, the network and its training run in libnsn's
kernels (the preconditioner-scale targets take dense inverses of the islands'
Schur blocks on the host).
"""
import argparse
import os
import time

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--envs", type=int, default=512)
    ap.add_argument("--seeds", type=int, nargs="+", default=[100, 101, 102, 103])
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--out", nargs="+", default=[os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights",
                                                               "warm_start_mlp.npy")])
    args = ap.parse_args()
    import torch
    torch.cuda.set_device(0)
    from . import learn, nsn
    nsn.lib()
    t0 = time.time()
    params, hist, n = learn.train_warm_start(seeds=args.seeds, n_envs=args.envs, steps=args.steps, epochs=args.epochs)
    print(f"{n} converged contact pairs, loss {hist[0]:.4g} -> {np.mean(hist[-20:]):.4g}, {time.time() - t0:.1f} s")
    for out in args.out:
        os.makedirs(os.path.dirname(os.path.abspath(out)), exist_ok=True)
        np.save(out, params)
        print("wrote", out)


if __name__ == "__main__":
    main()
