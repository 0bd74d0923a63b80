"""FP64 numpy reference of the warm-start network (test infrastructure).

16 -> 128 -> 128 -> 128 -> 4 with ReLU, y = W x + b per layer; loss
L = 1/(2n) sum_i sum_k w_k (y_ik - t_ik)^2.  Forward and backward are written
out layer by layer from the definition (chain rule), in double precision; the
CPU tests pin the gradient against central finite differences.  The parameter
vector layout is W1[128][16], b1, W2[128][128], b2, W3[128][128], b3,
W4[4][128], b4.
"""
import numpy as np

NIN, NH, NOUT = 16, 128, 4
SHAPES = [("W1", (NH, NIN)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("W3", (NH, NH)), ("b3", (NH,)),
          ("W4", (NOUT, NH)), ("b4", (NOUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(p):
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(p[o:o + n], np.float64).reshape(shp)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], np.float64).ravel() for name, _ in SHAPES])


def forward(p, X):
    P = unpack(p)
    a0 = np.asarray(X, np.float64)
    z1 = a0 @ P["W1"].T + P["b1"]; a1 = np.maximum(z1, 0)
    z2 = a1 @ P["W2"].T + P["b2"]; a2 = np.maximum(z2, 0)
    z3 = a2 @ P["W3"].T + P["b3"]; a3 = np.maximum(z3, 0)
    y = a3 @ P["W4"].T + P["b4"]
    return y, (a0, z1, a1, z2, a2, z3, a3)


def loss_and_grad(p, X, T, w):
    P = unpack(p)
    y, (a0, z1, a1, z2, a2, z3, a3) = forward(p, X)
    n = len(X)
    d = y - T
    loss = 0.5 * float((w * d * d).sum()) / n
    dy = w * d / n
    g = {"W4": dy.T @ a3, "b4": dy.sum(0)}
    da3 = dy @ P["W4"]; dz3 = da3 * (z3 > 0)
    g["W3"] = dz3.T @ a2; g["b3"] = dz3.sum(0)
    da2 = dz3 @ P["W3"]; dz2 = da2 * (z2 > 0)
    g["W2"] = dz2.T @ a1; g["b2"] = dz2.sum(0)
    da1 = dz2 @ P["W2"]; dz1 = da1 * (z1 > 0)
    g["W1"] = dz1.T @ a0; g["b1"] = dz1.sum(0)
    return loss, pack(g)
