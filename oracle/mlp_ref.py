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


# --------------------------------------------------------------------------
# The same network with the rounding of the tensor-core kernels: BF16 inputs,
# weights and hidden activations (round to nearest even of the FP32 value),
# FP32 biases and outputs, exact products, sums in FP64 (the kernels sum in
# FP32: their results differ from these by the FP32 accumulation error, and,
# where that moves a value across a BF16 rounding boundary, by one BF16 unit
# in that activation).  Backward as the training kernels round it: dY and
# dz in BF16 for the GEMM operands, in FP32 for the bias sums; the ReLU mask
# from the FP32 activation.

def round_bf16(a):
    """Round to the nearest BF16 value (ties to even), via the FP32 value."""
    f = np.ascontiguousarray(np.asarray(a, np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _f32(a):
    return np.asarray(a, np.float64).astype(np.float32).astype(np.float64)


def forward_bf16(p, X):
    P = unpack(p)
    W = {k: round_bf16(P[k]) for k in ("W1", "W2", "W3", "W4")}
    b = {k: _f32(P[k]) for k in ("b1", "b2", "b3", "b4")}
    a0 = round_bf16(X)
    z1 = _f32(a0 @ W["W1"].T + b["b1"]); a1f = np.maximum(z1, 0); a1 = round_bf16(a1f)
    z2 = _f32(a1 @ W["W2"].T + b["b2"]); a2f = np.maximum(z2, 0); a2 = round_bf16(a2f)
    z3 = _f32(a2 @ W["W3"].T + b["b3"]); a3f = np.maximum(z3, 0); a3 = round_bf16(a3f)
    y = _f32(a3 @ W["W4"].T + b["b4"])
    return y, (a0, a1f, a1, a2f, a2, a3f, a3, W)


def loss_and_grad_bf16(p, X, T, w):
    y, (a0, a1f, a1, a2f, a2, a3f, a3, W) = forward_bf16(p, X)
    n = len(X)
    d = y - np.asarray(T, np.float64)
    loss = 0.5 * float((w * d * d).sum()) / n
    dyf = _f32(w * d / n)
    dyb = round_bf16(dyf)
    g = {"W4": dyb.T @ a3, "b4": dyf.sum(0)}
    da = _f32(dyb @ W["W4"])
    dzf = da * (a3f > 0); dzb = round_bf16(dzf)
    g["W3"] = dzb.T @ a2; g["b3"] = dzf.sum(0)
    da = _f32(dzb @ W["W3"])
    dzf = da * (a2f > 0); dzb = round_bf16(dzf)
    g["W2"] = dzb.T @ a1; g["b2"] = dzf.sum(0)
    da = _f32(dzb @ W["W2"])
    dzf = da * (a1f > 0); dzb = round_bf16(dzf)
    g["W1"] = dzb.T @ a0; g["b1"] = dzf.sum(0)
    return loss, pack(g)
