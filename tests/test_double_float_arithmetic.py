"""The double-float arithmetic (FP32 pairs) that the device uses in two places instead of FP64,
checked on the CPU with an independent numpy restatement of the error-free transformations
(TwoSum: Knuth; TwoProd with a fused multiply-add: Ogita, Rump & Oishi, 2005):

  * the rank-1 row update (h, l) += s (xh + xl)(ah + al) of the sliced compose's neighbour
    rows (Cor. 1 across one flipped neuron): the result is within 2^-44 of the exact value,
    relative to |row| + |update|, on random pairs (exact reference: rational arithmetic);
  * the triggers' forward pass of a plain ReLU MLP (Eq. 1) evaluated on pairs: F agrees with
    an FP64 evaluation to about 1e-12 of sum |w||h| on nets of the bench's shape, and every
    pattern bit whose FP64 pre-activation is farther than 1e-9 of its own scale from zero is
    the same.

The FMA is modelled as the exact product plus the addend in FP64, rounded once to FP32 (a
product of two FP32 values is exact in FP64; the further FP64 rounding of the sum is below
the FP32 one).  This pins the arithmetic, not the CUDA code, whose seeds and meshes the GPU
tests compare with the oracle's.
"""
from fractions import Fraction

import numpy as np

F32, F64 = np.float32, np.float64


def fma32(a, b, c):
    return (a.astype(F64) * b.astype(F64) + c.astype(F64)).astype(F32)


def split(x):
    """An FP64 value as an FP32 pair (hi, lo), hi + lo = x to about 2^-48 relative."""
    h = np.asarray(x, dtype=F64).astype(F32)
    return h, (np.asarray(x, dtype=F64) - h.astype(F64)).astype(F32)


def df_fma(sh, sl, ah, al, zh, zl):
    """(sh, sl) += (ah + al)(zh + zl): TwoProd of the hi words, the cross terms into the error,
    TwoSum of the hi words, the error terms into the low word."""
    p = (ah * zh).astype(F32)
    pe = fma32(ah, zh, -p)
    pe = fma32(ah, zl, pe)
    pe = fma32(al, zh, pe)
    t = (sh + p).astype(F32)
    bp = (t - sh).astype(F32)
    te = ((sh - (t - bp)) + (p - bp)).astype(F32)
    return t, (sl + (te + pe)).astype(F32)


def df_norm(h, l):
    s = (h + l).astype(F32)
    return s, (l - (s - h)).astype(F32)


def exact(x):
    return Fraction(float(x))


def test_rank1_row_update_is_within_2_to_the_minus_44():
    rng = np.random.default_rng(11)
    n = 400
    h, l = split(rng.standard_normal(n) * np.exp(rng.uniform(-3, 3, n)))
    xh, xl = split(rng.standard_normal(n) * np.exp(rng.uniform(-3, 3, n)))
    ah, al = split(rng.standard_normal(n) * np.exp(rng.uniform(-3, 3, n)))
    sg = np.where(rng.random(n) < 0.5, F32(-1.0), F32(1.0))
    # the device's order: pp = xh ah, pe = its error + xh al + xl ah, then TwoSum into the row
    pp = (xh * ah).astype(F32)
    pe = fma32(xh, ah, -pp)
    pe = fma32(xh, al, pe)
    pe = fma32(xl, ah, pe)
    nh, nl = df_norm(*df_fma_add(h, l, (sg * pp).astype(F32), (sg * pe).astype(F32)))
    worst = 0.0
    for i in range(n):
        row = exact(h[i]) + exact(l[i])
        upd = exact(sg[i]) * (exact(xh[i]) + exact(xl[i])) * (exact(ah[i]) + exact(al[i]))
        got = exact(nh[i]) + exact(nl[i])
        scale = abs(row) + abs(upd)
        worst = max(worst, float(abs(got - (row + upd)) / scale))
    assert worst <= 2.0 ** -44, worst


def df_fma_add(sh, sl, bh, bl):
    """(sh, sl) += (bh, bl): TwoSum of the hi words, the low words added to the error."""
    t = (sh + bh).astype(F32)
    bp = (t - sh).astype(F32)
    te = ((sh - (t - bp)) + (bh - bp)).astype(F32)
    return t, (sl + (te + bl)).astype(F32)


def _net(rng, width, depth):
    """A plain ReLU MLP of the bench's shape: geometric initialisation plus N(0, 0.05^2)."""
    sizes = [3] + [width] * depth
    W = [rng.normal(0.0, np.sqrt(2.0 / sizes[i]), (sizes[i + 1], sizes[i])) + rng.normal(0, 0.05, (sizes[i + 1], sizes[i]))
         for i in range(depth)]
    b = [rng.normal(0.0, 0.05, sizes[i + 1]) for i in range(depth)]
    w_out = rng.normal(np.sqrt(np.pi / width), 1e-4, width) + rng.normal(0, 0.05, width)
    return W, b, w_out, -0.6


def _forward64(net, X):
    W, b, w_out, b_out = net
    h, pre, scale = X, [], []
    for Wl, bl in zip(W, b):
        a = h @ Wl.T + bl
        pre.append(a)
        scale.append(np.abs(h) @ np.abs(Wl).T + np.abs(bl))
        h = np.maximum(a, 0.0)
    return h @ w_out + b_out, pre, scale, np.abs(h) @ np.abs(w_out) + abs(b_out)


def _forward_df(net, X):
    W, b, w_out, b_out = net
    hh, hl = split(X)
    acts = []
    for Wl, bl in zip(W, b):
        Wh, Wl_ = split(Wl)
        bh, blo = split(bl)
        sh = np.broadcast_to(bh, (X.shape[0], len(bl))).astype(F32).copy()
        sl = np.broadcast_to(blo, (X.shape[0], len(bl))).astype(F32).copy()
        for j in range(Wl.shape[1]):               # the device's order: one input unit at a time
            sh, sl = df_fma(sh, sl, Wh[None, :, j], Wl_[None, :, j], hh[:, j:j + 1], hl[:, j:j + 1])
        t, lo = df_norm(sh, sl)
        act = t > 0
        acts.append(act)
        hh, hl = np.where(act, t, F32(0.0)), np.where(act, lo, F32(0.0))
    wh, wl = split(w_out)
    fh = np.zeros(X.shape[0], F32)
    fl = np.zeros(X.shape[0], F32)
    for k in range(len(w_out)):
        fh, fl = df_fma(fh, fl, wh[k], wl[k], hh[:, k], hl[:, k])
    return fh.astype(F64) + fl.astype(F64) + b_out, acts


def test_forward_pass_on_pairs_matches_fp64():
    rng = np.random.default_rng(5)
    net = _net(rng, width=256, depth=8)
    X = rng.uniform(-1.4, 1.4, (24, 3))
    F64v, pre, scale, fscale = _forward64(net, X)
    Fdf, acts = _forward_df(net, X)
    rel = np.abs(Fdf - F64v) / fscale
    assert rel.max() <= 1e-12, rel.max()
    for a, s, act in zip(pre, scale, acts):
        clear = np.abs(a) > 1e-9 * s
        assert np.array_equal((a > 0)[clear], act[clear])
