"""Host emulation (numpy float32, IEEE round-to-nearest) of the double-float multiply-add
chains of the D products: the running sum keeps its high word by two-sum and adds every
error term into an unrenormalised low word.  Summing one row of D q in a single chain over
all N terms -- the form of the regenerating double-float GEMM -- loses accuracy far faster
than 128 interleaved lane chains joined by a butterfly (the stored-pair GEMV), or than the
single chain with its low word renormalised every 16 terms.  The rows are 1/r rows of a
2-D cluster with a dipolar charge pattern (the large flakes' far field)."""
import math

import numpy as np

F32 = np.float32


def _split(v):
    h = v.astype(F32)
    return h, (v - h.astype(np.float64)).astype(F32)


def _df_mac(ah, al, bh, bl, sh, sl):
    # float32 products and sums rounded to nearest; an FMA is its exact float64 value
    # rounded once to float32 (products of two float32 values are exact in float64)
    p = (ah * bh).astype(F32)
    e = (ah.astype(np.float64) * bh - p).astype(F32)
    e = (ah.astype(np.float64) * bl + e).astype(F32)
    e = (al.astype(np.float64) * bh + e).astype(F32)
    s = (sh + p).astype(F32)
    v = (s - sh).astype(F32)
    t = ((sh - (s - v).astype(F32)).astype(F32) + (p - v).astype(F32)).astype(F32)
    return s, (sl + (t + e).astype(F32)).astype(F32)


def _renorm(sh, sl):
    s = (sh + sl).astype(F32)
    return s, (sl - (s - sh).astype(F32)).astype(F32)


def _rows(N, rows, seed):
    rng = np.random.default_rng(seed)
    Rd = 2.7 * math.sqrt(N / math.pi)
    r = Rd * np.sqrt(rng.random(N))
    th = 2 * math.pi * rng.random(N)
    X = np.stack([r * np.cos(th), r * np.sin(th)], 1) + 1000.0
    q = (X[:, 0] - X[:, 0].mean()) / Rd * (1 + 0.3 * rng.standard_normal(N))
    q -= q.mean()
    I = rng.choice(N, rows, replace=False)
    dx = X[I, None, :] - X[None, :, :]
    D = 1.0 / np.maximum(np.sqrt((dx ** 2).sum(-1)), 2.0)
    exact = np.array([math.fsum(D[k] * q) for k in range(rows)])
    scale = (np.abs(D) * np.abs(q)).sum(1)
    return D, np.broadcast_to(q, D.shape).copy(), exact, scale


def _errors(N, rows=8, seed=3):
    D, Q, exact, scale = _rows(N, rows, seed)
    Dh, Dl = _split(D)
    Qh, Ql = _split(Q)
    sh = np.zeros(rows, F32); sl = np.zeros(rows, F32)
    rh = np.zeros(rows, F32); rl = np.zeros(rows, F32)
    for j in range(N):
        sh, sl = _df_mac(Dh[:, j], Dl[:, j], Qh[:, j], Ql[:, j], sh, sl)
        rh, rl = _df_mac(Dh[:, j], Dl[:, j], Qh[:, j], Ql[:, j], rh, rl)
        if (j & 15) == 15:
            rh, rl = _renorm(rh, rl)
    L = 128
    pad = (-N) % L
    sh_l = np.zeros((rows, L), F32); sl_l = np.zeros((rows, L), F32)
    b = [np.pad(a, ((0, 0), (0, pad))).reshape(rows, -1, L) for a in (Dh, Dl, Qh, Ql)]
    for s_ in range(b[0].shape[1]):
        sh_l, sl_l = _df_mac(b[0][:, s_], b[1][:, s_], b[2][:, s_], b[3][:, s_], sh_l, sl_l)
    while sh_l.shape[1] > 1:
        h = sh_l.shape[1] // 2
        ah, al, bh, bl = sh_l[:, :h], sl_l[:, :h], sh_l[:, h:], sl_l[:, h:]
        s = (ah + bh).astype(F32)
        v = (s - ah).astype(F32)
        t = ((ah - (s - v).astype(F32)).astype(F32) + (bh - v).astype(F32)).astype(F32)
        sh_l, sl_l = s, (al + bl + t).astype(F32)
    out = {}
    for name, y in (("chain", sh.astype(np.float64) + sl), ("renorm16", rh.astype(np.float64) + rl),
                    ("lanes128", sh_l[:, 0].astype(np.float64) + sl_l[:, 0])):
        out[name] = float(np.median(np.abs(y - exact) / scale))
    return out


def test_single_chain_accumulation_error_grows_past_the_lane_chains():
    e_small, e_large = _errors(4000), _errors(40000)
    # the 128 lane chains stay near the double-float unit (2^-48 = 3.6e-15)
    assert e_large["lanes128"] < 2e-14
    # one chain over all N is at least 30 times worse at N = 40000 and grows faster than
    # sqrt(N); renormalising its low word every 16 terms recovers most of the gap
    assert e_large["chain"] > 30 * e_large["lanes128"]
    assert e_large["chain"] / e_small["chain"] > math.sqrt(10)
    assert e_large["renorm16"] < 0.2 * e_large["chain"]
