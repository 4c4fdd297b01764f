"""Learned choice of the randomized t-SVD's sketch size (the rank/oversampling
predictor), driven through the library's C entry points.

The plain adaptive method sketches every frequency with l = k + p = 50
columns (q = 2 power iterations) and truncates frequency k at the plain rank
rule's r_k (tol 1e-2, cap k = 40).  Many tensors need far fewer columns: the
predictor looks at a cheap sketch (17 columns, no power iteration), predicts
each frequency's rank r_k and the oversampling p_k a sketch needs to resolve
it, and the decomposition runs with l* = max_k (r_k + p_k) columns.  The
plain rule stays the arbiter: it re-derives the ranks from the l*-column
sketch, and if any frequency reaches its cap (l* - 2) the sketch was too
small and the method falls back to l = 50.

Training data: tensors the plain method decomposes.  For each frequency the
targets are the plain rule's rank r* on the 50-column sketch and the smallest
oversampling p* (over a grid of sketch sizes) at which the rule on a smaller
sketch gives the same rank.  Features, network, gradients and Adam steps are
the library's kernels (tp_rank_features, tp_mlp_forward, tp_mlp_train_step).
"""
from __future__ import annotations

import time

import numpy as np

from . import binding as tp
from . import synth

L_PLAIN, K_PLAIN, Q_PLAIN, TOL = 50, 40, 2, 1e-2
L_CHEAP, Q_CHEAP = 17, 0
L_GRID = (12, 16, 20, 24, 28, 32, 36, 40, 44, 50)
R_SCALE, P_SCALE = 40.0, 20.0          # output scaling of the network


def init_params(seed: int):
    """He-uniform initial weights (bound sqrt(6 / fan_in)), zero biases."""
    import torch
    g = np.random.default_rng(seed)
    parts = []
    for (fo, fi) in ((128, 16), (128, 128), (2, 128)):
        bound = np.sqrt(6.0 / fi)
        parts.append(g.uniform(-bound, bound, size=fo * fi))
        parts.append(np.zeros(fo))
    return torch.from_numpy(np.concatenate(parts).astype(np.float32)).cuda()


def cheap_features(X, seed=0):
    """Float16 features (h x 16) of every frequency of X from the cheap sketch."""
    return tp.rank_features(tp.sketch_spectrum(X, L_CHEAP, Q_CHEAP, seed=seed))


def targets(X, seed=0):
    """Per-frequency (r*, p*): the plain rule's rank on the 50-column sketch
    and the smallest oversampling over L_GRID that reproduces it."""
    import torch
    r_star = tp.rank_rule(tp.sketch_spectrum(X, L_PLAIN, Q_PLAIN, seed=seed), K_PLAIN, TOL)
    h = r_star.shape[0]
    need = torch.full((h,), L_PLAIN, dtype=torch.int32, device=r_star.device)
    for l in reversed(L_GRID[:-1]):       # largest first: the last match is the smallest l
        r_l = tp.rank_rule(tp.sketch_spectrum(X, l, Q_PLAIN, seed=seed), l - 2, TOL)
        ok = (r_l == r_star) & (r_star <= l - 2)
        need = torch.where(ok, torch.full_like(need, l), need)
    return r_star, need - r_star


TRAIN_SIZES = ((128, 128, 16), (128, 96, 32), (160, 128, 16), (96, 96, 64), (80, 64, 128),
               (64, 64, 256))


def training_set(count, seed0, sizes=TRAIN_SIZES):
    """Features (N x 16 float16) and scaled targets (N x 2 float32) from
    `count` tensors of the spectral family with decay exponents drawn in
    [1.5, 4] (per tensor) and jittered +-0.3 per frequency; the sizes cycle
    through tube lengths n3 = 16 .. 256 (the network sees one frequency at a
    time, so n3 sets how many samples a tensor gives)."""
    import torch
    g = np.random.default_rng(seed0)
    feats, tgts = [], []
    for c in range(count):
        n1, n2, n3 = sizes[c % len(sizes)]
        X, _ = synth.spectral_torch(n1, n2, n3, float(g.uniform(1.5, 4.0)), 0.3, seed0 + c)
        f = cheap_features(X, seed=c)
        r, p = targets(X, seed=c)
        feats.append(f)
        tgts.append(torch.stack([r.float() / R_SCALE, p.float() / P_SCALE], dim=1))
    return torch.cat(feats), torch.cat(tgts).contiguous()


def train(x16, t, steps=3000, lr=1e-3, batch=4096, seed=0, log_every=0):
    """Adam on the library's kernels; returns (theta, w16, losses)."""
    import torch
    theta = init_params(seed)
    w16 = tp.mlp_round(theta)
    m = torch.zeros_like(theta)
    v = torch.zeros_like(theta)
    n = x16.shape[0]
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    losses = []
    grad = None
    for step in range(1, steps + 1):
        if n > batch:
            sel = torch.randint(0, n, (batch,), generator=g, device="cuda")
            xb, tb = x16[sel].contiguous(), t[sel].contiguous()
        else:
            xb, tb = x16, t
        grad = tp.mlp_train_step(theta, w16, m, v, step, lr, xb, tb, grad)
        if step == 1 or step == steps or (log_every and step % log_every == 0):
            losses.append((step, float(grad[-1].item())))
    return theta, w16, losses


def predict(w16, x16):
    """Per-frequency predicted (rank, oversampling), integers."""
    import torch
    y = tp.mlp_forward(w16, x16)
    r = torch.clamp(torch.round(y[:, 0] * R_SCALE), 1, K_PLAIN).int()
    p = torch.clamp(torch.ceil(y[:, 1] * P_SCALE), 2, 20).int()
    return r, p


def sketch_size(w16, X, seed=0, margin=2):
    """l* for X: the largest predicted r + p over the frequencies (plus a
    margin), within [8, L_PLAIN]."""
    r, p = predict(w16, cheap_features(X, seed))
    l = int((r + p).max().item()) + margin
    return max(8, min(L_PLAIN, l + (l & 1)))


def decompose(X, w16=None, seed=0):
    """Per-frequency ranks of X by the plain method (w16 None) or by the
    predictor with the rule as judge.  Returns (ranks, sketch size used,
    fell_back)."""
    if w16 is None:
        return tp.rank_rule(tp.sketch_spectrum(X, L_PLAIN, Q_PLAIN, seed), K_PLAIN, TOL), L_PLAIN, False
    l = sketch_size(w16, X, seed)
    if l < L_PLAIN:
        r = tp.rank_rule(tp.sketch_spectrum(X, l, Q_PLAIN, seed), l - 2, TOL)
        if int(r.max().item()) < l - 2:
            return r, l, False
    r = tp.rank_rule(tp.sketch_spectrum(X, L_PLAIN, Q_PLAIN, seed), K_PLAIN, TOL)
    return r, L_PLAIN, True


def sketch_sizes(w16, X, ranks, l, seed=0):
    """Per-frequency sketch sizes l_f = r_f + p_f: the judged rank plus the
    network's predicted oversampling for that frequency, at most l."""
    import torch
    _, p = predict(w16, cheap_features(X, seed))
    return torch.clamp(ranks.int() + p, 1, l).int().contiguous()


def factorize(X, w16=None, seed=0, per_frequency=True):
    """The multi-rank factorisation X ~ U * S * V^T: per-frequency ranks from
    decompose(), then the randomized t-SVD (k the largest rank, q = 2)
    truncating every frequency to its own rank.  With the predictor and
    per_frequency, frequency f sketches with its own l_f = r_f + p_f columns
    (sketch_sizes) inside the one call; otherwise every frequency uses the
    call's sketch size l.  Returns (U, S, V, ranks, sketch size l)."""
    r, l, _ = decompose(X, w16, seed)
    k = max(1, int(r.max().item()))
    sizes = sketch_sizes(w16, X, r, l, seed) if (w16 is not None and per_frequency) else None
    U, S, V = tp.tsvd_randomized(X, k, l - k, Q_PLAIN, seed=seed, ranks=r.int().contiguous(),
                                 sketch_sizes=sizes)
    return U, S, V, r, l


def truncation_error(s, ranks, n3):
    """Relative error of the per-frequency best rank-r_k approximation, from
    the exact spectra s (h x m): frequencies other than 0 and n3/2 count
    twice (their conjugates)."""
    import torch
    h, m = s.shape
    w = torch.full((h,), 2.0, dtype=torch.float64, device=s.device)
    w[0] = 1.0
    if n3 % 2 == 0:
        w[h - 1] = 1.0
    idx = torch.arange(m, device=s.device)[None, :]
    tail = torch.where(idx >= ranks.long()[:, None], s * s, torch.zeros_like(s)).sum(1)
    return float(torch.sqrt((w * tail).sum() / (w * (s * s).sum(1)).sum()).item())


def time_call(fn, reps=3):
    import torch
    fn()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        fn()
    torch.cuda.synchronize()
    return (time.perf_counter() - t0) / reps * 1e3
