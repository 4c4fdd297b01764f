"""Per-frequency rank rule and the rank/oversampling predictor (oracle).

Test infrastructure: float64 NumPy restatement of
  * the plain adaptive rank rule used with the randomized t-SVD: at every
    Fourier frequency k, with sketch singular values s_1 >= ... >= s_l, the
    truncation rank is the smallest r (1 <= r <= cap) whose discarded energy
    sum_{i > r} s_i^2 is at most tol^2 sum_i s_i^2 (cap if none is; 0 for an
    all-zero slice).  The multi-rank of Section 2 (r_i = rank of the i-th
    Fourier frontal slice) is its tol -> 0 limit;
  * the predictor's features (log10 s_i / s_1, i = 2 .. 17, clipped at -8 and
    scaled by 1/8) and its network: a 16 -> 128 -> 128 -> 2 perceptron with
    ReLU, weights rounded to float16, mean-squared-error loss, and the Adam
    update (Kingma & Ba, 2015) on float32 master weights.
The paper has no learned component; these definitions fix what the CUDA
kernels must compute.
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID, N_OUT = 16, 128, 2
FEATURE_SV = N_IN + 1          # singular values a feature vector needs


def rank_rule(sig, tol: float, cap: int) -> np.ndarray:
    """Ranks of every row of sig (h x l, each row descending).  The tail sums
    run from the smallest value upwards in float64, one product and one sum
    per term (no fused multiply-add), so a decision made elsewhere with the
    same operations in the same order is identical."""
    sig = np.asarray(sig, dtype=np.float64)
    h, l = sig.shape
    out = np.zeros(h, dtype=np.int32)
    for k in range(h):
        tails = np.zeros(l + 1)                 # tails[r] = sum_{i > r} s_i^2 (1-based r)
        acc = 0.0
        for i in range(l - 1, -1, -1):
            acc = acc + sig[k, i] * sig[k, i]
            tails[i] = acc
        total = tails[0]
        if total == 0.0:
            out[k] = 0
            continue
        thr = (tol * tol) * total
        r = cap
        for rr in range(1, min(cap, l) + 1):
            if tails[rr] <= thr:
                r = rr
                break
        out[k] = r
    return out


def features(sig) -> np.ndarray:
    """Feature vectors (h x 16) from sketch singular values (h x >= 17)."""
    sig = np.asarray(sig, dtype=np.float64)
    s1 = sig[:, :1]
    ratio = np.where(s1 > 0, sig[:, 1:FEATURE_SV] / np.where(s1 > 0, s1, 1.0), 0.0)
    with np.errstate(divide="ignore"):
        lg = np.log10(np.maximum(ratio, 1e-8))
    return np.maximum(lg, -8.0) / 8.0


def as_f16(x) -> np.ndarray:
    """Round to float16 and return as float64 (the values the network uses)."""
    return np.asarray(x, dtype=np.float32).astype(np.float16).astype(np.float64)


def unpack(theta):
    """Packed parameter vector -> (W1 128x16, b1, W2 128x128, b2, W3 2x128, b3);
    matrices row-major (output index slowest)."""
    theta = np.asarray(theta, dtype=np.float64)
    o = 0
    out = []
    for shape in ((N_HID, N_IN), (N_HID,), (N_HID, N_HID), (N_HID,), (N_OUT, N_HID), (N_OUT,)):
        n = int(np.prod(shape))
        out.append(theta[o:o + n].reshape(shape))
        o += n
    return out


N_PARAMS = N_HID * N_IN + N_HID + N_HID * N_HID + N_HID + N_OUT * N_HID + N_OUT


def forward(theta, X):
    """Network outputs (B x 2) and the hidden activations."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    h1 = np.maximum(X @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    return h2 @ W3.T + b3, h1, h2


def loss_and_grad(theta, X, T):
    """Loss (1 / 2B) sum (y - t)^2 and its gradient with respect to the
    packed parameters, by back-propagation through the layers above."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    B = X.shape[0]
    y, h1, h2 = forward(theta, X)
    d = (y - T) / B
    loss = 0.5 * float(np.sum((y - T) ** 2)) / B
    gW3 = d.T @ h2
    gb3 = d.sum(0)
    d2 = (d @ W3) * (h2 > 0)
    gW2 = d2.T @ h1
    gb2 = d2.sum(0)
    d1 = (d2 @ W2) * (h1 > 0)
    gW1 = d1.T @ X
    gb1 = d1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g


def adam_step(theta, m, v, g, step: int, lr: float, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (theta, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
