"""Randomized slice selection and the rt-product, Section 3.1 (oracle).

Test infrastructure: float64 NumPy restatement of Algorithm 2 and of the two
probability choices of Section 3.1 (eqs. nearly_optimal_probs and
nonoptimal_probs, both taken with beta = 1, i.e. with equality).
"""
from __future__ import annotations

import math

import numpy as np

from . import philox_ref
from .tensor_ref import tprod

PROB_AB = 0     # p_j proportional to ||A_{:j:}||_F ||B_{j::}||_F   (choice i)
PROB_A2 = 1     # p_j proportional to ||A_{:j:}||_F^2                (choice ii)
PROB_GIVEN = 2  # caller-supplied p

SAMPLE_BERNOULLI = 0   # Algorithm 2: slice j kept with probability min{1, c p_j}
SAMPLE_IID = 1         # c independent draws with replacement (Drineas et al. 2006)


def lateral_norms_sq(A: np.ndarray) -> np.ndarray:
    """||A_{:j:}||_F^2 for every lateral slice j, summed in float64."""
    A = np.asarray(A, dtype=np.float64)
    return np.einsum("ijt,ijt->j", A, A)


def horizontal_norms_sq(B: np.ndarray) -> np.ndarray:
    """||B_{j::}||_F^2 for every horizontal slice j, summed in float64."""
    B = np.asarray(B, dtype=np.float64)
    return np.einsum("jlt,jlt->j", B, B)


def probabilities(a2: np.ndarray, b2: np.ndarray | None, mode: int) -> np.ndarray:
    """Sampling probabilities with beta = 1.

    mode PROB_AB: p_j = a_j b_j / sum_i a_i b_i  (eq. nearly_optimal_probs)
    mode PROB_A2: p_j = a_j^2 / ||A||_F^2        (eq. nonoptimal_probs)
    where a_j = ||A_{:j:}||_F and b_j = ||B_{j::}||_F.  The normaliser is
    summed with math.fsum (exactly rounded).  An all-zero weight vector gives
    all-zero probabilities (nothing is drawn).
    """
    if mode == PROB_AB:
        w = np.sqrt(a2) * np.sqrt(b2)
    elif mode == PROB_A2:
        w = np.asarray(a2, dtype=np.float64).copy()
    else:
        raise ValueError("mode")
    s = math.fsum(w.tolist())
    if s == 0.0:
        return np.zeros_like(w)
    return w / s


def keep_probabilities(p: np.ndarray, c: int) -> np.ndarray:
    """q_j = min{1, c p_j}: the chance that slice j is picked (Algorithm 2)."""
    return np.minimum(1.0, c * np.asarray(p, dtype=np.float64))


def draw(p: np.ndarray, c: int, seed: int, stream: int = philox_ref.STREAM_LATERAL):
    """Algorithm 2 picking loop: returns (idx ascending, q).  The rescale of a
    picked slice is 1/min{1, sqrt(c p_j)} = 1/sqrt(q_j) (Algorithm 2)."""
    q = keep_probabilities(p, c)
    idx = philox_ref.bernoulli_pick(q, seed, stream)
    return idx, q


def draw_iid(p: np.ndarray, c: int, seed: int, stream: int = philox_ref.STREAM_LATERAL):
    """c independent draws with replacement, index j with probability p_j (the
    sampling Algorithm 2 reduces to at n3 = 1 in Drineas, Kannan and Mahoney
    2006).  Integer form, so that any implementation given the same float64 p
    draws the same indices: W_j = floor(p_j 2^53), cdf_j = W_0 + ... + W_j
    (exact in integers), draw t takes the 53-bit U_t of counter
    (t, stream, 1), target_t = floor(U_t cdf_last / 2^53) and the first j with
    cdf_j > target_t.  Returns (idx in draw order, s) with s_t = c p_{j_t},
    the rescale of draw t being 1/sqrt(s_t).  No draws when sum W = 0."""
    p = np.asarray(p, dtype=np.float64)
    W = [int(w) for w in philox_ref.threshold53(np.clip(p, 0.0, 1.0))]
    cdf, acc = [], 0
    for w in W:
        acc += w
        cdf.append(acc)
    if acc == 0 or c <= 0:
        return np.zeros(0, dtype=np.int64), np.zeros(0)
    U = philox_ref.uniform53_iid(np.arange(c, dtype=np.uint64), stream, seed)
    idx = []
    for t in range(c):
        target = (int(U[t]) * acc) >> 53
        lo, hi = 0, len(cdf) - 1                 # first j with cdf_j > target
        while lo < hi:
            mid = (lo + hi) // 2
            if cdf[mid] > target:
                hi = mid
            else:
                lo = mid + 1
        idx.append(lo)
    idx = np.array(idx, dtype=np.int64)
    return idx, c * p[idx]


def sample_CR(A: np.ndarray, B: np.ndarray, idx: np.ndarray, q: np.ndarray):
    """C = A*S*D and R = D*S^T*B of Algorithm 2, without forming S or D:
    the picked lateral slices of A and horizontal slices of B, each divided by
    sqrt(q_j)."""
    s = 1.0 / np.sqrt(q[idx])
    C = np.asarray(A, dtype=np.float64)[:, idx, :] * s[None, :, None]
    R = np.asarray(B, dtype=np.float64)[idx, :, :] * s[:, None, None]
    return C, R


def tprod_sampled(A: np.ndarray, B: np.ndarray, c: int, seed: int,
                  mode: int = PROB_AB, p_given: np.ndarray | None = None,
                  sample: int = SAMPLE_BERNOULLI):
    """rt-product, Algorithm 2: Z = C * R.  Returns (Z, idx, q).

    Probabilities come from the slice norms (mode PROB_AB / PROB_A2) or from
    ``p_given`` (mode PROB_GIVEN).  With no slice picked, Z is zero.  With
    ``sample`` = SAMPLE_IID the c draws are independent with replacement
    (draw_iid); q then holds c p_j at the drawn positions (in draw order).
    """
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    if mode == PROB_GIVEN:
        p = np.asarray(p_given, dtype=np.float64)
    else:
        a2 = lateral_norms_sq(A)
        b2 = horizontal_norms_sq(B) if mode == PROB_AB else None
        p = probabilities(a2, b2, mode)
    n1, _, n3 = A.shape
    n4 = B.shape[1]
    if sample == SAMPLE_IID:
        idx, s = draw_iid(p, c, seed)
        if len(idx) == 0:
            return np.zeros((n1, n4, n3)), idx, s
        d = 1.0 / np.sqrt(s)
        C = A[:, idx, :] * d[None, :, None]
        R = B[idx, :, :] * d[:, None, None]
        return tprod(C, R), idx, s
    idx, q = draw(p, c, seed)
    if len(idx) == 0:
        return np.zeros((n1, n4, n3)), idx, q
    C, R = sample_CR(A, B, idx, q)
    return tprod(C, R), idx, q


def sampled_error_sq_expectation(A: np.ndarray, B: np.ndarray, q: np.ndarray) -> float:
    """E||A*B - C*R||_F^2 for independent Bernoulli picks with keep
    probabilities q and rescale 1/sqrt(q):  sum_j (1/q_j - 1) ||A_{:j:}*B_{j::}||_F^2
    (eq. prods splits A*B into the n2 slice products; the picks are independent)."""
    tot = 0.0
    for j in range(A.shape[1]):
        if q[j] <= 0.0:
            continue
        Pj = tprod(A[:, j:j + 1, :], B[j:j + 1, :, :])
        tot += (1.0 / q[j] - 1.0) * float(np.sum(Pj * Pj))
    return tot
