"""Philox4x32-10 and the integer Bernoulli decision (oracle; test infrastructure).

Philox4x32-10 is the counter-based generator of Salmon, Moraes, Dror and Shaw,
"Parallel Random Numbers: As Easy as 1, 2, 3" (SC'11): a 128-bit counter and a
64-bit key pass through ten rounds.  Each round multiplies words 0 and 2 by
fixed 32-bit constants, keeps both halves of the 64-bit products, XORs the
high halves with the other two words and the round key, and permutes; the key
is bumped by two Weyl constants between rounds.  This module writes that
definition out in NumPy uint64 arithmetic, vectorised over counters.

The paper draws slices with probability min{1, c p_i} (Algorithm 2, picking
loop) but does not say how the coin is tossed.  The reading used on both sides
of the parity test: for slice j the counter is (j mod 2^32, j >> 32, stream, 0)
and the key is (seed mod 2^32, seed >> 32); the 53-bit integer
U_j = (x0 >> 5) * 2^26 + (x1 >> 6) is compared with Q_j = floor(q_j * 2^53)
and j is picked iff U_j < Q_j.  q_j = 1 gives Q_j = 2^53, always picked; q_j = 0
is never picked.  Given the same float64 q_j, the decision is exact integer
arithmetic on both sides.
"""
from __future__ import annotations

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)

# Stream identifiers of the counter's third word.
STREAM_LATERAL = 0      # lateral-slice draws (Algorithm 2, Algorithm 4)
STREAM_HORIZONTAL = 1   # horizontal-slice draws (Algorithm 5)
STREAM_SKETCH = 2       # entries of the randomized t-SVD test matrix


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox rounds on uint32 words (given as integer arrays); returns x0..x3."""
    c0 = np.asarray(c0, dtype=np.uint64) & _MASK
    c1 = np.asarray(c1, dtype=np.uint64) & _MASK
    c2 = np.asarray(c2, dtype=np.uint64) & _MASK
    c3 = np.asarray(c3, dtype=np.uint64) & _MASK
    k0 = np.asarray(k0, dtype=np.uint64) & _MASK
    k1 = np.asarray(k1, dtype=np.uint64) & _MASK
    c0, c1, c2, c3, k0, k1 = np.broadcast_arrays(c0, c1, c2, c3, k0, k1)
    c0, c1, c2, c3 = c0.copy(), c1.copy(), c2.copy(), c3.copy()
    k0, k1 = k0.copy(), k1.copy()
    for r in range(10):
        if r > 0:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * c0          # < 2^64, exact in uint64
        p1 = _M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
    return c0, c1, c2, c3


def uniform53(index, stream: int, seed: int) -> np.ndarray:
    """53-bit integers U_j for counters j = index (uint64 array)."""
    j = np.asarray(index, dtype=np.uint64)
    seed = int(seed) & ((1 << 64) - 1)
    x0, x1, _, _ = philox4x32_10(j & _MASK, j >> np.uint64(32), stream, 0,
                                 seed & 0xFFFFFFFF, seed >> 32)
    return ((x0 >> np.uint64(5)) << np.uint64(26)) | (x1 >> np.uint64(6))


def uniform53_iid(t, stream: int, seed: int) -> np.ndarray:
    """53-bit integers of the i.i.d. draws t: counter (t mod 2^32, t >> 32,
    stream, 1) (the fourth word 1 keeps them apart from the Bernoulli coins)."""
    t = np.asarray(t, dtype=np.uint64)
    seed = int(seed) & ((1 << 64) - 1)
    x0, x1, _, _ = philox4x32_10(t & _MASK, t >> np.uint64(32), stream, 1,
                                 seed & 0xFFFFFFFF, seed >> 32)
    return ((x0 >> np.uint64(5)) << np.uint64(26)) | (x1 >> np.uint64(6))


def threshold53(q: np.ndarray) -> np.ndarray:
    """Q_j = floor(q_j * 2^53) for 0 <= q_j <= 1 (exact: scaling by 2^53 is exact)."""
    q = np.asarray(q, dtype=np.float64)
    return np.floor(q * 9007199254740992.0).astype(np.uint64)


def bernoulli_pick(q: np.ndarray, seed: int, stream: int = STREAM_LATERAL) -> np.ndarray:
    """Indices j (ascending) picked with probability q_j, Algorithm 2 picking loop."""
    n = len(q)
    U = uniform53(np.arange(n, dtype=np.uint64), stream, seed)
    Q = threshold53(q)
    picked = []
    for j in range(n):                 # the paper's loop over i = 1..n2, in order
        if U[j] < Q[j]:
            picked.append(j)
    return np.asarray(picked, dtype=np.int64)


def sketch_signs(n_rows: int, n_cols: int, h: int, n3: int, seed: int) -> np.ndarray:
    """Test matrix Omega_hat (n_rows x n_cols x h) for the randomized t-SVD.

    Entry (r, c, k) uses the counter e = r + n_rows*(c + n_cols*k) on the
    sketch stream.  Complex slices get (s0 + 1j s1)/sqrt(2) with s0, s1 = +-1
    from the top bits of x0, x1; the real slices (k = 0, and k = n3/2 for even
    n3) get the real sign s0.  Bit-identical on any IEEE machine.
    """
    e = np.arange(n_rows * n_cols * h, dtype=np.uint64)
    seed = int(seed) & ((1 << 64) - 1)
    x0, x1, _, _ = philox4x32_10(e & _MASK, e >> np.uint64(32), STREAM_SKETCH, 0,
                                 seed & 0xFFFFFFFF, seed >> 32)
    s0 = 1.0 - 2.0 * (x0 >> np.uint64(31)).astype(np.float64)
    s1 = 1.0 - 2.0 * (x1 >> np.uint64(31)).astype(np.float64)
    s0 = s0.reshape(h, n_cols, n_rows).transpose(2, 1, 0)
    s1 = s1.reshape(h, n_cols, n_rows).transpose(2, 1, 0)
    inv = 1.0 / np.sqrt(2.0)
    Om = (s0 + 1j * s1) * inv
    Om[:, :, 0] = s0[:, :, 0]
    if n3 % 2 == 0 and h - 1 == n3 // 2:
        Om[:, :, h - 1] = s0[:, :, h - 1]
    return Om
