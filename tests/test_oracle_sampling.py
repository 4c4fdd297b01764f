"""Pins of the sampling oracle: Philox, probabilities, Algorithm 2 (rt-product)."""
import itertools

import numpy as np
import pytest

from oracle import philox_ref as P
from oracle import sampling_ref as S
from oracle import tensor_ref as T


def test_philox_uniformity_and_avalanche():
    n = 1 << 16
    U = P.uniform53(np.arange(n, dtype=np.uint64), 0, 12345).astype(np.float64) / 2.0 ** 53
    assert abs(U.mean() - 0.5) < 0.01
    assert abs(U.var() - 1.0 / 12) < 0.005
    counts, _ = np.histogram(U, bins=64, range=(0, 1))
    chi2 = np.sum((counts - n / 64) ** 2 / (n / 64))
    assert chi2 < 120  # 63 dof: p ~ 1e-5 cut-off
    # flipping one counter bit changes about half of the 128 output bits
    base = np.array(P.philox4x32_10(7, 0, 0, 0, 1, 2), dtype=np.uint64)
    flips = []
    for b in range(32):
        o = np.array(P.philox4x32_10(7 ^ (1 << b), 0, 0, 0, 1, 2), dtype=np.uint64)
        flips.append(sum(bin(int(x)).count("1") for x in (base ^ o)))
    assert 50 < np.mean(flips) < 78
    # different streams and seeds give unrelated numbers
    a = P.uniform53(np.arange(1000, dtype=np.uint64), 0, 1)
    b = P.uniform53(np.arange(1000, dtype=np.uint64), 1, 1)
    c = P.uniform53(np.arange(1000, dtype=np.uint64), 0, 2)
    assert np.count_nonzero(a == b) == 0 and np.count_nonzero(a == c) == 0


# Known-answer vectors of Philox4x32-10 published with the generator's
# reference implementation (Salmon et al., SC'11, the Random123 distribution):
# (counter words 0..3, key words 0..1) -> output words 0..3.
PHILOX_KAT = [
    ((0x00000000, 0x00000000, 0x00000000, 0x00000000), (0x00000000, 0x00000000),
     (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
    ((0xffffffff, 0xffffffff, 0xffffffff, 0xffffffff), (0xffffffff, 0xffffffff),
     (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
    ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0xa4093822, 0x299f31d0),
     (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1)),
]


@pytest.mark.parametrize("ctr,key,want", PHILOX_KAT)
def test_philox_known_answer_vectors(ctr, key, want):
    got = tuple(int(x) for x in P.philox4x32_10(*ctr, *key))
    assert got == want, [hex(x) for x in got]


def test_threshold_exact_edges():
    Q = P.threshold53(np.array([0.0, 1.0, 0.5, 2.0 ** -53, 1 - 2.0 ** -53]))
    assert list(Q) == [0, 2 ** 53, 2 ** 52, 1, 2 ** 53 - 1]
    # q = 1 is always picked, q = 0 never
    idx = P.bernoulli_pick(np.array([1.0, 0.0, 1.0, 0.0]), seed=3)
    assert list(idx) == [0, 2]


def test_probabilities_definitions():
    rs = np.random.default_rng(0)
    A = rs.standard_normal((3, 6, 4))
    B = rs.standard_normal((6, 2, 4))
    a2 = S.lateral_norms_sq(A)
    b2 = S.horizontal_norms_sq(B)
    for j in range(6):
        assert abs(a2[j] - np.linalg.norm(A[:, j, :]) ** 2) < 1e-12
        assert abs(b2[j] - np.linalg.norm(B[j, :, :]) ** 2) < 1e-12
    p = S.probabilities(a2, b2, S.PROB_AB)
    assert abs(p.sum() - 1) < 1e-15
    w = np.array([np.linalg.norm(A[:, j, :]) * np.linalg.norm(B[j, :, :]) for j in range(6)])
    np.testing.assert_allclose(p, w / w.sum(), rtol=1e-14)
    p2 = S.probabilities(a2, None, S.PROB_A2)
    np.testing.assert_allclose(p2, a2 / np.linalg.norm(A) ** 2, rtol=1e-14)
    assert np.all(S.probabilities(np.zeros(3), np.zeros(3), S.PROB_AB) == 0)


def test_pick_count_statistics():
    q = np.linspace(0.05, 0.95, 40)
    counts = np.array([len(P.bernoulli_pick(q, seed=s)) for s in range(2000)])
    mean, var = q.sum(), np.sum(q * (1 - q))
    assert abs(counts.mean() - mean) < 4 * np.sqrt(var / 2000)
    assert abs(counts.var() - var) < 0.15 * var


def _all_outcomes(A, B, q):
    """Exact expectation over all 2^n2 Bernoulli outcomes of C*R and of the
    squared error, by enumeration."""
    n2 = A.shape[1]
    exact = T.tprod(A, B)
    EZ = np.zeros_like(exact)
    Eerr = 0.0
    for bits in itertools.product([0, 1], repeat=n2):
        pr = 1.0
        idx = []
        for j, b in enumerate(bits):
            pr *= q[j] if b else 1 - q[j]
            if b:
                idx.append(j)
        if pr == 0.0:
            continue
        if idx:
            C, R = S.sample_CR(A, B, np.array(idx), q)
            Z = T.tprod_circ(C, R)   # definition route, independent of Algorithm 1
        else:
            Z = np.zeros_like(exact)
        EZ += pr * Z
        Eerr += pr * np.sum((exact - Z) ** 2)
    return exact, EZ, Eerr


def test_rt_product_unbiased_brute_force():
    # Algorithm 2 with rescale 1/sqrt(q) is unbiased: E[C*R] = A*B, and the
    # squared error has the closed form sum_j (1/q_j - 1)||A_{:j:} * B_{j::}||^2.
    rs = np.random.default_rng(1)
    A = rs.standard_normal((3, 8, 3))
    B = rs.standard_normal((8, 2, 3))
    p = S.probabilities(S.lateral_norms_sq(A), S.horizontal_norms_sq(B), S.PROB_AB)
    q = S.keep_probabilities(p, 3)
    exact, EZ, Eerr = _all_outcomes(A, B, q)
    np.testing.assert_allclose(EZ, exact, atol=1e-11)
    assert abs(Eerr - S.sampled_error_sq_expectation(A, B, q)) < 1e-9 * max(1, Eerr)


def test_rt_product_deterministic_when_all_kept():
    # c p_j >= 1 for all j => q = 1 => exact product (Algorithm 2)
    rs = np.random.default_rng(2)
    A = rs.standard_normal((4, 5, 6))
    B = rs.standard_normal((5, 3, 6))
    Z, idx, q = S.tprod_sampled(A, B, c=10 ** 6, seed=0)
    assert list(idx) == list(range(5)) and np.all(q == 1)
    np.testing.assert_allclose(Z, T.tprod_circ(A, B), atol=1e-12)


def test_rt_product_matrix_case():
    # n3 = 1: column/row sampling of Drineas, Kannan and Mahoney (2006)
    rs = np.random.default_rng(3)
    A = rs.standard_normal((6, 10, 1))
    B = rs.standard_normal((10, 4, 1))
    Z, idx, q = S.tprod_sampled(A, B, c=4, seed=9)
    Am, Bm = A[:, :, 0], B[:, :, 0]
    expect = sum(np.outer(Am[:, j], Bm[j, :]) / q[j] for j in idx)
    np.testing.assert_allclose(Z[:, :, 0], expect, atol=1e-12)


def test_rt_product_zero_input():
    A = np.zeros((3, 4, 2))
    B = np.ones((4, 2, 2))
    Z, idx, q = S.tprod_sampled(A, B, c=2, seed=0)
    assert len(idx) == 0 and np.all(Z == 0)


def test_monte_carlo_error_matches_expectation():
    rs = np.random.default_rng(4)
    A = rs.standard_normal((5, 30, 4))
    B = rs.standard_normal((30, 3, 4))
    exact = T.tprod(A, B)
    errs = []
    q = None
    for s in range(300):
        Z, idx, q = S.tprod_sampled(A, B, c=8, seed=s)
        errs.append(np.sum((Z - exact) ** 2))
    expect = S.sampled_error_sq_expectation(A, B, q)
    assert abs(np.mean(errs) / expect - 1) < 0.2


def test_iid_draw_brute_force_expectation_is_the_exact_product():
    # all n^c ordered draw sequences with their probabilities prod p_{j_t}
    import itertools
    from oracle import sampling_ref as S, tensor_ref as T
    g = np.random.default_rng(90)
    A = g.standard_normal((3, 4, 3))
    B = g.standard_normal((4, 2, 3))
    p = np.array([0.1, 0.4, 0.2, 0.3])
    c = 3
    exact = T.tprod(A, B)
    mean = np.zeros_like(exact)
    var = 0.0
    for seq in itertools.product(range(4), repeat=c):
        w = np.prod(p[list(seq)])
        d = 1.0 / np.sqrt(c * p[list(seq)])
        Z = T.tprod(A[:, seq, :] * d[None, :, None], B[seq, :, :] * d[:, None, None])
        mean += w * Z
        var += w * np.sum((Z - exact) ** 2)
    np.testing.assert_allclose(mean, exact, atol=1e-12)
    # Drineas et al.: E||AB - CR||^2 = (sum_j ||A_j B_j||^2 / p_j - ||AB||^2) / c
    terms = sum(np.sum(T.tprod(A[:, j:j + 1, :], B[j:j + 1, :, :]) ** 2) / p[j] for j in range(4))
    assert abs(var - (terms - np.sum(exact ** 2)) / c) < 1e-10


def test_iid_draw_frequencies_and_degenerate_weights():
    from oracle import sampling_ref as S
    p = np.array([0.5, 0.0, 0.25, 0.125, 0.125])
    idx, s = S.draw_iid(p, 20000, 7)
    assert len(idx) == 20000 and not np.any(idx == 1)            # zero weight never drawn
    counts = np.bincount(idx, minlength=5)
    exp = 20000 * p
    chi2 = sum((counts[j] - exp[j]) ** 2 / exp[j] for j in (0, 2, 3, 4))
    assert chi2 < 20.0                                            # 3 dof, p ~ 2e-4
    np.testing.assert_allclose(s, 20000 * p[idx])
    one = np.zeros(6)
    one[4] = 1.0
    assert np.array_equal(S.draw_iid(one, 9, 3)[0], np.full(9, 4))
    assert len(S.draw_iid(np.zeros(6), 9, 3)[0]) == 0
    # the integer search by hand: cdf = (2^52, 2^52 + 2^51, ...), target below
    # 2^52 takes index 0
    a, _ = S.draw_iid(np.array([0.5, 0.25, 0.25]), 64, 11)
    from oracle import philox_ref as P
    U = P.uniform53_iid(np.arange(64, dtype=np.uint64), 0, 11)
    want = np.where(U < 2 ** 52, 0, np.where(U < 2 ** 52 + 2 ** 51, 1, 2))
    assert np.array_equal(a, want)


def test_iid_sampled_product_with_n3_one_is_drineas_kannan_mahoney():
    from oracle import sampling_ref as S
    g = np.random.default_rng(91)
    A = g.standard_normal((5, 8, 1))
    B = g.standard_normal((8, 4, 1))
    Z, idx, s = S.tprod_sampled(A, B, 6, 13, sample=S.SAMPLE_IID)
    p = S.probabilities(S.lateral_norms_sq(A), S.horizontal_norms_sq(B), S.PROB_AB)
    want = sum(np.outer(A[:, j, 0], B[j, :, 0]) / (6 * p[j]) for j in idx)
    np.testing.assert_allclose(Z[:, :, 0], want, atol=1e-12)
