"""Pins of the t-product oracle (Section 2, Def. 2.1, Algorithm 1, Eq. circ1).

Every check compares the oracle with something other than itself: a value
worked by hand, a library routine in a special case, or an identity the
mathematics fixes.
"""
import numpy as np
import pytest

from oracle import tensor_ref as T


def rng(seed=0):
    return np.random.default_rng(seed)


def test_dft_matches_numpy_fft():
    # Section 2 "Operators": fft(X, [], 3) is numpy's fft along the last axis.
    X = rng().standard_normal((3, 4, 7))
    np.testing.assert_allclose(T.fft3(X), np.fft.fft(X, axis=2), atol=1e-12)
    np.testing.assert_allclose(T.ifft3(T.fft3(X)).real, X, atol=1e-12)
    for n3 in (1, 2, 5, 16, 17, 64, 120):
        Y = rng(n3).standard_normal((2, 3, n3))
        np.testing.assert_allclose(T.fft3(Y), np.fft.fft(Y, axis=2), atol=1e-10 * n3)


def test_contraction_and_library_routes_agree():
    # the explicit F_{n3} contraction (used up to 256) and numpy.fft (above)
    X = rng(11).standard_normal((2, 3, 300))
    F = T.dft_matrix(300)
    np.testing.assert_allclose(T.fft3(X), X.astype(complex) @ F.T, atol=1e-9)
    Y = rng(12).standard_normal((2, 2, 2000))
    np.testing.assert_allclose(T.ifft3(T.fft3(Y)).real, Y, atol=1e-12)


def test_tube_circular_convolution_by_hand():
    # Def. 2.1 with n1 = n2 = n4 = 1: circ of the tube (1,2,3) is
    # [[1,3,2],[2,1,3],[3,2,1]]; times (4,5,6): (4+15+12, 8+5+18, 12+10+6).
    a = np.array([1.0, 2.0, 3.0]).reshape(1, 1, 3)
    b = np.array([4.0, 5.0, 6.0]).reshape(1, 1, 3)
    expect = np.array([31.0, 31.0, 28.0])
    np.testing.assert_array_equal(T.tprod_circ(a, b).ravel(), expect)
    np.testing.assert_allclose(T.tprod(a, b).ravel(), expect, atol=1e-12)


def test_circ_layout_by_hand():
    # First block column of circ(Z) is slices 1..n3 in order; first block row
    # is slice 1 followed by slices n3, n3-1, ..., 2 (Def. 2.1).
    Z = np.arange(1, 4, dtype=float).reshape(1, 1, 3)
    np.testing.assert_array_equal(T.circ(Z), [[1, 3, 2], [2, 1, 3], [3, 2, 1]])


def test_n3_one_is_matrix_product():
    A = rng(1).standard_normal((5, 4, 1))
    B = rng(2).standard_normal((4, 3, 1))
    np.testing.assert_allclose(T.tprod(A, B)[:, :, 0], A[:, :, 0] @ B[:, :, 0], atol=1e-12)
    np.testing.assert_allclose(T.tprod_circ(A, B)[:, :, 0], A[:, :, 0] @ B[:, :, 0], atol=1e-12)


@pytest.mark.parametrize("n3", [1, 2, 3, 4, 5, 8])
def test_fourier_route_equals_definition(n3):
    # Algorithm 1 reaches the block-circulant definition exactly (Eq. circ1).
    A = rng(n3).standard_normal((4, 3, n3))
    B = rng(n3 + 10).standard_normal((3, 5, n3))
    C, imag = T.tprod(A, B, return_imag=True)
    np.testing.assert_allclose(C, T.tprod_circ(A, B), atol=1e-12)
    assert imag < 1e-12


def test_identity_tensor():
    A = rng(3).standard_normal((4, 3, 5))
    np.testing.assert_allclose(T.tprod_circ(T.identity(4, 5), A), A, atol=1e-14)
    np.testing.assert_allclose(T.tprod(A, T.identity(3, 5)), A, atol=1e-12)


def test_associativity_and_transpose_rule():
    A = rng(4).standard_normal((3, 4, 6))
    B = rng(5).standard_normal((4, 2, 6))
    C = rng(6).standard_normal((2, 5, 6))
    np.testing.assert_allclose(T.tprod(T.tprod(A, B), C), T.tprod(A, T.tprod(B, C)), atol=1e-11)
    # (A*B)^T = B^T * A^T with the conjugate transpose of Section 2.1
    np.testing.assert_allclose(T.ttranspose(T.tprod_circ(A, B)),
                               T.tprod_circ(T.ttranspose(B), T.ttranspose(A)), atol=1e-12)


def test_transpose_by_hand():
    X = np.arange(8, dtype=float).reshape(2, 2, 2, order="F")  # X[:,:,0]=[[0,2],[1,3]]
    Xt = T.ttranspose(X)
    np.testing.assert_array_equal(Xt[:, :, 0], X[:, :, 0].T)
    np.testing.assert_array_equal(Xt[:, :, 1], X[:, :, 1].T)  # n3=2: slice 2 maps to itself
    Y = rng(7).standard_normal((2, 3, 4))
    Yt = T.ttranspose(Y)
    np.testing.assert_array_equal(Yt[:, :, 1], Y[:, :, 3].T)
    np.testing.assert_array_equal(Yt[:, :, 3], Y[:, :, 1].T)


def test_block_diagonalisation_eq_circ1():
    # (F kron I_n1) circ(X) (F^-1 kron I_n2) = bdiag(X_hat)
    n1, n2, n3 = 3, 2, 5
    X = rng(8).standard_normal((n1, n2, n3))
    F = T.dft_matrix(n3)
    L = np.kron(F, np.eye(n1))
    R = np.kron(np.linalg.inv(F), np.eye(n2))
    D = L @ T.circ(X) @ R
    Xh = T.fft3(X)
    expect = np.zeros_like(D)
    for k in range(n3):
        expect[k * n1:(k + 1) * n1, k * n2:(k + 1) * n2] = Xh[:, :, k]
    np.testing.assert_allclose(D, expect, atol=1e-12)


def test_parseval_and_norms():
    X = rng(9).standard_normal((4, 5, 7))
    Xh = T.fft3(X)
    assert abs(T.fro(X) ** 2 - np.sum(np.abs(Xh) ** 2) / 7) < 1e-10
    # ||X||_TNN = ||circ(X)||_* / n3 (Section 2.1 display after Eq. tnuc)
    nuc = np.linalg.svd(T.circ(X), compute_uv=False).sum() / 7
    assert abs(T.tnn(X) - nuc) < 1e-10
    # spectral norm = ||circ(X)||_2 (Def. 2.7 with Eq. circ1)
    assert abs(T.tspectral(X) - np.linalg.norm(T.circ(X), 2)) < 1e-10


def test_conjugate_symmetry_of_half_spectrum():
    for n3 in (1, 2, 7, 8):
        X = rng(n3).standard_normal((2, 3, n3))
        Xh = T.fft3(X)
        np.testing.assert_allclose(T.hermitian_fill(T.half_spectrum(Xh), n3), Xh, atol=1e-12)


def test_hand_worked_fixtures():
    # tests/golden: values worked by hand from Def. 2.1, the t-transpose of
    # Section 2 and Theorem 2.6 (derivations in the files)
    from oracle import decomp_ref, tensor_ref
    from tests.util import golden, golden_tensor
    g = golden("tprod_2x2x2_by_hand.txt")
    A, B, C, AT = (golden_tensor(g[k], 2, 2, 2) for k in ("A", "B", "C", "AT"))
    np.testing.assert_allclose(tensor_ref.tprod(A, B), C, atol=1e-12)
    np.testing.assert_allclose(tensor_ref.ttranspose(A), AT, atol=0)
    t = golden("tube_1x1x3_by_hand.txt")
    a = np.array([1.0, 2.0, 3.0]).reshape(1, 1, 3)
    b = np.array([4.0, 5.0, 6.0]).reshape(1, 1, 3)
    np.testing.assert_allclose(tensor_ref.tprod(a, b).ravel(), t["prod"][0], atol=1e-12)
    U, S, V = decomp_ref.tsvd(a)
    np.testing.assert_allclose(S.ravel(), t["svd_s"][0], atol=1e-12)
    assert abs(tensor_ref.tnn(a) - t["tnn"][0][0]) < 1e-12
