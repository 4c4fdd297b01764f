"""Pins of the decomposition oracles: t-SVD (Theorem 2.6), the randomized
t-SVD, t-project / t-CX (Algorithms 3-4) and the completion ADMM (Algorithm 7)."""
import numpy as np
import pytest

from oracle import completion_ref as Cm
from oracle import decomp_ref as D
from oracle import philox_ref as P
from oracle import tensor_ref as T


def rs(seed):
    return np.random.default_rng(seed)


@pytest.mark.parametrize("shape", [(5, 3, 4), (3, 5, 5), (4, 4, 1), (6, 2, 2)])
def test_tsvd_reconstruction_and_orthogonality(shape):
    X = rs(sum(shape)).standard_normal(shape)
    U, S, V = D.tsvd(X)
    n1, n2, n3 = shape
    m = min(n1, n2)
    assert U.shape == (n1, m, n3) and S.shape == (m, m, n3) and V.shape == (n2, m, n3)
    # X = U * S * V^T through the block-circulant definition (not Algorithm 1)
    np.testing.assert_allclose(T.tprod_circ(T.tprod_circ(U, S), T.ttranspose(V)), X, atol=1e-12)
    # U^T * U = I and V^T * V = I (Def. 2.4, economy form)
    np.testing.assert_allclose(T.tprod_circ(T.ttranspose(U), U), T.identity(m, n3), atol=1e-12)
    np.testing.assert_allclose(T.tprod_circ(T.ttranspose(V), V), T.identity(m, n3), atol=1e-12)
    # S is f-diagonal (Def. 2.5)
    for t in range(n3):
        assert np.allclose(S[:, :, t] - np.diag(np.diag(S[:, :, t])), 0, atol=1e-13)


def test_tsvd_spectrum_is_spectrum_of_circ():
    # Eq. circ1: the singular values of circ(X) are the union over all n3
    # Fourier slices of their singular values.
    X = rs(11).standard_normal((6, 4, 5))
    _, s, _ = D.tsvd_hat(X)
    full = np.concatenate([s[:, 0], s[:, 1], s[:, 2], s[:, 2], s[:, 1]])
    ref = np.linalg.svd(T.circ(X), compute_uv=False)
    np.testing.assert_allclose(np.sort(full), np.sort(ref[: full.size]), atol=1e-12)
    assert np.all(ref[full.size:] < 1e-10)


def test_tsvd_matrix_case():
    X = rs(12).standard_normal((7, 5, 1))
    U, S, V = D.tsvd(X)
    np.testing.assert_allclose(np.diag(S[:, :, 0]), np.linalg.svd(X[:, :, 0], compute_uv=False), atol=1e-13)


def test_eckart_young_truncation():
    X = rs(13).standard_normal((6, 5, 4))
    Uh, s, Vh = D.tsvd_hat(X)
    U, S, V = D.tsvd(X)
    r = 2
    Xr = T.tprod(T.tprod(U[:, :r, :], S[:r, :r, :]), T.ttranspose(V[:, :r, :]))
    err = np.sum((X - Xr) ** 2)
    assert abs(err - D.truncate_error_sq(s, 4, r)) < 1e-10
    # no random tubal-rank-r tensor P*Q does better
    for seed in range(20):
        Pm = rs(100 + seed).standard_normal((6, r, 4))
        Qm = rs(200 + seed).standard_normal((r, 5, 4))
        assert np.sum((X - T.tprod(Pm, Qm)) ** 2) >= err - 1e-9


def _lowrank(n1, n2, n3, r, seed):
    return T.tprod(rs(seed).standard_normal((n1, r, n3)), rs(seed + 1).standard_normal((r, n2, n3)))


def test_randomized_tsvd_exact_on_low_rank():
    X = _lowrank(20, 16, 6, 3, 20)
    k, p = 3, 4
    Om = P.sketch_signs(16, k + p, 4, 6, seed=5)
    U, S, V = D.tsvd_randomized(X, k, p, 1, Om)
    Xr = T.tprod(T.tprod(U, S), T.ttranspose(V))
    np.testing.assert_allclose(Xr, X, atol=1e-10)
    _, s_exact, _ = D.tsvd_hat(X)
    _, s_rand, _ = D.tsvd_randomized_hat(X, k, p, 1, Om)
    np.testing.assert_allclose(s_rand, s_exact[:k], rtol=1e-10)


def test_randomized_tsvd_full_sketch_is_exact_topk():
    # ell >= n2: the sketch spans the whole row space, so the result is the
    # exact top-k truncation whatever the test matrix.
    X = rs(21).standard_normal((12, 6, 5))
    k, p = 3, 3
    Om = P.sketch_signs(6, k + p, 3, 5, seed=1)
    _, s_rand, _ = D.tsvd_randomized_hat(X, k, p, 0, Om)
    _, s_exact, _ = D.tsvd_hat(X)
    np.testing.assert_allclose(s_rand, s_exact[:k], rtol=1e-10)


def test_randomized_tsvd_near_optimal_with_power_iterations():
    X = _lowrank(40, 30, 4, 5, 30) + 1e-3 * rs(31).standard_normal((40, 30, 4))
    k, p = 5, 5
    Om = P.sketch_signs(30, k + p, 3, 4, seed=2)
    U, S, V = D.tsvd_randomized(X, k, p, 2, Om)
    err = np.sum((X - T.tprod(T.tprod(U, S), T.ttranspose(V))) ** 2)
    _, s, _ = D.tsvd_hat(X)
    opt = D.truncate_error_sq(s, 4, k)
    assert err <= 1.01 * opt


def test_sketch_signs_values():
    Om = P.sketch_signs(5, 3, 3, 4, seed=0)
    assert np.all(np.abs(Om) > 0)
    np.testing.assert_allclose(np.abs(Om), 1.0, atol=1e-15)
    assert np.all(Om[:, :, 0].imag == 0) and np.all(Om[:, :, 2].imag == 0)  # DC, Nyquist


def test_tproject_least_squares_optimality():
    # Eq. ell2reg: Pi_C(X) is the best approximation of X by C * Y
    X = rs(40).standard_normal((6, 8, 3))
    C = X[:, [1, 4, 6], :]
    Z = D.tproject(X, C)
    best = np.sum((X - Z) ** 2)
    for s in range(20):
        Y = rs(300 + s).standard_normal((3, 8, 3))
        assert np.sum((X - T.tprod(C, Y)) ** 2) >= best - 1e-10
    np.testing.assert_allclose(D.tproject(Z, C), Z, atol=1e-10)  # idempotent
    np.testing.assert_allclose(D.tproject(C, C), C, atol=1e-10)


def test_tcx_all_slices_kept_is_exact():
    X = rs(41).standard_normal((7, 5, 4))
    Z, idx, q = D.tcx(X, c=10 ** 6, seed=0)
    assert len(idx) == 5
    np.testing.assert_allclose(Z, X, atol=1e-10)


def test_tcx_low_rank_recovered():
    X = _lowrank(10, 30, 4, 2, 42)
    Z, idx, q = D.tcx(X, c=12, seed=3)
    assert len(idx) >= 2
    np.testing.assert_allclose(Z, X, atol=1e-8 * np.abs(X).max())


def test_pinv_matches_numpy():
    M = rs(43).standard_normal((5, 3)) + 1j * rs(44).standard_normal((5, 3))
    np.testing.assert_allclose(D.pinv_matlab(M), np.linalg.pinv(M), atol=1e-12)


def test_svt_matrix_is_prox_of_nuclear_norm():
    M = rs(50).standard_normal((6, 4))
    tau = 0.7
    L = Cm.svt_matrix(M, tau)
    f = lambda Z: tau * np.linalg.svd(Z, compute_uv=False).sum() + 0.5 * np.sum((Z - M) ** 2)
    best = f(L)
    for s in range(50):
        assert f(L + 1e-3 * rs(500 + s).standard_normal(L.shape)) >= best - 1e-12


def test_svt_tensor_is_prox_of_tnn():
    # prox of ||.||_TNN with weight 1/tau: argmin ||L||_TNN + 1/(2 tau) ||L - M||_F^2,
    # with ||L||_TNN evaluated as ||circ(L)||_* / n3 (independent of the SVT code).
    M = rs(51).standard_normal((4, 3, 5))
    tau = 0.9
    L = Cm.svt_tensor(M, tau)
    tnn = lambda Z: np.linalg.svd(T.circ(Z), compute_uv=False).sum() / 5
    f = lambda Z: tnn(Z) + 0.5 / tau * np.sum((Z - M) ** 2)
    best = f(L)
    for s in range(40):
        assert f(L + 1e-3 * rs(600 + s).standard_normal(L.shape)) >= best - 1e-12
    # n3 = 1 reduces to matrix SVT
    M1 = M[:, :, :1]
    np.testing.assert_allclose(Cm.svt_tensor(M1, tau)[:, :, 0], Cm.svt_matrix(M1[:, :, 0], tau), atol=1e-12)


def test_admm_completion_recovers_low_rank():
    X = _lowrank(20, 20, 6, 2, 60)
    mask = rs(61).random(X.shape) < 0.6
    L, E, Y, mu = Cm.tcomplete_svt(X, mask, iters=150)
    assert np.all(E[mask] == 0)
    rse = np.linalg.norm(L - X) / np.linalg.norm(X)
    assert rse < 1e-3
    # constraint residual L + E - P_Omega(X) is small at the end
    assert np.abs(L + E - np.where(mask, X, 0)).max() < 1e-5 * np.abs(X).max()
    assert abs(mu - min(1e-3 * 1.1 ** 150, 1e10)) < 1e-9 * mu


def test_admm_resume_equals_continuous_run():
    X = _lowrank(8, 7, 4, 2, 70)
    mask = rs(71).random(X.shape) < 0.5
    a = Cm.tcomplete_svt(X, mask, iters=10)
    b = Cm.tcomplete_svt(X, mask, iters=4)
    b = Cm.tcomplete_svt(X, mask, iters=6, state=b)
    for x, y in zip(a[:3], b[:3]):
        np.testing.assert_allclose(x, y, atol=1e-12)


def test_soft_threshold_is_prox_of_l1():
    # argmin_E lam |E|_1 + 1/2 |E - V|^2: no perturbation does better
    from oracle import completion_ref as C
    g = np.random.default_rng(31)
    V = g.standard_normal((4, 5, 3))
    lam = 0.4
    E = C.soft_threshold(V, lam)
    f = lambda Z: lam * np.abs(Z).sum() + 0.5 * np.sum((Z - V) ** 2)
    for s in range(20):
        assert f(E) <= f(E + 1e-3 * g.standard_normal(V.shape)) + 1e-12
    np.testing.assert_array_equal(C.soft_threshold(np.array([-2.0, -0.3, 0.0, 0.5, 1.5]), 0.5),
                                  [-1.5, 0.0, 0.0, 0.0, 1.0])


def test_robust_admm_recovers_low_rank_plus_sparse():
    # Algorithm 7 on X = L0 + S0, S0 5% large spikes: L is recovered
    from oracle import completion_ref as C
    from paper_1704_04362_gb300 import synth
    L0 = synth.lowrank_np(30, 30, 6, 2, seed=41).astype(np.float64)
    L0 /= np.sqrt(np.mean(L0 ** 2))
    g = np.random.default_rng(42)
    S0 = np.where(g.random(L0.shape) < 0.05, 10.0 * g.standard_normal(L0.shape), 0.0)
    L, E, Y, mu = C.trpca(L0 + S0, 120)
    assert np.linalg.norm(L - L0) / np.linalg.norm(L0) < 1e-3
    assert np.linalg.norm(E - S0) / np.linalg.norm(S0) < 1e-3


def test_robust_admm_with_huge_lambda_keeps_e_zero():
    # lambda large: the soft threshold kills E, the iteration is SVT of X - Y/mu
    from oracle import completion_ref as C
    X = np.random.default_rng(43).standard_normal((6, 5, 4))
    L, E, Y, mu = C.trpca(X, 5, lam=1e12)
    assert np.all(E == 0.0)
    # ... and the iteration is the completion form with every entry observed
    Lc, Ec, Yc, muc = C.tcomplete_svt(X, np.ones(X.shape, dtype=bool), 5)
    np.testing.assert_allclose(L, Lc, atol=1e-12)
    np.testing.assert_allclose(Y, Yc, atol=1e-12)
    assert mu == muc


def test_tcur_keeps_everything_when_every_slice_is_picked():
    from oracle import decomp_ref as D
    A = np.random.default_rng(61).standard_normal((8, 6, 4))
    Z, ci, ri, _ = D.tcur(A, 10 ** 6, 10 ** 6, 3)
    assert len(ci) == 6 and len(ri) == 8
    np.testing.assert_allclose(Z, A, atol=1e-10)


def test_tcur_reconstructs_low_tubal_rank_exactly():
    from oracle import decomp_ref as D
    from paper_1704_04362_gb300 import synth
    A = synth.lowrank_np(20, 16, 5, 2, seed=62, dtype=np.float64)
    Z, ci, ri, _ = D.tcur(A, 12, 14, 7)
    assert len(ci) >= 2 and len(ri) >= 2
    assert np.linalg.norm(Z - A) / np.linalg.norm(A) < 1e-9


def test_tcur_with_n3_one_is_matrix_cur():
    # Drineas et al.'s CUR: Z = C pinv(W) R with W the picked rows of C
    from oracle import decomp_ref as D, sampling_ref as S, philox_ref as P
    A = np.random.default_rng(63).standard_normal((12, 10, 1))
    Z, ci, ri, pr = D.tcur(A, 6, 7, 11)
    M = A[:, :, 0]
    _, qc = S.draw(S.probabilities(S.lateral_norms_sq(A), None, S.PROB_A2), 6, 11)
    C = M[:, ci] / np.sqrt(qc[ci])
    qr = S.keep_probabilities(pr, 7)
    W = C[ri, :] / np.sqrt(qr[ri])[:, None]
    R = M[ri, :] / np.sqrt(qr[ri])[:, None]
    np.testing.assert_allclose(Z[:, :, 0], C @ np.linalg.pinv(W) @ R, atol=1e-10)


def test_row_leverage_of_an_orthonormal_basis_is_uniform():
    from oracle import decomp_ref as D
    Q, _ = np.linalg.qr(np.random.default_rng(64).standard_normal((9, 9)))
    p = D.row_leverage(Q[:, :, None])                  # n3 = 1, full rank: U U^H = I
    np.testing.assert_allclose(p, np.full(9, 1 / 9), atol=1e-12)


def test_row_leverage_is_the_projector_diagonal_summed_over_frequencies():
    # for C of full column rank in every slice, ||U_hat_k(i, :)||^2 is the
    # i-th diagonal entry of the projector C_k (C_k^H C_k)^{-1} C_k^H: no SVD
    from oracle import decomp_ref as D
    C = np.random.default_rng(65).standard_normal((11, 4, 5))
    Ch = np.fft.fft(C, axis=2)
    lev = np.zeros(11)
    for f in range(5):
        M = Ch[:, :, f]
        lev += np.real(np.diag(M @ np.linalg.solve(M.conj().T @ M, M.conj().T)))
    np.testing.assert_allclose(D.row_leverage(C), lev / lev.sum(), atol=1e-12)
    assert abs(lev.sum() - 4 * 5) < 1e-9                 # trace of a rank-4 projector, 5 times


def test_top_r_row_leverage_is_the_top_eigenspace_of_c_ct():
    # n3 = 1: ||U_r(i, :)||^2 is the i-th diagonal entry of the projector on
    # the top-r eigenvectors of C C^T (a symmetric eigensolver, not an SVD)
    from oracle import decomp_ref as D
    C = np.random.default_rng(66).standard_normal((14, 6)) @ np.diag([9, 7, 5, 1, 0.5, 0.2])
    w, V = np.linalg.eigh(C @ C.T)
    top = V[:, np.argsort(w)[::-1][:3]]
    lev = np.sum(top ** 2, axis=1)
    np.testing.assert_allclose(D.row_leverage(C[:, :, None], 3), lev / 3, atol=1e-12)


def test_top_r_row_leverage_of_exact_rank_r_equals_the_cut_off_leverage():
    from oracle import decomp_ref as D
    from paper_1704_04362_gb300 import synth
    C = synth.lowrank_np(20, 9, 6, 3, seed=67, dtype=np.float64)
    np.testing.assert_allclose(D.row_leverage(C, 3), D.row_leverage(C, 0), atol=1e-10)
    assert abs(D.row_leverage(C, 5).sum() - 1) < 1e-12
    assert np.max(np.abs(D.row_leverage(C, 2) - D.row_leverage(C, 0))) > 1e-3


def test_cur_combine_with_n3_one_is_a_library_pinv():
    from oracle import decomp_ref as D
    g = np.random.default_rng(68)
    Ct = g.standard_normal((12, 5, 1))
    Rt = g.standard_normal((7, 9, 1))
    ridx = np.array([0, 2, 3, 5, 8, 10, 11])
    got = D.cur_combine(Ct, Rt, ridx, 1e-4)[:, :, 0]
    want = Ct[:, :, 0] @ np.linalg.pinv(Ct[ridx, :, 0], rcond=1e-4) @ Rt[:, :, 0]
    np.testing.assert_allclose(got, want, atol=1e-10)


def test_cur_tnn_with_every_slice_is_the_full_admm():
    # W~ = C~ = R~ = ADMM(X): L~ = C~ C~^dagger C~ = C~
    from oracle import completion_ref, decomp_ref as D
    from paper_1704_04362_gb300 import synth
    X = synth.lowrank_np(14, 12, 4, 2, seed=69, noise=0.05, dtype=np.float64)
    L, Ct, Rt, ci, ri, _ = D.cur_tnn(X, 10 ** 6, 10 ** 6, 1, 15, rtol=0.0)
    assert len(ci) == 12 and len(ri) == 14
    full = completion_ref.trpca(X, 15)[0]
    np.testing.assert_allclose(Ct, full, atol=1e-12)
    np.testing.assert_allclose(L, full, atol=1e-9 * np.abs(full).max())
    mask = np.random.default_rng(70).random(X.shape) < 0.6
    L, *_ = D.cur_tnn(X, 10 ** 6, 10 ** 6, 1, 15, mask=mask, rtol=0.0)
    full = completion_ref.tcomplete_svt(X, mask, 15)[0]
    np.testing.assert_allclose(L, full, atol=1e-9 * np.abs(full).max())


def test_cur_tnn_recovers_low_rank_plus_sparse_from_sampled_slices():
    from oracle import decomp_ref as D
    from paper_1704_04362_gb300 import synth
    L0 = synth.lowrank_np(60, 50, 4, 2, seed=71, dtype=np.float64)
    L0 /= np.sqrt(np.mean(L0 ** 2))
    g = np.random.default_rng(72)
    S0 = np.where(g.random(L0.shape) < 0.05, 10.0 * g.standard_normal(L0.shape), 0.0)
    L, Ct, Rt, ci, ri, _ = D.cur_tnn(L0 + S0, 25, 30, 3, 80, r=2)
    assert len(ci) < 50 and len(ri) < 60
    err = np.linalg.norm(L - L0) / np.linalg.norm(L0)
    assert err < 1e-3, err


def test_per_frequency_ranks_give_the_multi_rank_truncation():
    # with l = n2 the sketch is exact: frequency f truncated to r_f leaves
    # exactly the per-slice Eckart-Young error sum_{i > r_f} s_i^2 (counted
    # twice for the conjugate slices), against the exact t-SVD
    from oracle import decomp_ref as D, philox_ref as P
    g = np.random.default_rng(73)
    X = g.standard_normal((10, 8, 6))
    h = 4
    Om = P.sketch_signs(8, 8, h, 6, 2)
    ranks = np.array([3, 1, 0, 5])
    U, S, V = D.tsvd_randomized(X, 6, 2, 1, Om, ranks=ranks)
    from oracle.tensor_ref import tprod, ttranspose
    R = tprod(tprod(U, S), ttranspose(V))
    s_exact = [np.linalg.svd(np.fft.fft(X, axis=2)[:, :, f], compute_uv=False) for f in range(h)]
    w = [1, 2, 2, 1]
    err = sum(w[f] * np.sum(s_exact[f][ranks[f]:] ** 2) for f in range(h)) / 6
    assert abs(np.linalg.norm(X - R) ** 2 - err) < 1e-9 * np.linalg.norm(X) ** 2
    U0, S0, V0 = D.tsvd_randomized(X, 6, 2, 1, Om)
    Uf, Sf, Vf = D.tsvd_randomized(X, 6, 2, 1, Om, ranks=np.full(h, 6))
    assert np.array_equal(U0, Uf) and np.array_equal(S0, Sf)


def test_slice_sketch_recovers_exact_low_tubal_rank():
    # the sketch is rescaled picked columns of X_hat: with tubal rank r <= l
    # and generic picks their span is X's range, so the rank-r result is X
    from oracle import decomp_ref as D
    from oracle.tensor_ref import tprod, ttranspose
    from paper_1704_04362_gb300 import synth
    X = synth.lowrank_np(24, 30, 6, 3, seed=76, dtype=np.float64)
    Om = D.slice_sketch(X, 8, 4)
    assert Om.shape == (30, 8, 4) and np.count_nonzero(Om[:, :, 0]) == 8
    assert np.array_equal(Om[:, :, 0] != 0, Om[:, :, 3] != 0)         # same picks at every f
    U, S, V = D.tsvd_randomized(X, 3, 5, 0, Om)
    R = tprod(tprod(U, S), ttranspose(V))
    assert np.linalg.norm(R - X) / np.linalg.norm(X) < 1e-10
    # the columns of Omega select and rescale: X_hat Omega = picked columns / sqrt(l p)
    Xh = np.fft.fft(X, axis=2)
    j, c = np.nonzero(Om[:, :, 0])
    np.testing.assert_allclose((Xh[:, :, 1] @ Om[:, :, 1])[:, c], Xh[:, j, 1] * Om[j, c, 1], atol=1e-12)


def test_per_frequency_sketch_sizes():
    # slice f sketches with the first l_f columns of Omega and keeps
    # min(k, l_f) triplets: (a) l_f >= the tubal rank recovers X exactly and
    # the exact singular values; (b) a smaller l_f gives exactly min(k, l_f)
    # nonzero values, none above the exact ones (interlacing: the singular
    # values of Q^H X_hat with orthonormal Q); (c) only the first l_f columns
    # of Omega matter; (d) l_f = k + p everywhere is the plain call
    from oracle.tensor_ref import tprod, ttranspose
    g = np.random.default_rng(91)
    k, p, h = 4, 3, 4
    X = _lowrank(20, 16, 6, 3, 92)
    Om = P.sketch_signs(16, k + p, h, 6, seed=9)
    sizes = np.array([4, 3, 7, 5])
    U, S, V = D.tsvd_randomized(X, k, p, 1, Om, sketch_sizes=sizes)
    np.testing.assert_allclose(tprod(tprod(U, S), ttranspose(V)), X, atol=1e-10)
    _, s_exact, _ = D.tsvd_hat(X)
    _, s_rand, _ = D.tsvd_randomized_hat(X, k, p, 1, Om, sizes)
    for f in range(h):
        kf = min(k, sizes[f])
        np.testing.assert_allclose(s_rand[:kf, f], s_exact[:kf, f], rtol=1e-9, atol=1e-9)
        assert np.all(s_rand[kf:, f] == 0)
    Y = g.standard_normal((14, 12, 6))
    Om = P.sketch_signs(12, k + p, h, 6, seed=3)
    small = np.array([2, 1, 6, 3])
    _, s_small, _ = D.tsvd_randomized_hat(Y, k, p, 1, Om, small)
    _, s_full, _ = D.tsvd_hat(Y)
    for f in range(h):
        kf = min(k, small[f])
        assert np.count_nonzero(s_small[:, f]) == kf
        assert np.all(s_small[:kf, f] <= s_full[:kf, f] * (1 + 1e-12))
    Om2 = Om.copy()
    for f in range(h):
        Om2[:, small[f]:, f] = g.standard_normal((12, k + p - small[f]))
    _, s_other, _ = D.tsvd_randomized_hat(Y, k, p, 1, Om2, small)
    np.testing.assert_array_equal(s_other, s_small)
    U0, S0, V0 = D.tsvd_randomized(Y, k, p, 1, Om)
    U1, S1, V1 = D.tsvd_randomized(Y, k, p, 1, Om, sketch_sizes=np.full(h, k + p))
    assert np.array_equal(U0, U1) and np.array_equal(S0, S1) and np.array_equal(V0, V1)
