"""Decompositions (oracle; test infrastructure).

tsvd            Theorem 2.6 computed through Eq. (circ1): SVD of every Fourier
                frontal slice, economy size m = min(n1, n2), singular values
                descending, conjugate-symmetric slices filled from the half
                spectrum so that U, S, V are real.
tsvd_randomized Randomized low-tubal-rank t-SVD: per Fourier slice the
                range finder with q power iterations of Halko, Martinsson and
                Tropp (SIAM Review 2011, Algorithms 4.3/5.1), test matrix
                passed in.  The paper names randomized approximations
                (Section 5.2) without fixing one; this is the reading used.
tproject, tcx   Algorithm 3 (t-project) and Algorithm 4 (t-CX).
tcur            Algorithm 5 (t-CUR) with the row leverage probabilities of
                eq. (colprob_rows_exact).
cur_tnn         Algorithm 6 (CUR t-NN): ADMM on the picked lateral and
                horizontal slices, then C~ * W~^dagger * R~.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from . import sampling_ref
from .tensor_ref import fft3, ifft3, half_spectrum, hermitian_fill


def _real_slice(k: int, n3: int) -> bool:
    return k == 0 or (n3 % 2 == 0 and k == n3 // 2)


def tsvd_hat(X: np.ndarray):
    """Half-spectrum facewise SVD: returns (Uh, s, Vh) with Uh n1 x m x h,
    s m x h (descending), Vh n2 x m x h, and X_hat_k = Uh_k diag(s_k) Vh_k^H."""
    n1, n2, n3 = X.shape
    m = min(n1, n2)
    h = n3 // 2 + 1
    Xh = half_spectrum(fft3(X))
    Uh = np.zeros((n1, m, h), dtype=np.complex128)
    Vh = np.zeros((n2, m, h), dtype=np.complex128)
    s = np.zeros((m, h))
    for k in range(h):
        M = Xh[:, :, k]
        if _real_slice(k, n3):
            M = M.real
        u, sv, vt = scipy.linalg.svd(M, full_matrices=False, lapack_driver="gesvd")
        Uh[:, :, k] = u
        s[:, k] = sv
        Vh[:, :, k] = np.conj(vt).T
    return Uh, s, Vh


def tsvd(X: np.ndarray):
    """t-SVD X = U * S * V^T (Theorem 2.6), economy: U n1 x m x n3,
    S m x m x n3 (f-diagonal), V n2 x m x n3."""
    n1, n2, n3 = X.shape
    m = min(n1, n2)
    Uh, s, Vh = tsvd_hat(X)
    Sh = np.zeros((m, m, s.shape[1]), dtype=np.complex128)
    for k in range(s.shape[1]):
        Sh[:, :, k] = np.diag(s[:, k])
    U = ifft3(hermitian_fill(Uh, n3)).real
    S = ifft3(hermitian_fill(Sh, n3)).real
    V = ifft3(hermitian_fill(Vh, n3)).real
    return U, S, V


def truncate_error_sq(s: np.ndarray, n3: int, r: int) -> float:
    """||X - X_r||_F^2 for the tubal-rank-r truncation of the t-SVD:
    (1/n3) sum over all n3 slices of sum_{i>r} sigma_{i,k}^2 (Parseval), with
    the half spectrum counted twice for its conjugate partners."""
    h = s.shape[1]
    tot = 0.0
    for k in range(h):
        w = 1.0 if _real_slice(k, n3) else 2.0
        tot += w * float(np.sum(s[r:, k] ** 2))
    return tot / n3


def _orth(Y: np.ndarray) -> np.ndarray:
    """Orthonormal basis of range(Y) (economy Householder QR)."""
    Q, _ = np.linalg.qr(Y)
    return Q


def tsvd_randomized_hat(X: np.ndarray, k: int, p: int, q: int, Omega: np.ndarray,
                        sketch_sizes=None):
    """Per half-spectrum slice: Y = X_hat Omega; q power iterations
    Q <- orth(X_hat^H Q), Q <- orth(X_hat Q); B = Q^H X_hat; SVD of B; keep k.
    Omega is n2 x (k+p) x h.  sketch_sizes (h integers, the per-frequency
    sketch sizes of the multi-rank form of Section 2): slice f sketches with
    the first l_f = min(max(size_f, 1), k + p) columns of Omega and keeps its
    top min(k, l_f) triplets (the rest zero).  Returns (Uh n1 x k x h,
    s k x h, Vh n2 x k x h)."""
    n1, n2, n3 = X.shape
    h = n3 // 2 + 1
    ell = k + p
    assert Omega.shape == (n2, ell, h)
    Xh = half_spectrum(fft3(X))
    Uh = np.zeros((n1, k, h), dtype=np.complex128)
    Vh = np.zeros((n2, k, h), dtype=np.complex128)
    s = np.zeros((k, h))
    for f in range(h):
        lf = ell if sketch_sizes is None else min(max(int(sketch_sizes[f]), 1), ell)
        kf = min(k, lf)
        M = Xh[:, :, f]
        if _real_slice(f, n3):
            M = M.real.astype(np.complex128)
        Q = _orth(M @ Omega[:, :lf, f])
        for _ in range(q):
            Q = _orth(np.conj(M).T @ Q)
            Q = _orth(M @ Q)
        Bm = np.conj(Q).T @ M
        ub, sb, vbt = scipy.linalg.svd(Bm, full_matrices=False, lapack_driver="gesvd")
        Uh[:, :kf, f] = (Q @ ub)[:, :kf]
        s[:kf, f] = sb[:kf]
        Vh[:, :kf, f] = np.conj(vbt).T[:, :kf]
    return Uh, s, Vh


def slice_sketch(X: np.ndarray, ell: int, seed: int) -> np.ndarray:
    """Test matrix of the slice (t-CX) sketch: ell lateral slices drawn i.i.d.
    with probability p_j = ||X(:,j,:)||_F^2 / ||X||_F^2 (Philox stream 2,
    with-replacement draws), Omega(j_c, c, f) = 1/sqrt(ell p_{j_c}) at every
    half-spectrum frequency f, so that X_hat_f Omega_f is the rescaled picked
    columns.  Returns Omega (n2 x ell x h, real)."""
    from .philox_ref import STREAM_SKETCH
    X = np.asarray(X, dtype=np.float64)
    n2, n3 = X.shape[1], X.shape[2]
    h = n3 // 2 + 1
    p = sampling_ref.probabilities(sampling_ref.lateral_norms_sq(X), None, sampling_ref.PROB_A2)
    idx, s = sampling_ref.draw_iid(p, ell, seed, STREAM_SKETCH)
    Om = np.zeros((n2, ell, h))
    for c, j in enumerate(idx):
        Om[j, c, :] = 1.0 / np.sqrt(s[c])
    return Om


def tsvd_randomized(X: np.ndarray, k: int, p: int, q: int, Omega: np.ndarray, ranks=None,
                    sketch_sizes=None):
    """Randomized tubal-rank-k t-SVD; same output form as ``tsvd`` with m = k.
    ranks (h integers): half-spectrum slice f keeps only its top
    min(max(r_f, 0), k) triplets (the multi-rank of Section 2);
    sketch_sizes: per-frequency sketch sizes (see tsvd_randomized_hat)."""
    n3 = X.shape[2]
    Uh, s, Vh = tsvd_randomized_hat(X, k, p, q, Omega, sketch_sizes)
    if ranks is not None:
        for f in range(s.shape[1]):
            r = min(max(int(ranks[f]), 0), k)
            Uh[:, r:, f] = 0.0
            Vh[:, r:, f] = 0.0
            s[r:, f] = 0.0
    Sh = np.zeros((k, k, s.shape[1]), dtype=np.complex128)
    for f in range(s.shape[1]):
        Sh[:, :, f] = np.diag(s[:, f])
    U = ifft3(hermitian_fill(Uh, n3)).real
    S = ifft3(hermitian_fill(Sh, n3)).real
    V = ifft3(hermitian_fill(Vh, n3)).real
    return U, S, V


def pinv_matlab(M: np.ndarray) -> np.ndarray:
    """Moore-Penrose pseudo-inverse with MATLAB's default cut-off
    max(size) * eps(sigma_max)."""
    u, sv, vt = np.linalg.svd(M, full_matrices=False)
    if sv.size == 0:
        return np.zeros((M.shape[1], M.shape[0]), dtype=M.dtype)
    tol = max(M.shape) * np.spacing(sv[0])
    inv = np.where(sv > tol, 1.0 / np.where(sv > tol, sv, 1.0), 0.0)
    return (np.conj(vt).T * inv) @ np.conj(u).T


def tproject(X: np.ndarray, C: np.ndarray) -> np.ndarray:
    """t-project Pi_C(X) = C * C^dagger * X, Algorithm 3 (all n3 slices)."""
    Xh = fft3(X)
    Ch = fft3(C)
    Zh = np.empty_like(Xh)
    for f in range(X.shape[2]):
        Zh[:, :, f] = Ch[:, :, f] @ (pinv_matlab(Ch[:, :, f]) @ Xh[:, :, f])
    return ifft3(Zh).real


def tcx(A: np.ndarray, c: int, seed: int, mode: int = sampling_ref.PROB_A2,
        p_given: np.ndarray | None = None):
    """t-CX, Algorithm 4: draw lateral slices with probability min{1, c p_i},
    C = rescaled picked slices, Z = Pi_C(A).  Returns (Z, idx, q)."""
    A = np.asarray(A, dtype=np.float64)
    if mode == sampling_ref.PROB_GIVEN:
        p = np.asarray(p_given, dtype=np.float64)
    else:
        p = sampling_ref.probabilities(sampling_ref.lateral_norms_sq(A), None,
                                       sampling_ref.PROB_A2)
    idx, q = sampling_ref.draw(p, c, seed)
    if len(idx) == 0:
        return np.zeros_like(A), idx, q
    C = A[:, idx, :] / np.sqrt(q[idx])[None, :, None]
    return tproject(A, C), idx, q


def row_leverage(C: np.ndarray, r: int = 0) -> np.ndarray:
    """Horizontal-slice probabilities of Algorithm 5 (eq. colprob_rows_exact,
    beta = 1): p_i proportional to ||U_hat_{i::}||_F^2, U_hat_k the left
    singular vectors of every Fourier slice C_hat_k (all n3 frequencies) whose
    singular values pass MATLAB's pinv cut-off max(n1, c) eps(s_max), and with
    r > 0 only the top r of them (the rank parameter of Algorithm 5; the
    top-r estimate of the remark after Corollary 3.7); normalised to sum 1."""
    C = np.asarray(C, dtype=np.float64)
    n1, c, n3 = C.shape
    Ch = fft3(C)
    lev = np.zeros(n1)
    for f in range(n3):
        u, sv, _ = np.linalg.svd(Ch[:, :, f], full_matrices=False)
        if sv.size == 0 or sv[0] == 0:
            continue
        keep = sv > max(n1, c) * np.spacing(sv[0])
        if r > 0:
            keep[r:] = False                   # sv is descending
        lev += np.sum(np.abs(u[:, keep]) ** 2, axis=1)
    tot = lev.sum()
    return lev / tot if tot > 0 else lev


def tcur(A: np.ndarray, c: int, l: int, seed: int, mode: int = sampling_ref.PROB_A2,
         p_cols: np.ndarray | None = None, p_rows: np.ndarray | None = None, r: int = 0):
    """t-CUR, Algorithm 5: lateral slices as t-CX (Philox stream 0), horizontal
    slices with probability min{1, l p_i} (stream 1; p_i the row leverage of
    C unless given), R_hat_k = D S^T A_hat_k, U_hat_k = (D S^T C_hat_k)^dagger,
    Z_hat_k = C_hat_k U_hat_k R_hat_k.  Returns (Z, col_idx, row_idx, p_rows)."""
    from .philox_ref import STREAM_HORIZONTAL
    A = np.asarray(A, dtype=np.float64)
    n1, n2, n3 = A.shape
    if mode == sampling_ref.PROB_GIVEN:
        p = np.asarray(p_cols, dtype=np.float64)
    else:
        p = sampling_ref.probabilities(sampling_ref.lateral_norms_sq(A), None,
                                       sampling_ref.PROB_A2)
    cidx, qc = sampling_ref.draw(p, c, seed)
    if len(cidx) == 0:
        return np.zeros_like(A), cidx, np.zeros(0, dtype=cidx.dtype), np.zeros(n1)
    C = A[:, cidx, :] / np.sqrt(qc[cidx])[None, :, None]
    pr = row_leverage(C, r) if p_rows is None else np.asarray(p_rows, dtype=np.float64)
    ridx, qr = sampling_ref.draw(pr, l, seed, STREAM_HORIZONTAL)
    if len(ridx) == 0:
        return np.zeros_like(A), cidx, ridx, pr
    d = 1.0 / np.sqrt(qr[ridx])
    Ah = fft3(A)
    Ch = fft3(C)
    Zh = np.empty_like(Ah)
    for f in range(n3):
        R = d[:, None] * Ah[ridx, :, f]
        W = d[:, None] * Ch[ridx, :, f]
        Zh[:, :, f] = Ch[:, :, f] @ (pinv_matlab(W) @ R)
    return ifft3(Zh).real, cidx, ridx, pr


def pinv_rtol(M: np.ndarray, rtol: float) -> np.ndarray:
    """Pseudo-inverse over the singular values above rtol * sigma_max (MATLAB's
    pinv(M, tol) with tol = rtol sigma_max); rtol <= 0 gives pinv_matlab."""
    if rtol <= 0:
        return pinv_matlab(M)
    u, sv, vt = np.linalg.svd(M, full_matrices=False)
    if sv.size == 0:
        return np.zeros((M.shape[1], M.shape[0]), dtype=M.dtype)
    keep = sv > rtol * sv[0]
    inv = np.where(keep, 1.0 / np.where(keep, sv, 1.0), 0.0)
    return (np.conj(vt).T * inv) @ np.conj(u).T


def cur_combine(Ct: np.ndarray, Rt: np.ndarray, ridx: np.ndarray, rtol: float) -> np.ndarray:
    """Steps 6-7 of Algorithm 6: W~ = the horizontal slices ridx of C~,
    U~ = W~^dagger and L~ = C~ * U~ * R~, per Fourier slice."""
    Ch = fft3(Ct)
    Rh = fft3(Rt)
    n1, n3 = Ct.shape[0], Ct.shape[2]
    Lh = np.empty((n1, Rt.shape[1], n3), dtype=complex)
    for f in range(n3):
        Lh[:, :, f] = Ch[:, :, f] @ (pinv_rtol(Ch[ridx, :, f], rtol) @ Rh[:, :, f])
    return ifft3(Lh).real


def cur_tnn(X: np.ndarray, c: int, l: int, seed: int, iters: int, r: int = 0, mask=None,
            lam=None, mode: int = sampling_ref.PROB_A2, p_cols=None, p_rows=None,
            rtol: float = 1e-4, mu0: float = 1e-3, rho: float = 1.1, mu_max: float = 1e10):
    """CUR t-NN, Algorithm 6.  Lateral slices C of X are picked with
    probability min{1, c p_j} (Philox stream 0; p from the lateral norms of
    the observed data, or given), horizontal slices R with probability
    min{1, l p_i} (stream 1; p_i the top-r row leverage of C, or given); the
    picked slices are not rescaled.  C~ and R~ are the ADMM solutions of
    problem tlow7 (mask None; lambda per sub-tensor from its own sizes unless
    given) or of problem tlow6 (the mask's observed entries).  Returns
    (L~, C~, R~, col_idx, row_idx, p_rows)."""
    from . import completion_ref
    from .philox_ref import STREAM_HORIZONTAL
    X = np.asarray(X, dtype=np.float64)
    n1, n2, n3 = X.shape
    obs = None if mask is None else np.asarray(mask).astype(bool)
    Xo = X if obs is None else np.where(obs, X, 0.0)
    if mode == sampling_ref.PROB_GIVEN:
        p = np.asarray(p_cols, dtype=np.float64)
    else:
        p = sampling_ref.probabilities(sampling_ref.lateral_norms_sq(Xo), None,
                                       sampling_ref.PROB_A2)
    cidx, _ = sampling_ref.draw(p, c, seed)
    empty = np.zeros(0, dtype=cidx.dtype)
    if len(cidx) == 0:
        return (np.zeros_like(X), np.zeros((n1, 0, n3)), np.zeros((0, n2, n3)), cidx, empty,
                np.zeros(n1))
    C = Xo[:, cidx, :]
    pr = row_leverage(C, r) if p_rows is None else np.asarray(p_rows, dtype=np.float64)
    ridx, _ = sampling_ref.draw(pr, l, seed, STREAM_HORIZONTAL)
    if len(ridx) == 0:
        return np.zeros_like(X), np.zeros((n1, 0, n3)), np.zeros((0, n2, n3)), cidx, ridx, pr
    R = Xo[ridx, :, :]

    def admm(T, M):
        if M is None:
            return completion_ref.trpca(T, iters, lam, mu0, rho, mu_max)[0]
        return completion_ref.tcomplete_svt(T, M, iters, mu0, rho, mu_max)[0]
    Ct = admm(C, None if obs is None else obs[:, cidx, :])
    Rt = admm(R, None if obs is None else obs[ridx, :, :])
    return cur_combine(Ct, Rt, ridx, rtol), Ct, Rt, cidx, ridx, pr
