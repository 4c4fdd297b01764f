"""Tensor completion by ADMM with tensor singular-value thresholding (oracle).

Test infrastructure.  Appendix Algorithm 7 solves the robust problem (tlow7);
the paper says a small change gives the completion problem (tlow6).  The
reading used here (Lu et al.'s TNN completion form): minimise ||L||_TNN
subject to L + E = X with E zero on the observed set Omega, where X is zero
off Omega.  One iteration, with tau = 1/mu:

    L <- SVT_tau(X - E - Y/mu)           (tensor SVT, below)
    E <- P_{Omega^c}(X - L - Y/mu)       (E is free where nothing is observed)
    Y <- Y + mu (L + E - X)
    mu <- min(rho mu, mu_max)

Tensor SVT: by Parseval, ||L - M||_F^2 = (1/n3) sum_k ||L_hat_k - M_hat_k||_F^2,
and ||L||_TNN = (1/n3) sum_k ||L_hat_k||_*, so the proximal step splits into
matrix singular-value soft-thresholding of every Fourier slice with the same
threshold tau (unnormalised transform).  Constants of Algorithm 7:
rho = 1.1, mu0 = 1e-3, mu_max = 1e10.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from .tensor_ref import fft3, ifft3, half_spectrum, hermitian_fill


def svt_matrix(M: np.ndarray, tau: float) -> np.ndarray:
    """U max(Sigma - tau, 0) V^H (Cai, Candes and Shen's shrinkage)."""
    if M.size == 0:
        return M.copy()
    u, sv, vt = scipy.linalg.svd(M, full_matrices=False, lapack_driver="gesvd")
    return (u * np.maximum(sv - tau, 0.0)) @ vt


def svt_tensor(M: np.ndarray, tau: float) -> np.ndarray:
    """Tensor SVT: shrink the singular values of every Fourier slice by tau."""
    n3 = M.shape[2]
    Mh = half_spectrum(fft3(M))
    Lh = np.empty_like(Mh)
    for k in range(Mh.shape[2]):
        S = Mh[:, :, k]
        if k == 0 or (n3 % 2 == 0 and k == n3 // 2):
            S = S.real
        Lh[:, :, k] = svt_matrix(S, tau)
    return ifft3(hermitian_fill(Lh, n3)).real


def admm_step(X, mask, L, E, Y, mu, rho=1.1, mu_max=1e10):
    """One iteration of the completion ADMM (module docstring).  mask is
    True/1 on observed entries.  Returns (L, E, Y, mu_next)."""
    obs = np.asarray(mask).astype(bool)
    L = svt_tensor(X - E - Y / mu, 1.0 / mu)
    E = np.where(obs, 0.0, X - L - Y / mu)
    Y = Y + mu * (L + E - X)
    return L, E, Y, min(rho * mu, mu_max)


def tcomplete_svt(X, mask, iters: int, mu0=1e-3, rho=1.1, mu_max=1e10,
                  state=None):
    """Run ``iters`` ADMM iterations from (L, E, Y, mu) = state or zeros/mu0.
    X is taken as P_Omega(X).  Returns (L, E, Y, mu)."""
    obs = np.asarray(mask).astype(bool)
    Xo = np.where(obs, np.asarray(X, dtype=np.float64), 0.0)
    if state is None:
        L = np.zeros_like(Xo)
        E = np.zeros_like(Xo)
        Y = np.zeros_like(Xo)
        mu = float(mu0)
    else:
        L, E, Y = (np.array(s, dtype=np.float64) for s in state[:3])
        mu = float(state[3])
    for _ in range(iters):
        L, E, Y, mu = admm_step(Xo, obs, L, E, Y, mu, rho, mu_max)
    return L, E, Y, mu


# ---------------------------------------------------------------- robust form
# Algorithm 7 as printed, for problem (tlow7): minimise ||L||_TNN + lambda ||E||_1
# subject to X = L + E.  The E-step's closed form is the entrywise soft
# threshold of X - L - Y/mu at lambda/mu (the proximal map of lambda ||.||_1
# with weight 1/mu).  The paper leaves lambda open; the default is Lu et al.'s
# 1 / sqrt(max(n1, n2) n3).

def default_lambda(n1: int, n2: int, n3: int) -> float:
    return 1.0 / np.sqrt(max(n1, n2) * n3)


def soft_threshold(V: np.ndarray, t: float) -> np.ndarray:
    return np.sign(V) * np.maximum(np.abs(V) - t, 0.0)


def admm_robust_step(X, L, E, Y, mu, lam, rho=1.1, mu_max=1e10):
    """One iteration of Algorithm 7 (tlow7).  Returns (L, E, Y, mu_next)."""
    L = svt_tensor(X - E - Y / mu, 1.0 / mu)
    E = soft_threshold(X - L - Y / mu, lam / mu)
    Y = Y + mu * (L + E - X)
    return L, E, Y, min(rho * mu, mu_max)


def trpca(X, iters: int, lam=None, mu0=1e-3, rho=1.1, mu_max=1e10, state=None):
    """Run ``iters`` iterations of Algorithm 7 from (L, E, Y, mu) = state or
    zeros/mu0.  Returns (L, E, Y, mu)."""
    X = np.asarray(X, dtype=np.float64)
    n1, n2, n3 = X.shape
    lam = default_lambda(n1, n2, n3) if lam is None else float(lam)
    if state is None:
        L, E, Y = np.zeros_like(X), np.zeros_like(X), np.zeros_like(X)
        mu = float(mu0)
    else:
        L, E, Y = (np.array(s, dtype=np.float64) for s in state[:3])
        mu = float(state[3])
    for _ in range(iters):
        L, E, Y, mu = admm_robust_step(X, L, E, Y, mu, lam, rho, mu_max)
    return L, E, Y, mu
