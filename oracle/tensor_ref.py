"""Tensor algebra of Section 2 in plain float64 (oracle; test infrastructure).

Conventions (Section 2, "Operators"): a third-order tensor X has shape
(n1, n2, n3) and entry X[i, j, t]; X[:, :, t] is the t-th frontal slice,
X[:, j, :] the j-th lateral slice, X[i, :, :] the i-th horizontal slice and
X[i, j, :] a tube.  The transform along mode 3 is MATLAB's ``fft(X, [], 3)``:
unnormalised, kernel exp(-2*pi*1j*k*t/n3); the inverse carries 1/n3.
"""
from __future__ import annotations

import numpy as np


def dft_matrix(n3: int) -> np.ndarray:
    """F_{n3}[k, t] = exp(-2 pi i (k t mod n3) / n3)  (the F_{n3} of Eq. circ1).

    The angle is built from the integer residue (k*t) mod n3 so that large n3
    does not lose accuracy in the argument.
    """
    k = np.arange(n3, dtype=np.int64)
    r = np.outer(k, k) % n3
    ang = -2.0 * np.pi * r.astype(np.float64) / n3
    return np.cos(ang) + 1j * np.sin(ang)


# Above this tube length the transform is taken from numpy.fft (a library
# primitive computing the same sum); below it the F_{n3} contraction is
# written out.  tests/test_oracle_tensor.py pins both against each other.
LIBRARY_FFT_ABOVE = 256


def fft3(X: np.ndarray) -> np.ndarray:
    """X_hat = fft(X, [], 3): X_hat[:, :, k] = sum_t X[:, :, t] F[k, t] (Section 2)."""
    X = np.asarray(X)
    if X.shape[2] > LIBRARY_FFT_ABOVE:
        return np.fft.fft(np.asarray(X, dtype=np.complex128), axis=2)
    F = dft_matrix(X.shape[2])
    return np.asarray(X, dtype=np.complex128) @ F.T


def ifft3(Xh: np.ndarray) -> np.ndarray:
    """ifft(X_hat, [], 3): X[:, :, t] = (1/n3) sum_k X_hat[:, :, k] conj(F[k, t])."""
    n3 = Xh.shape[2]
    if n3 > LIBRARY_FFT_ABOVE:
        return np.fft.ifft(np.asarray(Xh, dtype=np.complex128), axis=2)
    F = dft_matrix(n3)
    return (np.asarray(Xh, dtype=np.complex128) @ np.conj(F)) / n3


def circ(Z: np.ndarray) -> np.ndarray:
    """Block-circulant matrix of Def. 2.1: block (a, b) is Z[:, :, (a - b) mod n3]."""
    n1, n2, n3 = Z.shape
    M = np.zeros((n1 * n3, n2 * n3), dtype=Z.dtype)
    for a in range(n3):
        for b in range(n3):
            M[a * n1:(a + 1) * n1, b * n2:(b + 1) * n2] = Z[:, :, (a - b) % n3]
    return M


def unfold(X: np.ndarray) -> np.ndarray:
    """unfold(X) of Def. 2.1: frontal slices stacked vertically, (n2*n3) x n4."""
    n2, n4, n3 = X.shape
    return np.concatenate([X[:, :, t] for t in range(n3)], axis=0)


def fold(M: np.ndarray, n3: int) -> np.ndarray:
    """Inverse of unfold: split the rows of M into n3 frontal slices."""
    rows, n4 = M.shape
    n1 = rows // n3
    return np.stack([M[t * n1:(t + 1) * n1, :] for t in range(n3)], axis=2)


def tprod_circ(Z: np.ndarray, X: np.ndarray) -> np.ndarray:
    """t-product by its definition, Eq. (tprod): fold(circ(Z) . unfold(X)).

    Literal and O((n1 n3)(n2 n3) n4); for tiny inputs only.
    """
    n1, n2, n3 = Z.shape
    assert X.shape[0] == n2 and X.shape[2] == n3
    return fold(circ(Z) @ unfold(X), n3)


def facewise(Ah: np.ndarray, Bh: np.ndarray) -> np.ndarray:
    """C_hat[:, :, k] = A_hat[:, :, k] B_hat[:, :, k] for every k (Algorithm 1, loop)."""
    Ca = np.transpose(Ah, (2, 0, 1)) @ np.transpose(Bh, (2, 0, 1))
    return np.transpose(Ca, (1, 2, 0))


def tprod(Z: np.ndarray, X: np.ndarray, *, return_imag: bool = False):
    """t-product in the Fourier domain, Algorithm 1 (all n3 frontal slices).

    Returns the real part of the inverse transform; with ``return_imag`` also
    the largest imaginary magnitude (zero up to rounding for real inputs).
    """
    Zh = fft3(Z)
    Xh = fft3(X)
    Ch = facewise(Zh, Xh)
    C = ifft3(Ch)
    if return_imag:
        return C.real, float(np.max(np.abs(C.imag))) if C.size else 0.0
    return C.real


def ttranspose(X: np.ndarray) -> np.ndarray:
    """Conjugate transpose (Section 2.1): transpose each frontal slice, then
    reverse the order of slices 2..n3."""
    n1, n2, n3 = X.shape
    Y = np.empty((n2, n1, n3), dtype=X.dtype)
    Y[:, :, 0] = np.conj(X[:, :, 0]).T
    for t in range(1, n3):
        Y[:, :, t] = np.conj(X[:, :, n3 - t]).T
    return Y


def identity(n: int, n3: int) -> np.ndarray:
    """Identity tensor (Section 2.1): first frontal slice I_n, the rest zero."""
    I = np.zeros((n, n, n3))
    I[:, :, 0] = np.eye(n)
    return I


def fro(X: np.ndarray) -> float:
    """Frobenius norm sqrt(sum |x_ijk|^2) (Section 2, "Norms")."""
    return float(np.sqrt(np.sum(np.abs(np.asarray(X, dtype=np.complex128)) ** 2)))


def tnn(X: np.ndarray) -> float:
    """Tensor nuclear norm, Eq. (tnuc): (1/n3) sum_k ||X_hat_k||_*."""
    Xh = fft3(X)
    n3 = X.shape[2]
    return float(sum(np.linalg.svd(Xh[:, :, k], compute_uv=False).sum()
                     for k in range(n3)) / n3)


def tspectral(X: np.ndarray) -> float:
    """Tensor spectral norm, Def. 2.7: max_k ||X_hat_k||_2."""
    Xh = fft3(X)
    return float(max(np.linalg.svd(Xh[:, :, k], compute_uv=False)[0]
                     for k in range(X.shape[2])))


def half_spectrum(Xh: np.ndarray) -> np.ndarray:
    """Slices 0..floor(n3/2) of a transform; the rest follow by conjugation
    (X_hat_{n3-k} = conj(X_hat_k) for real X)."""
    return Xh[:, :, : Xh.shape[2] // 2 + 1]


def hermitian_fill(Hh: np.ndarray, n3: int) -> np.ndarray:
    """Rebuild all n3 slices from the half spectrum via X_hat_{n3-k} = conj(X_hat_k)."""
    h = n3 // 2 + 1
    assert Hh.shape[2] == h
    out = np.empty(Hh.shape[:2] + (n3,), dtype=np.complex128)
    out[:, :, :h] = Hh
    for k in range(h, n3):
        out[:, :, k] = np.conj(Hh[:, :, n3 - k])
    return out
