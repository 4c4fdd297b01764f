"""Seeded synthetic inputs shaped like the paper's workloads.

This module draws inputs only.  It holds none of the library's arithmetic and
none of the oracle's: where a workload is defined as a t-product of random
factors (low tubal rank), the product is formed with the FFT and batched
matmul of NumPy or PyTorch, library routines that neither side under test
uses.  Every generator is deterministic given its seed.

Tensors are n1 x n2 x n3 with entry (i, j, t) stored at i + n1*(j + n2*t)
(column-major, frontal slices contiguous).  NumPy results are Fortran-ordered
arrays of shape (n1, n2, n3); PyTorch results are tensors of logical shape
(n1, n2, n3) with strides (1, n1, n1*n2).
"""
from __future__ import annotations

import numpy as np


# ---------------------------------------------------------------- layout helpers

def fortran_empty_torch(n1, n2, n3, dtype=None, device="cuda"):
    """Uninitialised torch tensor of logical shape (n1, n2, n3), column-major."""
    import torch
    dtype = dtype or torch.float32
    return torch.empty((n3, n2, n1), dtype=dtype, device=device).permute(2, 1, 0)


def to_fortran_torch(x):
    """Copy a torch tensor of logical shape (n1, n2, n3) into column-major storage."""
    return x.permute(2, 1, 0).contiguous().permute(2, 1, 0)


# ---------------------------------------------------------------- NumPy (small)

def iid_normal(shape, seed: int, dtype=np.float32) -> np.ndarray:
    """Entries iid N(0, 1) drawn in storage order by PCG64(seed)."""
    n = int(np.prod(shape))
    raw = np.random.default_rng(seed).standard_normal(n).astype(dtype)
    return raw.reshape(shape, order="F")


def _tprod_lib_np(P: np.ndarray, Q: np.ndarray) -> np.ndarray:
    """P*Q formed with numpy.fft + matmul (input synthesis only)."""
    n3 = P.shape[2]
    Ph = np.fft.rfft(P.astype(np.float64), axis=2)
    Qh = np.fft.rfft(Q.astype(np.float64), axis=2)
    Ch = np.einsum("irk,rjk->ijk", Ph, Qh)
    return np.fft.irfft(Ch, n=n3, axis=2)


def lowrank_np(n1, n2, n3, r, seed, noise=0.0, factor="normal", dtype=np.float32):
    """t-product of two random factors of tubal rank r plus Gaussian noise of
    standard deviation ``noise`` x RMS(clean).  factor: "normal" (N(0,1)) or
    "gamma" (Gamma(2, 1), nonnegative)."""
    g = np.random.default_rng(seed)
    if factor == "normal":
        P = g.standard_normal((n1, r, n3))
        Q = g.standard_normal((r, n2, n3))
    elif factor == "gamma":
        P = g.gamma(2.0, 1.0, (n1, r, n3))
        Q = g.gamma(2.0, 1.0, (r, n2, n3))
    else:
        raise ValueError(factor)
    X = _tprod_lib_np(P, Q)
    if noise:
        rms = np.sqrt(np.mean(X * X))
        X = X + noise * rms * g.standard_normal(X.shape)
    return np.asfortranarray(X.astype(dtype))


def msi_like_np(n1=128, n2=128, n3=2000, r=15, seed=0, spike_density=1e-3,
                spike_scale=5.0, noise=5e-3, dtype=np.float32):
    """Mass-spectrometry-imaging-shaped tensor (pixels x pixels x channels):
    t-product of Gamma(2,1) factors at tubal rank r scaled to unit RMS, plus
    sparse positive spikes (density spike_density, Exp with mean spike_scale)
    and Gaussian noise of std ``noise`` (unit-RMS units)."""
    g = np.random.default_rng(seed)
    X = lowrank_np(n1, n2, n3, r, seed, noise=0.0, factor="gamma", dtype=np.float64)
    X = X / np.sqrt(np.mean(X * X))
    spikes = (g.random(X.shape) < spike_density) * g.exponential(spike_scale, X.shape)
    X = X + spikes + noise * g.standard_normal(X.shape)
    return np.asfortranarray(X.astype(dtype))


def video_sizes(count=256, seed=0, lo=(64, 64, 16), hi=(480, 360, 120)):
    """(H, W, T) drawn uniformly and independently per axis."""
    g = np.random.default_rng(seed)
    return [tuple(int(g.integers(lo[a], hi[a] + 1)) for a in range(3)) for _ in range(count)]


def video_np(n1, n2, n3, r=10, seed=0, sigma=0.01, observed=0.5, dtype=np.float32):
    """Completion workload: tubal rank r (N(0,1) factors) scaled to unit RMS,
    plus N(0, sigma^2) noise, with a uniform observation mask of the given
    fraction.  Returns (truth, noisy, mask uint8)."""
    g = np.random.default_rng(seed + 7919)
    L = lowrank_np(n1, n2, n3, r, seed, noise=0.0, dtype=np.float64)
    L = L / np.sqrt(np.mean(L * L))
    Xn = L + sigma * g.standard_normal(L.shape)
    mask = (g.random(L.shape) < observed).astype(np.uint8)
    return (np.asfortranarray(L.astype(dtype)), np.asfortranarray(Xn.astype(dtype)),
            np.asfortranarray(mask))


# ---------------------------------------------------------------- PyTorch (large, on device)

def lowrank_torch(n1, n2, n3, r, seed, noise=0.0, device="cuda", chunk=8):
    """Device-side version of ``lowrank_np`` (normal factors) for workloads too
    large to draw on the host: torch.Generator(seed), torch.fft, torch.matmul.
    Returns a column-major float32 tensor of logical shape (n1, n2, n3)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    P = torch.randn((n3, r, n1), generator=g, device=device).permute(2, 1, 0)
    Q = torch.randn((n3, n2, r), generator=g, device=device).permute(2, 1, 0)
    Ph = torch.fft.rfft(P, dim=2).permute(2, 0, 1)          # h x n1 x r
    Qh = torch.fft.rfft(Q, dim=2).permute(2, 0, 1)          # h x r x n2
    h = Ph.shape[0]
    out = fortran_empty_torch(n1, n2, n3, device=device)
    # build the spectrum column-block by column-block to bound memory
    step = max(1, n2 // chunk)
    for j0 in range(0, n2, step):
        j1 = min(n2, j0 + step)
        Ch = torch.matmul(Ph, Qh[:, :, j0:j1])               # h x n1 x w
        X = torch.fft.irfft(Ch.permute(1, 2, 0), n=n3, dim=2)  # n1 x w x n3
        out[:, j0:j1, :] = X
        del Ch, X
    if noise:
        rms = (torch.linalg.vector_norm(out, dtype=torch.float64) / (out.numel() ** 0.5)).item()
        z = torch.randn((n3, n2, n1), generator=g, device=device).permute(2, 1, 0)
        out.add_(z, alpha=noise * rms)
        del z
    return out


def spectral_torch(n1, n2, n3, alpha, jitter, seed, device="cuda"):
    """Tensor with a prescribed spectrum at every Fourier frequency (the
    rank-predictor workload): X_hat_k = U_k diag(s_k) V_k^H with Haar-like
    unitary factors (QR of complex Gaussians; real orthogonal at the real
    frequencies k = 0 and, n3 even, k = n3/2) and s_{k,i} = i^(-a_k),
    a_k = alpha + jitter * u_k, u_k uniform in [-1, 1].  The transform back
    is torch.fft.irfft (the conjugate half is implied).  Returns the
    column-major real tensor and the exact spectra (h x min(n1, n2),
    float64, of X_hat_k as formed by the unnormalised forward transform)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    h, m = n3 // 2 + 1, min(n1, n2)
    a = alpha + jitter * (2.0 * torch.rand(h, generator=g, device=device, dtype=torch.float64) - 1.0)
    i = torch.arange(1, m + 1, device=device, dtype=torch.float64)
    s = i[None, :] ** (-a[:, None])                                     # h x m
    def factor(rows):
        re = torch.randn((h, rows, m), generator=g, device=device, dtype=torch.float64)
        im = torch.randn((h, rows, m), generator=g, device=device, dtype=torch.float64)
        im[0] = 0.0
        if n3 % 2 == 0:
            im[h - 1] = 0.0
        q, r = torch.linalg.qr(torch.complex(re, im))
        d = torch.diagonal(r, dim1=-2, dim2=-1)
        return q * (d / d.abs().clamp_min(1e-300)).conj()[:, None, :]   # unique phases
    U, V = factor(n1), factor(n2)
    Xh = (U * s[:, None, :].to(U.dtype)) @ V.conj().transpose(-1, -2)   # h x n1 x n2
    X = torch.fft.irfft(Xh, n=n3, dim=0)                                # n3 x n1 x n2, real
    out = fortran_empty_torch(n1, n2, n3, device=device)
    out.copy_(X.permute(1, 2, 0))
    return out, s
