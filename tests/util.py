"""Shared helpers of the test suite (layout conversion, error measures)."""
import numpy as np


def to_np(x) -> np.ndarray:
    """Column-major torch tensor of logical shape (n1, n2, n3) -> float64 numpy."""
    return x.detach().permute(2, 1, 0).contiguous().cpu().numpy().astype(np.float64).transpose(2, 1, 0)


def rel_fro(a, b) -> float:
    """||a - b||_F / ||b||_F (0/0 -> 0); complex arguments keep their
    imaginary parts."""
    a = np.asarray(a)
    b = np.asarray(b)
    dt = np.complex128 if (np.iscomplexobj(a) or np.iscomplexobj(b)) else np.float64
    a = a.astype(dt)
    b = b.astype(dt)
    nb = np.linalg.norm(b)
    na = np.linalg.norm(a - b)
    if nb == 0:
        return float(na)
    return float(na / nb)


# relative Frobenius tolerance of every FP32 output against the float64 oracle
TOL_FP32 = 1e-5

# BF16x3 split (bf16 hi + bf16 lo, the lo*lo term dropped).  Each operand keeps
# 16 significand bits: |x - hi - lo| <= 2^-16 |x|, and the dropped lo*lo term
# is at most 2^-16 |x y|, so one real product is exact to 3 * 2^-16 = 4.6e-5
# relative in the worst case (about 5e-6 root-mean-square).  The tolerance is
# the worst-case bound plus the float32 transform and accumulation error.
TOL_BF16X3 = 5e-5


def tol_for(precision: int) -> float:
    """Relative Frobenius tolerance of a t-product output at this precision
    (0 FP32, 1 3xTF32, 2 BF16x3)."""
    return TOL_BF16X3 if precision == 2 else TOL_FP32


def golden(name):
    """Entries of a hand-worked fixture under tests/golden/: {key: [rows of
    numbers]} (lines "key numbers..."; '#' starts a comment line)."""
    import os
    out = {}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            out.setdefault(key, []).append([float(v) for v in vals])
    return out


def golden_tensor(rows, n1, n2, n3):
    """Tensor from fixture rows "slice row values..." (1-based slice and row)."""
    X = np.zeros((n1, n2, n3))
    for r in rows:
        X[int(r[1]) - 1, :, int(r[0]) - 1] = r[2:]
    return X
