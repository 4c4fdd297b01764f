"""Shared helpers of the test suite (layout conversion, error measures)."""
import numpy as np


def to_np(x) -> np.ndarray:
    """Column-major torch tensor of logical shape (n1, n2, n3) -> float64 numpy."""
    return x.detach().permute(2, 1, 0).contiguous().cpu().numpy().astype(np.float64).transpose(2, 1, 0)


def rel_fro(a, b) -> float:
    """||a - b||_F / ||b||_F (0/0 -> 0)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    na = np.linalg.norm(a - b)
    if nb == 0:
        return float(na)
    return float(na / nb)


# relative Frobenius tolerance of every FP32 output against the float64 oracle
TOL_FP32 = 1e-5
