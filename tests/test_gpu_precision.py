"""Error of the three facewise-GEMM precisions against the float64 oracle as
the inner dimension grows (exact t-product, Algorithm 1).

The split forms round every operand to a hi + lo pair and accumulate in the
tensor cores' float32 accumulators; their error is set by that accumulation
(it grows with the number of accumulator updates, about 6 per 8 tf32 or per 16
bf16 inner elements), while the plain FP32 form accumulates with fused
multiply-adds in registers.  The test prints the table and holds every form
to its tolerance: FP32 to 1e-5 at every K, the split forms to the bound of
split_tolerance (measured: 3xTF32 about 1.3e-8 K, BF16x3 about 4e-6 + 6e-9 K,
so both are within 1e-5 up to K of about 700 and 1000)."""
import numpy as np
import pytest

import paper_1704_04362_gb300 as tp
from paper_1704_04362_gb300 import synth
from oracle import tensor_ref
from tests.util import TOL_FP32, rel_fro, to_np

pytestmark = pytest.mark.gpu

NAMES = {tp.TP_FP32: "fp32", tp.TP_TF32X3: "tf32x3", tp.TP_BF16X3: "bf16x3"}


def split_tolerance(prec: int, K: int) -> float:
    """Bound of the relative error of a split form at inner dimension K: the
    operand split (3 * 2^-22 for tf32 hi + lo, 3 * 2^-16 for bf16 hi + lo) plus
    one float32 ulp (2^-23) lost at each accumulator update.  An output's
    real-part accumulator takes 6 updates per K step (three split products of
    Ar Br and of Ai Bi), and a K step is 8 tf32 or 16 bf16 elements."""
    rep = 3 * 2.0 ** -22 if prec == tp.TP_TF32X3 else 3 * 2.0 ** -16
    step = 8 if prec == tp.TP_TF32X3 else 16
    updates = 6 * -(-K // step)
    return rep + updates * 2.0 ** -23


def dev(x):
    import torch
    return tp.as_tprod_layout(torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda())


@pytest.mark.parametrize("n2", [64, 512, 4096])
def test_error_against_inner_dimension(n2):
    n1, n4, n3 = 48, 40, 8
    A = synth.iid_normal((n1, n2, n3), seed=11)
    B = synth.iid_normal((n2, n4, n3), seed=12)
    ref = tensor_ref.tprod(A.astype(np.float64), B.astype(np.float64))
    errs = {}
    for prec in NAMES:
        C = tp.tprod(dev(A), dev(B), precision=prec)
        errs[NAMES[prec]] = rel_fro(to_np(C), ref)
    print(f"K = {n2}: relative error " + ", ".join(f"{k} {v:.2e}" for k, v in errs.items()))
    assert errs["fp32"] < TOL_FP32
    for prec in (tp.TP_TF32X3, tp.TP_BF16X3):
        assert errs[NAMES[prec]] < split_tolerance(prec, n2)
