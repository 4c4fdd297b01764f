"""Error of the three facewise-GEMM precisions against the float64 oracle as
the inner dimension grows (exact t-product, Algorithm 1), and on the shape of
the paper's tensor-multiplication experiment (its Table 1: U_r^T * U_r with
a long inner dimension n1), exactly and sampled (Algorithm 2).

The split forms round every operand to a hi + lo pair (3xTF32: 3 * 2^-22,
BF16x3: 3 * 2^-16 per real product in the worst case, a few 1e-6 root mean
square) and multiply on the tensor cores, whose float32 accumulators lose
accuracy with every update they absorb.  The kernel drains the accumulators
every 128 (tf32) or 256 (bf16) inner elements and adds the chunk sums in
float32 registers, so the error no longer grows with the inner dimension:
every form is held to the float32 tolerance 1e-5 at every K."""
import numpy as np
import pytest

import paper_1704_04362_gb300 as tp
from paper_1704_04362_gb300 import synth
from oracle import sampling_ref, tensor_ref
from tests.util import TOL_FP32, rel_fro, to_np

pytestmark = pytest.mark.gpu

NAMES = {tp.TP_FP32: "fp32", tp.TP_TF32X3: "tf32x3", tp.TP_BF16X3: "bf16x3"}


def dev(x):
    import torch
    return tp.as_tprod_layout(torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda())


@pytest.mark.parametrize("n2", [64, 512, 4096, 32768])
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
    for name, e in errs.items():
        assert e < TOL_FP32, (name, e)


def test_table1_shape_exact_and_sampled():
    """U^T * U for a 10^4 x 100 x 5 tensor U (the paper's experiment has
    n1 = 10^5 rows and r up to 500), exact (inner dimension 10^4) and with
    l = 460 slices drawn under the norm probabilities."""
    n1, r, n3, l = 10000, 100, 5, 460
    U = synth.iid_normal((n1, r, n3), seed=31) / np.sqrt(n1)
    Ut = tensor_ref.ttranspose(U.astype(np.float64)).astype(np.float32)
    ref = tensor_ref.tprod(Ut.astype(np.float64), U.astype(np.float64))
    Zref, ref_idx, _ = sampling_ref.tprod_sampled(Ut, U, l, 4)
    for prec in NAMES:
        C = tp.tprod(dev(Ut), dev(U), precision=prec)
        e = rel_fro(to_np(C), ref)
        Z, idx, cnt = tp.tprod_sampled(dev(Ut), dev(U), l, seed=4, precision=prec)
        assert np.array_equal(idx[: int(cnt.item())].cpu().numpy(), ref_idx)
        es = rel_fro(to_np(Z), Zref)
        print(f"{NAMES[prec]}: exact {e:.2e}, sampled (c' = {int(cnt.item())}) {es:.2e}")
        assert e < TOL_FP32 and es < TOL_FP32, (NAMES[prec], e, es)


@pytest.mark.parametrize("prec", [tp.TP_TF32X3, tp.TP_BF16X3])
def test_pipeline_wait_timeout_is_reported_and_recovered(prec):
    """Failure detection of the tensor-core GEMM: with the test hook's wait
    limit of one clock tick, the MMA warp's wait for the first loaded stage
    runs out; the kernel must flag TP_DEV_TIMEOUT, wait for the copies it
    issued and return, and the next call (default limit) must be correct."""
    import torch
    n1, n2, n4, n3 = 300, 1024, 200, 8
    A = synth.iid_normal((n1, n2, n3), seed=41)
    B = synth.iid_normal((n2, n4, n3), seed=42)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    tp.tprod(dev(A), dev(B), precision=prec, status=st, wait_limit=1)
    torch.cuda.synchronize()
    assert int(st.item()) & 0x4, "timeout not reported"
    st.zero_()
    C = tp.tprod(dev(A), dev(B), precision=prec, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    ref = tensor_ref.tprod(A.astype(np.float64), B.astype(np.float64))
    assert rel_fro(to_np(C), ref) < TOL_FP32
