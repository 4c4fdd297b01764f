"""Parity at the full benchmark size, in the configuration bench.py times:
rt-product of A 2000 x 4000 x 64 and B 4000 x 1500 x 64 (tubal rank 20 plus 1%
noise), c = 400.  The oracle recomputes the slice norms and the draw from the
same inputs (indices must agree exactly) and then a sample of output tubes one
by one; the outputs of all three precisions (FP32, 3xTF32, BF16x3) must match
them within 1e-5 (the split forms' accumulation error grows with the number of
picked slices, c' = 426 here; see test_gpu_precision.py)."""
import numpy as np
import pytest

import paper_1704_04362_gb300 as tp
from paper_1704_04362_gb300 import synth
from oracle import sampling_ref, tensor_ref
from tests.util import TOL_FP32

pytestmark = pytest.mark.gpu

N1, N2, N4, N3, C = 2000, 4000, 1500, 64, 400


def host(x):
    return x.permute(2, 1, 0).contiguous().cpu().numpy().transpose(2, 1, 0)


@pytest.fixture(scope="module")
def workload():
    A = synth.lowrank_torch(N1, N2, N3, 20, seed=1000, noise=0.01)
    B = synth.lowrank_torch(N2, N4, N3, 20, seed=2000, noise=0.01)
    return A, B


def test_fullsize_sampled_product_tubes(workload):
    import torch
    A, B = workload
    outs = {}
    for prec in (tp.TP_FP32, tp.TP_TF32X3, tp.TP_BF16X3):
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        Z, idx, cnt = tp.tprod_sampled(A, B, C, seed=0, precision=prec, status=st)
        assert int(st.item()) == 0
        outs[prec] = (Z, idx[: int(cnt.item())].cpu().numpy())
    Ah = host(A)
    Bh = host(B)
    a2 = sampling_ref.lateral_norms_sq(Ah)
    b2 = sampling_ref.horizontal_norms_sq(Bh)
    p = sampling_ref.probabilities(a2, b2, sampling_ref.PROB_AB)
    ref_idx, q = sampling_ref.draw(p, C, 0)
    for prec, (Z, gidx) in outs.items():
        assert np.array_equal(gidx, ref_idx), f"draws differ for precision {prec}"
    s = 1.0 / np.sqrt(q[ref_idx])
    rng = np.random.default_rng(5)
    pairs = [(0, 0), (N1 - 1, N4 - 1)] + [(int(rng.integers(N1)), int(rng.integers(N4)))
                                          for _ in range(14)]
    num = {prec: 0.0 for prec in outs}
    den = 0.0
    for i, l in pairs:
        Ci = (Ah[i:i + 1, ref_idx, :].astype(np.float64) * s[None, :, None])
        Rl = (Bh[ref_idx, l:l + 1, :].astype(np.float64) * s[:, None, None])
        tube = tensor_ref.tprod(Ci, Rl)[0, 0, :]
        den += float(np.sum(tube ** 2))
        for prec, (Z, _) in outs.items():
            g = Z[i, l, :].double().cpu().numpy()
            num[prec] += float(np.sum((g - tube) ** 2))
    errs = {prec: np.sqrt(num[prec] / den) for prec in outs}
    print("relative error on sampled tubes by precision:", {k: f"{v:.2e}" for k, v in errs.items()})
    for prec, err in errs.items():
        assert err < TOL_FP32, f"precision {prec}: relative error {err:.2e} on sampled tubes"
