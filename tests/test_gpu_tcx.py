"""GPU parity of t-CX (Algorithm 4 with the t-project of Algorithm 3)
against the float64 oracle, through the C ABI."""
import numpy as np
import pytest

import paper_1704_04362_gb300 as tp
from paper_1704_04362_gb300 import synth
from oracle import decomp_ref, tensor_ref
from tests.util import TOL_FP32, rel_fro, to_np

pytestmark = pytest.mark.gpu


def dev(x):
    return tp.as_tprod_layout(x)


@pytest.mark.parametrize("n1,n2,n3,c", [(20, 30, 6, 12), (40, 25, 7, 10), (8, 40, 5, 20),
                                        (16, 16, 1, 5), (64, 48, 16, 20)])
def test_tcx_matches_oracle(n1, n2, n3, c):
    import torch
    A = synth.iid_normal((n1, n2, n3), seed=n1 + n2)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    Z, idx, cnt = tp.tcx(dev(A), c, seed=9, status=st)
    assert int(st.item()) == 0
    Zr, ridx, q = decomp_ref.tcx(A, c, 9)
    assert np.array_equal(idx[: int(cnt.item())].cpu().numpy(), ridx)
    assert rel_fro(to_np(Z), Zr) < TOL_FP32


def test_tcx_least_squares_and_special_cases():
    import torch
    A = synth.lowrank_np(30, 40, 6, 2, seed=5)
    Z, idx, cnt = tp.tcx(dev(A), 12, seed=3)
    assert int(cnt.item()) >= 2
    assert rel_fro(to_np(Z), A.astype(np.float64)) < TOL_FP32     # rank 2 recovered
    B = synth.iid_normal((10, 12, 4), seed=6)
    Z, idx, cnt = tp.tcx(dev(B), 10 ** 6, seed=0)                  # every slice kept
    assert int(cnt.item()) == 12
    assert rel_fro(to_np(Z), B.astype(np.float64)) < TOL_FP32
    p = np.full(12, 1 / 12)
    Z, idx, cnt = tp.tcx(dev(B), 4, seed=2, prob_mode=tp.TP_PROB_GIVEN,
                         p_given=torch.from_numpy(p).cuda())
    Zr, ridx, _ = decomp_ref.tcx(B, 4, 2, mode=2, p_given=p)
    assert np.array_equal(idx[: int(cnt.item())].cpu().numpy(), ridx)
    assert rel_fro(to_np(Z), Zr) < TOL_FP32
    # Eq. ell2reg: no C * Y does better than the projection
    C = B.astype(np.float64)[:, ridx, :]
    best = np.linalg.norm(B - to_np(Z))
    for s in range(5):
        Yr = np.random.default_rng(s).standard_normal((len(ridx), 12, 4))
        assert np.linalg.norm(B - tensor_ref.tprod(C, Yr)) >= best * (1 - 1e-6)
