"""GPU parity of t-CUR (Algorithm 5) against the float64 oracle, through the
C ABI.  The lateral picks depend only on the input and the Philox coins, so
they are compared bit for bit.  The row leverage probabilities come from the
SVD of the float32 transform of C, so they are compared within tolerance.  The
horizontal picks are then compared bit for bit against the oracle's draw on
the device's probabilities (the decision u < min{1, l p_i} taken on the same
float64 p_i), and Z against the oracle's t-CUR with those probabilities."""
import numpy as np
import pytest

import paper_1704_04362_gb300 as tp
from paper_1704_04362_gb300 import synth
from oracle import decomp_ref, philox_ref, sampling_ref
from tests.util import TOL_FP32, rel_fro, to_np

pytestmark = pytest.mark.gpu


def dev(x):
    return tp.as_tprod_layout(x)


def check_against_oracle(A, c, l, seed, **kw):
    import torch
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    Z, ci, cc, ri, rc, pr = tp.tcur(dev(A), c, l, seed=seed, status=st, **kw)
    assert int(st.item()) == 0
    cidx = ci[: int(cc.item())].cpu().numpy()
    ridx = ri[: int(rc.item())].cpu().numpy()
    p_dev = pr.cpu().numpy()
    mode = kw.get("prob_mode", sampling_ref.PROB_A2)
    pc = kw["p_cols"].cpu().numpy() if "p_cols" in kw else None
    _, cref, _, pref = decomp_ref.tcur(A, c, l, seed, mode=mode, p_cols=pc,
                                       p_rows=kw["p_rows"].cpu().numpy() if "p_rows" in kw else None)
    assert np.array_equal(cidx, cref)
    assert rel_fro(p_dev, pref) < TOL_FP32
    want, _ = sampling_ref.draw(p_dev, l, seed, philox_ref.STREAM_HORIZONTAL)
    assert np.array_equal(ridx, want)
    Zr, _, ridx_r, _ = decomp_ref.tcur(A, c, l, seed, mode=mode, p_cols=pc, p_rows=p_dev)
    assert np.array_equal(ridx_r, ridx)
    err = rel_fro(to_np(Z), Zr)
    print(f"tcur {A.shape} c={c} l={l}: c'={len(cidx)} l'={len(ridx)} rel err {err:.2e}")
    assert err < TOL_FP32
    return Z, cidx, ridx


# n1 >= c' and n1 < c' (the leverage SVD transposed), l' >= c' and l' < c'
# (the pseudo-inverse's SVD transposed), odd and even n3, n3 = 1
@pytest.mark.parametrize("n1,n2,n3,c,l", [(40, 30, 6, 8, 24), (20, 40, 7, 30, 16),
                                          (64, 48, 16, 12, 8), (33, 50, 5, 10, 33),
                                          (16, 16, 1, 5, 12), (96, 128, 32, 20, 60)])
def test_tcur_matches_oracle(n1, n2, n3, c, l):
    A = synth.iid_normal((n1, n2, n3), seed=n1 + n2 + n3)
    check_against_oracle(A, c, l, seed=n3)


def test_tcur_given_probabilities():
    import torch
    A = synth.iid_normal((30, 24, 8), seed=71)
    pc = torch.full((24,), 1 / 24, dtype=torch.float64, device="cuda")
    g = np.random.default_rng(72).random(30)
    pr = torch.from_numpy(g / g.sum()).cuda()
    _, _, ridx = check_against_oracle(A, 10, 14, 5, prob_mode=tp.TP_PROB_GIVEN, p_cols=pc,
                                      p_rows=pr)
    assert len(ridx) > 0


def test_tcur_special_cases():
    import torch
    # every slice kept: W = A's slice itself, Z = A
    B = synth.iid_normal((12, 10, 4), seed=73)
    Z, ci, cc, ri, rc, pr = tp.tcur(dev(B), 10 ** 6, 10 ** 6, seed=0)
    assert int(cc.item()) == 10 and int(rc.item()) == 12
    assert rel_fro(to_np(Z), B.astype(np.float64)) < TOL_FP32
    assert abs(float(pr.sum().item()) - 1.0) < 1e-12
    # low tubal rank: rank-3 lateral and horizontal picks reproduce A
    A = synth.lowrank_np(48, 40, 8, 3, seed=74)
    Z, ci, cc, ri, rc, pr = tp.tcur(dev(A), 16, 24, seed=2)
    err = rel_fro(to_np(Z), A.astype(np.float64))
    print(f"tcur low tubal rank 3: c'={int(cc.item())} l'={int(rc.item())} rel err {err:.2e}")
    assert int(cc.item()) >= 3 and int(rc.item()) >= 3
    assert err < 1e-4
    # a zero tensor picks nothing: Z = 0, no rows, zero probabilities
    O = np.zeros((8, 6, 3), dtype=np.float32)
    Z, ci, cc, ri, rc, pr = tp.tcur(dev(O), 4, 4, seed=1)
    assert int(cc.item()) == 0 and int(rc.item()) == 0
    assert float(torch.abs(Z).max().item()) == 0.0 and float(pr.abs().max().item()) == 0.0
    # given row probabilities that are all zero: no rows, Z = 0
    zr = torch.zeros(8, dtype=torch.float64, device="cuda")
    C = synth.iid_normal((8, 6, 3), seed=75)
    Z, ci, cc, ri, rc, pr = tp.tcur(dev(C), 4, 4, seed=1, p_rows=zr)
    assert int(cc.item()) > 0 and int(rc.item()) == 0
    assert float(torch.abs(Z).max().item()) == 0.0


@pytest.mark.parametrize("n1,n2,n3,c,l,r", [(40, 30, 6, 12, 24, 3), (20, 40, 7, 30, 16, 2)])
def test_tcur_top_r_leverage_matches_oracle(n1, n2, n3, c, l, r):
    # low tubal rank r plus noise: the top r directions are well separated
    A = synth.lowrank_np(n1, n2, n3, r, seed=n1 * r, noise=0.05)
    import torch
    Z, ci, cc, ri, rc, pr = tp.tcur(dev(A), c, l, seed=4, rank=r)
    cidx = ci[: int(cc.item())].cpu().numpy()
    ridx = ri[: int(rc.item())].cpu().numpy()
    p_dev = pr.cpu().numpy()
    _, cref, _, pref = decomp_ref.tcur(A, c, l, 4, r=r)
    assert np.array_equal(cidx, cref)
    assert rel_fro(p_dev, pref) < TOL_FP32
    want, _ = sampling_ref.draw(p_dev, l, 4, philox_ref.STREAM_HORIZONTAL)
    assert np.array_equal(ridx, want)
    Zr, *_ = decomp_ref.tcur(A, c, l, 4, p_rows=p_dev)
    assert rel_fro(to_np(Z), Zr) < TOL_FP32
