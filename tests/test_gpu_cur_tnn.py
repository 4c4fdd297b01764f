"""GPU parity of CUR t-NN (Algorithm 6) against the float64 oracle, through
the C ABI.  Lateral picks are compared bit for bit; the top-r row leverage of
C within tolerance and the horizontal picks bit for bit against the oracle's
draw on the device's probabilities.  The two ADMM results C~ and R~ carry
the float32 state of many iterations (compared as the robust ADMM is, within
1e-4); the last step, C~ (S^T C~)^dagger R~, is compared with the oracle's on
the device's own C~ and R~ within the float32 tolerance scaled by the
condition number of the intersection W~."""
import numpy as np
import pytest

import paper_1704_04362_gb300 as tp
from paper_1704_04362_gb300 import synth
from oracle import completion_ref, decomp_ref, philox_ref, sampling_ref
from tests.util import TOL_FP32, rel_fro, to_np

pytestmark = pytest.mark.gpu
TOL_ADMM = 1e-4       # float32 ADMM state over tens of iterations


def dev(x, dtype=None):
    return tp.as_tprod_layout(x, dtype) if dtype is not None else tp.as_tprod_layout(x)


def t_np(x):
    return x.detach().double().cpu().numpy()


def low_rank_plus_sparse(n1, n2, n3, r, seed, frac=0.05):
    L0 = synth.lowrank_np(n1, n2, n3, r, seed=seed).astype(np.float64)
    L0 /= np.sqrt(np.mean(L0 ** 2))
    g = np.random.default_rng(seed + 1)
    S0 = np.where(g.random(L0.shape) < frac, 10.0 * g.standard_normal(L0.shape), 0.0)
    return L0, (L0 + S0).astype(np.float32)


def intersection_condition(Ct, ridx, rtol):
    """Largest ratio s_max / s_min over the kept singular values of the Fourier
    slices of W~ = C~(ridx, :, :)."""
    W = np.fft.fft(Ct[ridx, :, :], axis=2)
    kappa = 1.0
    for f in range(W.shape[2]):
        s = np.linalg.svd(W[:, :, f], compute_uv=False)
        s = s[s > rtol * s[0]]
        kappa = max(kappa, s[0] / s[-1])
    return kappa


def check(X, c, l, iters, r, seed, mask=None, **kw):
    import torch
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    md = dev(mask, torch.uint8) if mask is not None else None
    L, Ct, Rt, ci, cc, ri, rc, pr = tp.cur_tnn(dev(X), c, l, iters, seed=seed, rank=r, mask=md,
                                               status=st, **kw)
    assert int(st.item()) == 0
    cidx = ci[: int(cc.item())].cpu().numpy()
    ridx = ri[: int(rc.item())].cpu().numpy()
    p_dev = pr.cpu().numpy()
    Lr, Ctr, Rtr, cref, rref, pref = decomp_ref.cur_tnn(X, c, l, seed, iters, r=r, mask=mask,
                                                        p_rows=p_dev)
    assert np.array_equal(cidx, cref)
    Xo = X.astype(np.float64) if mask is None else np.where(mask, X, 0.0)
    assert rel_fro(p_dev, decomp_ref.row_leverage(Xo[:, cidx, :], r)) < TOL_FP32
    want, _ = sampling_ref.draw(p_dev, l, seed, philox_ref.STREAM_HORIZONTAL)
    assert np.array_equal(ridx, want) and np.array_equal(rref, ridx)
    ct, rt = t_np(Ct), t_np(Rt)
    e_c, e_r = rel_fro(ct, Ctr), rel_fro(rt, Rtr)
    # the last step on the device's own C~ and R~
    rtol = kw.get("pinv_rtol", 1e-4)
    kappa = intersection_condition(ct, ridx, rtol)
    e_comb = rel_fro(to_np(L), decomp_ref.cur_combine(ct, rt, ridx, rtol))
    e_all = rel_fro(to_np(L), Lr)
    print(f"cur_tnn {X.shape} c'={len(cidx)} l'={len(ridx)}: C~ {e_c:.1e} R~ {e_r:.1e} "
          f"combine {e_comb:.1e} (kappa {kappa:.1f}) all {e_all:.1e}")
    assert e_c < TOL_ADMM and e_r < TOL_ADMM
    assert e_comb < TOL_FP32 * max(1.0, kappa)
    assert e_all < TOL_ADMM * max(1.0, kappa)
    return L, cidx, ridx


@pytest.mark.parametrize("n1,n2,n3,c,l,r", [(40, 36, 6, 16, 20, 3), (30, 64, 5, 20, 18, 2),
                                            (48, 40, 8, 30, 12, 2)])
def test_cur_tnn_robust_matches_oracle(n1, n2, n3, c, l, r):
    L0, X = low_rank_plus_sparse(n1, n2, n3, r, seed=n1 + n2)
    check(X, c, l, 40, r, seed=n3)


def test_cur_tnn_completion_matches_oracle():
    L0 = synth.lowrank_np(36, 40, 8, 3, seed=81).astype(np.float64)
    mask = np.random.default_rng(82).random(L0.shape) < 0.6
    check(L0.astype(np.float32), 18, 20, 40, 3, seed=2, mask=mask)


def test_cur_tnn_recovers_low_rank_plus_sparse():
    L0, X = low_rank_plus_sparse(96, 80, 8, 3, seed=83)
    L, *_ = tp.cur_tnn(dev(X), 30, 36, 100, seed=1, rank=3)
    err = rel_fro(to_np(L), L0)
    print(f"cur_tnn recovery 96x80x8 rank 3 + 5% spikes: {err:.2e}")
    assert err < 1e-3


def test_cur_tnn_special_cases():
    import torch
    # every slice kept: L~ = C~ C~^dagger C~ = the full robust ADMM
    L0, X = low_rank_plus_sparse(20, 16, 4, 2, seed=84)
    L, Ct, Rt, ci, cc, ri, rc, pr = tp.cur_tnn(dev(X), 10 ** 6, 10 ** 6, 20, seed=0,
                                               pinv_rtol=0.0)
    assert int(cc.item()) == 16 and int(rc.item()) == 20
    full = tp.trpca_admm(dev(X), 20)[0]
    assert rel_fro(t_np(Ct), to_np(full)) < 1e-6      # the same kernels, the same iterations
    assert rel_fro(to_np(L), to_np(full)) < TOL_ADMM
    # a zero tensor picks nothing: L = 0
    O = np.zeros((8, 6, 3), dtype=np.float32)
    L, Ct, Rt, ci, cc, ri, rc, pr = tp.cur_tnn(dev(O), 4, 4, 5, seed=1)
    assert int(cc.item()) == 0 and int(rc.item()) == 0
    assert float(torch.abs(L).max().item()) == 0.0
