"""GPU parity of the per-frequency truncation-rank calls against the float64
oracle, through the C ABI: sketch spectra (the randomized t-SVD's core
singular values), the plain rank rule (bit-exact on the same spectra), the
predictor's features, and the predictor network's forward pass, gradient
and Adam step."""
import numpy as np
import pytest

import paper_1704_04362_gb300 as tp
from paper_1704_04362_gb300 import synth
from oracle import decomp_ref, learned_ref as R, philox_ref
from tests.util import TOL_FP32, rel_fro

pytestmark = pytest.mark.gpu


def cuda(x, dtype=None):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to(dtype or torch.float32).cuda()


@pytest.mark.parametrize("n1,n2,n3,l,q", [(40, 30, 6, 17, 1), (64, 48, 16, 24, 2), (33, 50, 5, 17, 0)])
def test_sketch_spectrum_matches_oracle(n1, n2, n3, l, q):
    # a smoothly decaying spectrum (no noise-level tail): every value is determined
    X = synth.lowrank_np(n1, n2, n3, min(n1, n2), seed=21, factor="normal")
    sig = tp.sketch_spectrum(tp.as_tprod_layout(X), l, q, seed=4).cpu().numpy()
    Om = philox_ref.sketch_signs(n2, l, n3 // 2 + 1, n3, 4)
    _, s_ref, _ = decomp_ref.tsvd_randomized_hat(X.astype(np.float64), l, 0, q, Om)
    assert sig.shape == (n3 // 2 + 1, l)
    assert np.all(np.diff(sig, axis=1) <= 0)
    assert rel_fro(sig, s_ref.T) < TOL_FP32


def test_rank_rule_is_bit_exact():
    g = np.random.default_rng(5)
    h, l = 300, 50
    alpha = g.uniform(0.5, 4.0, size=(h, 1))
    sig = (np.arange(1, l + 1)[None, :] ** -alpha) * g.uniform(0.5, 2.0, size=(h, 1))
    sig = np.sort(sig.astype(np.float32), axis=1)[:, ::-1].copy()
    sig[7] = 0.0                                              # a zero slice
    sig[8, 3:] = 0.0                                          # an exact rank-3 slice
    for tol, cap in ((1e-2, 40), (5e-2, 40), (1e-1, 10), (0.0, 50)):
        got = tp.rank_rule(cuda(sig), cap, tol).cpu().numpy()
        ref = R.rank_rule(sig.astype(np.float64), tol, cap)
        assert np.array_equal(got, ref), (tol, cap)
    assert tp.rank_rule(cuda(sig), 40, 1e-2).cpu().numpy()[7] == 0


def test_features_match_oracle():
    g = np.random.default_rng(6)
    sig = np.sort(g.random((40, 20)).astype(np.float32) ** 3, axis=1)[:, ::-1].copy()
    sig[3, 5:] = 0.0
    f = tp.rank_features(cuda(sig)).float().cpu().numpy()
    ref = R.features(sig.astype(np.float64))
    assert np.max(np.abs(f - ref)) < 1e-3                     # float16 rounding of values in [-1, 0]


def network_case(B, seed):
    import torch
    g = np.random.default_rng(seed)
    theta = (0.2 * g.standard_normal(R.N_PARAMS)).astype(np.float32)
    X16 = g.uniform(-1, 0, size=(B, R.N_IN)).astype(np.float16)
    T = g.uniform(0, 1, size=(B, R.N_OUT)).astype(np.float32)
    th = cuda(theta)
    w16 = tp.mlp_round(th)
    return theta, X16, T, th, w16, cuda(X16, torch.float16), cuda(T)


@pytest.mark.parametrize("B", [1, 63, 1000])
def test_forward_and_gradient_match_oracle(B):
    import torch
    theta, X16, T, th, w16, x, t = network_case(B, B)
    theta16 = R.as_f16(theta)                                 # the weights the kernels use
    assert np.array_equal(w16.cpu().numpy(), theta.astype(np.float16))
    y = tp.mlp_forward(w16, x).cpu().numpy()
    y_ref, _, _ = R.forward(theta16, X16.astype(np.float64))
    assert rel_fro(y, y_ref) < 1e-5
    m = torch.zeros_like(th)
    v = torch.zeros_like(th)
    grad = tp.mlp_train_step(th, w16, m, v, 1, 0.0, x, t).cpu().numpy()
    loss_ref, g_ref = R.loss_and_grad(theta16, X16.astype(np.float64), T.astype(np.float64))
    assert abs(grad[-1] - loss_ref) <= 1e-5 * loss_ref
    for a, b in ((0, 2048), (2048, 2176), (2176, 18560), (18560, 18688), (18688, 18944), (18944, 18946)):
        assert rel_fro(grad[a:b], g_ref[a:b]) < 1e-5, (a, b)
    # deterministic: the same call gives the same bits
    grad2 = tp.mlp_train_step(th, w16, m, v, 1, 0.0, x, t).cpu().numpy()
    assert np.array_equal(grad, grad2)


def test_adam_step_matches_oracle():
    import torch
    theta, X16, T, th, w16, x, t = network_case(500, 9)
    m = torch.zeros_like(th)
    v = torch.zeros_like(th)
    th0 = th.clone()
    grad = tp.mlp_train_step(th, w16, m, v, 1, 1e-3, x, t)
    g = grad[:-1].double().cpu().numpy()
    ref, m_ref, v_ref = R.adam_step(th0.double().cpu().numpy(), 0.0, 0.0, g, 1, 1e-3)
    assert np.max(np.abs(th.double().cpu().numpy() - ref)) < 1e-6
    assert rel_fro(m.cpu().numpy(), m_ref) < 1e-6 and rel_fro(v.cpu().numpy(), v_ref) < 1e-5
    assert np.array_equal(w16.cpu().numpy(), th.cpu().numpy().astype(np.float16))
    # a second step from the updated moments
    th1 = th.double().cpu().numpy()
    grad2 = tp.mlp_train_step(th, w16, m, v, 2, 1e-3, x, t)
    ref2, _, _ = R.adam_step(th1, m_ref, v_ref, grad2[:-1].double().cpu().numpy(), 2, 1e-3)
    assert np.max(np.abs(th.double().cpu().numpy() - ref2)) < 1e-6
