"""GPU parity of the t-product path against the float64 oracle (Algorithm 1,
Algorithm 2 and their stages), called through the C ABI."""
import numpy as np
import pytest

import paper_1704_04362_gb300 as tp
from paper_1704_04362_gb300 import synth
from oracle import philox_ref, sampling_ref, tensor_ref
from tests.util import TOL_FP32, rel_fro, to_np, tol_for

pytestmark = pytest.mark.gpu


def dev(x):
    return tp.as_tprod_layout(x)


@pytest.mark.parametrize("n3", [1, 2, 3, 4, 5, 8, 16, 17, 32, 64, 120, 128, 256, 257, 260, 512,
                                600, 1001, 2000, 4096])
def test_rdft_irdft_match_oracle(n3):
    X = synth.iid_normal((37, 5, n3), seed=n3)
    Xr, Xi = tp.rdft3(dev(X))
    ref = tensor_ref.half_spectrum(tensor_ref.fft3(X))
    scale = np.sqrt(n3)
    assert rel_fro(to_np(Xr) + 1j * to_np(Xi), ref) < TOL_FP32
    back = tp.irdft3(Xr, Xi, n3)
    assert rel_fro(to_np(back), X) < TOL_FP32
    # inverse alone against the oracle's inverse of the same spectrum
    Hr = synth.iid_normal((37, 5, n3 // 2 + 1), seed=100 + n3) * scale
    Hi = synth.iid_normal((37, 5, n3 // 2 + 1), seed=200 + n3) * scale
    Hi[:, :, 0] = 0
    if n3 % 2 == 0:
        Hi[:, :, -1] = 0
    out = tp.irdft3(dev(Hr), dev(Hi), n3)
    ref_inv = tensor_ref.ifft3(tensor_ref.hermitian_fill(Hr.astype(np.float64) + 1j * Hi, n3))
    assert np.max(np.abs(ref_inv.imag)) < 1e-9 * np.abs(ref_inv).max()
    assert rel_fro(to_np(out), ref_inv.real) < TOL_FP32


SHAPES = [
    (64, 48, 32, 16),     # the exact-product workload: A 64x48x16, B 48x32x16
    (1, 1, 1, 1),
    (3, 1, 2, 3),
    (5, 3, 7, 7),
    (130, 70, 67, 17),    # ragged against the 128 x 64 x 16 tiles
    (257, 33, 129, 2),
    (40, 200, 30, 64),
    (33, 20, 40, 128),    # power-of-two tube lengths: the register FFT
    (70, 37, 41, 32),
    (9, 8, 7, 4),
    (5, 6, 3, 8),
]


PRECISIONS = [tp.TP_FP32, tp.TP_TF32X3, tp.TP_BF16X3]


def status_word():
    import torch
    return torch.zeros(1, dtype=torch.int32, device="cuda")


@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("n1,n2,n4,n3", SHAPES)
def test_tprod_matches_oracle(n1, n2, n4, n3, prec):
    A = synth.iid_normal((n1, n2, n3), seed=1)
    B = synth.iid_normal((n2, n4, n3), seed=2)
    st = status_word()
    C = tp.tprod(dev(A), dev(B), precision=prec, status=st)
    ref = tensor_ref.tprod(A.astype(np.float64), B.astype(np.float64))
    assert int(st.item()) == 0
    assert rel_fro(to_np(C), ref) < tol_for(prec)


def test_tprod_identity_and_definition_tiny():
    A = synth.iid_normal((4, 3, 5), seed=3)
    I = tensor_ref.identity(3, 5).astype(np.float32)
    C = tp.tprod(dev(A), dev(I))
    assert rel_fro(to_np(C), A) < 1e-6
    B = synth.iid_normal((3, 2, 5), seed=4)
    assert rel_fro(to_np(tp.tprod(dev(A), dev(B))), tensor_ref.tprod_circ(A.astype(float), B.astype(float))) < TOL_FP32


@pytest.mark.parametrize("n1,n2,n3,which", [(2000, 40, 8, 0), (37, 41, 3, 0), (64, 48, 16, 1),
                                            (4000, 7, 5, 1), (1, 1, 1, 0), (3, 5, 2, 1)])
def test_slice_norms_match_oracle(n1, n2, n3, which):
    X = synth.iid_normal((n1, n2, n3), seed=5)
    got = tp.slice_norms(dev(X), which).cpu().numpy()
    ref = sampling_ref.lateral_norms_sq(X) if which == 0 else sampling_ref.horizontal_norms_sq(X)
    np.testing.assert_allclose(got, ref, rtol=1e-11)
    again = tp.slice_norms(dev(X), which).cpu().numpy()
    assert np.array_equal(got, again)   # deterministic


@pytest.mark.parametrize("n,c,seed", [(1, 1, 0), (5, 2, 1), (1000, 40, 7), (4000, 400, 0),
                                      (5000, 5000, 3), (70000, 100, 11)])
def test_draw_bit_exact_given_p(n, c, seed):
    import torch
    g = np.random.default_rng(seed)
    w = g.gamma(0.5, 1.0, n)
    p = w / w.sum()
    pt = torch.from_numpy(p).cuda()
    idx, scale, count, q = tp.sample_draw(pt, None, c, seed, tp.TP_PROB_GIVEN)
    cnt = int(count.item())
    ref_idx, ref_q = sampling_ref.draw(p, c, seed)
    assert cnt == len(ref_idx)
    assert np.array_equal(idx[:cnt].cpu().numpy(), ref_idx)
    assert np.array_equal(q.cpu().numpy(), ref_q)
    np.testing.assert_allclose(scale[:cnt].cpu().numpy(), 1 / np.sqrt(ref_q[ref_idx]), rtol=1e-7)


def test_draw_edge_cases():
    import torch
    # all-zero weights: nothing picked
    z = torch.zeros(10, dtype=torch.float64, device="cuda")
    idx, scale, count, q = tp.sample_draw(z, z, 3, 0, tp.TP_PROB_AB)
    assert int(count.item()) == 0
    # c p_j >= 1 everywhere: all picked, scale 1
    w = torch.ones(9, dtype=torch.float64, device="cuda")
    idx, scale, count, q = tp.sample_draw(w, None, 100, 0, tp.TP_PROB_A2)
    assert int(count.item()) == 9 and idx[:9].tolist() == list(range(9))
    assert torch.all(scale[:9] == 1)


@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("mode", [tp.TP_PROB_AB, tp.TP_PROB_A2])
@pytest.mark.parametrize("n1,n2,n4,n3,c", [(64, 48, 32, 16, 12), (50, 300, 41, 7, 60),
                                           (33, 130, 20, 64, 400), (20, 9, 5, 4, 1),
                                           (260, 500, 300, 8, 100), (70, 90, 45, 128, 30),
                                           (40, 64, 30, 32, 20), (17, 25, 9, 2, 10)])
def test_tprod_sampled_matches_oracle(mode, n1, n2, n4, n3, c, prec):
    A = synth.lowrank_np(n1, n2, n3, 4, seed=6, noise=0.01)
    B = synth.lowrank_np(n2, n4, n3, 4, seed=7, noise=0.01)
    st = status_word()
    Z, idx, count = tp.tprod_sampled(dev(A), dev(B), c, seed=123, prob_mode=mode,
                                     precision=prec, status=st)
    assert int(st.item()) == 0
    cnt = int(count.item())
    Zref, ref_idx, q = sampling_ref.tprod_sampled(A, B, c, 123, mode=mode)
    # index draws: the float64 probabilities agree to rounding, so the picks agree
    assert np.array_equal(idx[:cnt].cpu().numpy(), ref_idx)
    assert rel_fro(to_np(Z), Zref) < tol_for(prec)


def test_tprod_sampled_given_p_and_nothing_kept():
    import torch
    A = synth.iid_normal((10, 12, 6), seed=8)
    B = synth.iid_normal((12, 7, 6), seed=9)
    p = np.full(12, 1 / 12)
    Z, idx, count = tp.tprod_sampled(dev(A), dev(B), 3, seed=5, prob_mode=tp.TP_PROB_GIVEN,
                                     p_given=torch.from_numpy(p).cuda())
    Zref, ref_idx, _ = sampling_ref.tprod_sampled(A, B, 3, 5, mode=sampling_ref.PROB_GIVEN, p_given=p)
    assert np.array_equal(idx[:int(count.item())].cpu().numpy(), ref_idx)
    assert rel_fro(to_np(Z), Zref) < TOL_FP32
    Z0, _, c0 = tp.tprod_sampled(dev(np.zeros_like(A)), dev(B), 3, seed=5)
    assert int(c0.item()) == 0 and float(Z0.abs().max()) == 0.0


@pytest.mark.parametrize("n,c,seed", [(1, 1, 0), (7, 5, 1), (1000, 300, 2), (5000, 4096, 3),
                                      (70000, 1000, 4)])
def test_iid_draw_bit_exact_given_p(n, c, seed):
    import torch
    g = np.random.default_rng(seed)
    w = g.gamma(0.5, 1.0, n)
    w[g.random(n) < 0.2] = 0.0                     # zero weights are never drawn
    if w.sum() == 0:
        w[0] = 1.0
    p = w / w.sum()
    pt = torch.from_numpy(p).cuda()
    idx, scale, count, q = tp.sample_draw(pt, None, c, seed, tp.TP_PROB_GIVEN,
                                          sample_mode=tp.TP_SAMPLE_IID)
    ref_idx, ref_s = sampling_ref.draw_iid(p, c, seed)
    assert int(count.item()) == c == len(ref_idx)
    assert np.array_equal(idx[:c].cpu().numpy(), ref_idx)
    np.testing.assert_allclose(scale[:c].cpu().numpy(), 1 / np.sqrt(ref_s), rtol=1e-7)
    np.testing.assert_allclose(q.cpu().numpy(), c * p, rtol=1e-15)
    # the norm modes draw the oracle's indices from the same weights
    wt = torch.from_numpy(w).cuda()
    idx2, _, count2, _ = tp.sample_draw(wt, None, c, seed, tp.TP_PROB_A2,
                                        sample_mode=tp.TP_SAMPLE_IID)
    ref2, _ = sampling_ref.draw_iid(sampling_ref.probabilities(w, None, sampling_ref.PROB_A2), c, seed)
    assert np.array_equal(idx2[:c].cpu().numpy(), ref2)


def test_iid_draw_edge_cases():
    import torch
    z = torch.zeros(10, dtype=torch.float64, device="cuda")
    idx, scale, count, q = tp.sample_draw(z, z, 3, 0, tp.TP_PROB_AB, sample_mode=tp.TP_SAMPLE_IID)
    assert int(count.item()) == 0
    one = torch.zeros(10, dtype=torch.float64, device="cuda")
    one[6] = 1.0
    idx, scale, count, q = tp.sample_draw(one, None, 10, 5, tp.TP_PROB_GIVEN,
                                          sample_mode=tp.TP_SAMPLE_IID)
    assert int(count.item()) == 10 and idx.tolist() == [6] * 10
    assert torch.allclose(scale, torch.full_like(scale, 10 ** -0.5))
    with pytest.raises(tp.TprodError):
        tp.sample_draw(one, None, 11, 5, tp.TP_PROB_GIVEN, sample_mode=tp.TP_SAMPLE_IID)


@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("n1,n2,n4,n3,c", [(64, 48, 32, 16, 12), (50, 300, 41, 7, 60),
                                           (33, 130, 20, 64, 130), (260, 500, 300, 8, 100)])
def test_tprod_sampled_iid_matches_oracle(n1, n2, n4, n3, c, prec):
    A = synth.lowrank_np(n1, n2, n3, 4, seed=16, noise=0.01)
    B = synth.lowrank_np(n2, n4, n3, 4, seed=17, noise=0.01)
    st = status_word()
    Z, idx, count = tp.tprod_sampled(dev(A), dev(B), c, seed=321, precision=prec, status=st,
                                     sample_mode=tp.TP_SAMPLE_IID)
    assert int(st.item()) == 0 and int(count.item()) == c
    Zref, ref_idx, _ = sampling_ref.tprod_sampled(A, B, c, 321, sample=sampling_ref.SAMPLE_IID)
    assert np.array_equal(idx[:c].cpu().numpy(), ref_idx)
    assert rel_fro(to_np(Z), Zref) < tol_for(prec)


def test_hand_worked_fixtures_on_the_device():
    # tests/golden: the t-product of Def. 2.1 worked by hand (2 x 2 x 2 and
    # the tube (1,2,3) * (4,5,6) = (31,31,28)), through the C ABI
    from tests.util import golden, golden_tensor
    g = golden("tprod_2x2x2_by_hand.txt")
    A, B, C = (golden_tensor(g[k], 2, 2, 2).astype(np.float32) for k in ("A", "B", "C"))
    for prec in PRECISIONS:
        Z = tp.tprod(dev(A), dev(B), precision=prec)
        np.testing.assert_allclose(to_np(Z), C, atol=1e-5)
    t = golden("tube_1x1x3_by_hand.txt")
    a = np.array([1, 2, 3], dtype=np.float32).reshape(1, 1, 3)
    b = np.array([4, 5, 6], dtype=np.float32).reshape(1, 1, 3)
    np.testing.assert_allclose(to_np(tp.tprod(dev(a), dev(b))).ravel(), t["prod"][0], rtol=1e-6)
