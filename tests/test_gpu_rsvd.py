"""GPU parity of the randomized low-tubal-rank t-SVD against the float64
oracle (same random-sign test matrix, drawn from Philox on both sides).

The rank-k result is unique only where the spectrum has a gap after k, so
the comparisons are: singular values and the approximation U * S * V^T where
the rank-k truncation is well defined (exact low rank, or a clear gap), and
for the mass-spectrometry-shaped workload (k = 40 over a rank-15 signal plus
noise, no gap at 40) the signal singular values, the approximation error and
the orthogonality of the factors."""
import numpy as np
import pytest

import paper_1704_04362_gb300 as tp
from paper_1704_04362_gb300 import synth
from oracle import decomp_ref, philox_ref, tensor_ref
from tests.util import TOL_FP32, rel_fro, to_np

pytestmark = pytest.mark.gpu


def dev(x):
    return tp.as_tprod_layout(x)


def sing_vals(S):
    Sh = tensor_ref.half_spectrum(tensor_ref.fft3(S))
    return np.stack([np.diag(Sh[:, :, f]).real for f in range(Sh.shape[2])], axis=1)


def approx(U, S, V):
    return tensor_ref.tprod(tensor_ref.tprod(U, S), tensor_ref.ttranspose(V))


PRECISIONS = [tp.TP_FP32, tp.TP_TF32X3, tp.TP_BF16X3]


def run_both(X, k, p, q, seed, precision=tp.TP_FP32):
    import torch
    n1, n2, n3 = X.shape
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    U, S, V = tp.tsvd_randomized(dev(X), k, p, q, seed=seed, status=st, precision=precision)
    assert int(st.item()) == 0
    h = n3 // 2 + 1
    Om = philox_ref.sketch_signs(n2, k + p, h, n3, seed)
    ref = decomp_ref.tsvd_randomized(X.astype(np.float64), k, p, q, Om)
    return (to_np(U), to_np(S), to_np(V)), ref


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("n1,n2,n3,r,k,p,q", [(40, 30, 6, 3, 4, 3, 1), (30, 40, 7, 2, 3, 2, 0),
                                              (64, 48, 16, 5, 6, 4, 2), (20, 20, 1, 4, 5, 5, 1),
                                              # more than 256 rows: CholeskyQR2 in global memory
                                              (300, 40, 4, 3, 4, 3, 1), (40, 300, 5, 3, 4, 4, 1),
                                              # the Householder variants' row counts (64, 65,
                                              # 129, 256 rows) and a one-column sketch
                                              (64, 65, 3, 2, 3, 3, 1), (129, 256, 2, 4, 5, 3, 1),
                                              (256, 70, 3, 5, 6, 2, 2), (12, 9, 5, 1, 1, 0, 1)])
def test_exact_low_rank_is_recovered(n1, n2, n3, r, k, p, q, precision):
    X = synth.lowrank_np(n1, n2, n3, r, seed=7)
    (U, S, V), (Ur, Sr, Vr) = run_both(X, k, p, q, seed=3, precision=precision)
    assert rel_fro(approx(U, S, V), X.astype(np.float64)) < TOL_FP32
    s, sr = sing_vals(S), sing_vals(Sr)
    assert rel_fro(s[:r], sr[:r]) < TOL_FP32
    assert np.all(s[r:] < 1e-4 * s[0])


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("n3", [16, 2000])
def test_gap_case_matches_oracle(n3, precision):
    X = synth.lowrank_np(48, 36, n3, 5, seed=11, noise=1e-4)
    (U, S, V), (Ur, Sr, Vr) = run_both(X, 5, 5, 2, seed=1, precision=precision)
    assert rel_fro(sing_vals(S), sing_vals(Sr)) < TOL_FP32
    assert rel_fro(approx(U, S, V), approx(Ur, Sr, Vr)) < TOL_FP32
    I = tensor_ref.identity(5, n3)
    assert np.linalg.norm(tensor_ref.tprod(tensor_ref.ttranspose(U), U) - I) < 1e-4
    assert np.linalg.norm(tensor_ref.tprod(tensor_ref.ttranspose(V), V) - I) < 1e-4


@pytest.fixture(scope="module")
def msi_oracle():
    X = synth.msi_like_np()
    k, p, q = 40, 10, 2
    Om = philox_ref.sketch_signs(128, k + p, 1001, 2000, 0)
    return X, decomp_ref.tsvd_randomized(X.astype(np.float64), k, p, q, Om)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_msi_workload_full_size(msi_oracle, precision):
    """128 x 128 pixels x 2000 channels, Gamma(2,1) factors at tubal rank 15,
    sparse positive spikes and 0.5% noise; k = 40, oversampling 10, 2 power
    iterations; the plain FP32 form and both split tensor-core forms."""
    import torch
    X, (Ur, Sr, Vr) = msi_oracle
    k, p, q = 40, 10, 2
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    U, S, V = tp.tsvd_randomized(dev(X), k, p, q, seed=0, status=st, precision=precision)
    assert int(st.item()) == 0
    U, S, V = to_np(U), to_np(S), to_np(V)
    s, sr = sing_vals(S), sing_vals(Sr)
    # the rank-15 signal part of every slice, and the whole top-k spectrum
    e15 = rel_fro(s[:15], sr[:15])
    ek = rel_fro(s, sr)
    X64 = X.astype(np.float64)
    err = np.linalg.norm(X64 - approx(U, S, V))
    err_ref = np.linalg.norm(X64 - approx(Ur, Sr, Vr))
    print(f"precision {precision}: signal singular values {e15:.2e}, top-{k} {ek:.2e}, "
          f"approximation error ratio {err / err_ref - 1:.2e}")
    assert e15 < TOL_FP32 and ek < TOL_FP32
    assert abs(err / err_ref - 1) < 1e-4
    # factors orthonormal slice by slice
    Uh = tensor_ref.half_spectrum(tensor_ref.fft3(U))
    for f in (0, 1, 500, 1000):
        G = Uh[:, :, f].conj().T @ Uh[:, :, f]
        assert np.abs(G - np.eye(k)).max() < 1e-4


def test_breakdown_is_flagged_not_hung():
    """Slices of more than 256 rows are orthonormalised by CholeskyQR2 in
    global memory.  An all-zero tensor makes every Gram matrix zero: the
    Cholesky fails even after the shift and must raise the device breakdown
    bit."""
    import torch
    X = np.zeros((300, 10, 4), dtype=np.float32)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    tp.tsvd_randomized(dev(X), 3, 2, 1, seed=0, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) & 0x2


def test_zero_tensor_householder_path():
    """The shared-memory Householder QR cannot break down: an all-zero tensor
    gives zero singular values, orthonormal U (the reflectors are all the
    identity, so Q is the first columns of I) and no status bit."""
    import torch
    X = np.zeros((12, 10, 4), dtype=np.float32)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    U, S, V = tp.tsvd_randomized(dev(X), 3, 2, 1, seed=0, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    U, S, V = to_np(U), to_np(S), to_np(V)
    assert np.all(np.isfinite(U)) and np.all(np.isfinite(V))
    assert np.all(S == 0) and np.all(V == 0)
    Uh = tensor_ref.half_spectrum(tensor_ref.fft3(U))
    for f in range(Uh.shape[2]):
        assert np.abs(Uh[:, :, f].conj().T @ Uh[:, :, f] - np.eye(3)).max() < 1e-6


def test_per_frequency_ranks_match_oracle():
    # a spectrum with clear gaps at every rank used (tubal rank 6 with
    # decaying factors): each frequency keeps its own r_f <= 6
    import torch
    n1, n2, n3, k, p, q = 48, 40, 10, 6, 4, 1
    X = synth.lowrank_np(n1, n2, n3, 6, seed=21)
    h = n3 // 2 + 1
    ranks = np.array([6, 2, 0, 4, 1, 3], dtype=np.int32)
    rk = torch.from_numpy(ranks).cuda()
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    U, S, V = tp.tsvd_randomized(dev(X), k, p, q, seed=5, status=st, ranks=rk)
    assert int(st.item()) == 0
    Om = philox_ref.sketch_signs(n2, k + p, h, n3, 5)
    Ur, Sr, Vr = decomp_ref.tsvd_randomized(X.astype(np.float64), k, p, q, Om, ranks=ranks)
    s, sr = sing_vals(to_np(S)), sing_vals(Sr)
    for f in range(h):            # zero in the Fourier domain up to the round trip of S
        assert np.all(np.abs(s[ranks[f]:, f]) < 1e-6 * s.max())
    assert rel_fro(s, sr) < TOL_FP32
    # the truncated approximations agree (each frequency's top r_f subspace is
    # separated from the rest)
    assert rel_fro(approx(to_np(U), to_np(S), to_np(V)), approx(Ur, Sr, Vr)) < TOL_FP32
    # ranks = k everywhere is the plain call
    U2, S2, V2 = tp.tsvd_randomized(dev(X), k, p, q, seed=5,
                                    ranks=torch.full((h,), k, dtype=torch.int32, device="cuda"))
    U0, S0, V0 = tp.tsvd_randomized(dev(X), k, p, q, seed=5)
    assert torch.equal(U2, U0) and torch.equal(S2, S0) and torch.equal(V2, V0)


@pytest.mark.parametrize("n1,n2,n3,r,k,p,q", [(48, 40, 8, 4, 4, 6, 1), (30, 64, 7, 3, 3, 5, 0),
                                              (64, 48, 16, 5, 6, 4, 2)])
def test_slice_sketch_matches_oracle(n1, n2, n3, r, k, p, q):
    # t-CX sketch: Y = rescaled picked columns of X_hat (i.i.d. picks)
    import torch
    X = synth.lowrank_np(n1, n2, n3, r, seed=n1 + r)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    U, S, V = tp.tsvd_randomized(dev(X), k, p, q, seed=7, status=st, sketch=tp.TP_SKETCH_SLICES)
    assert int(st.item()) == 0
    Om = decomp_ref.slice_sketch(X, k + p, 7)
    Ur, Sr, Vr = decomp_ref.tsvd_randomized(X.astype(np.float64), k, p, q, Om)
    A = approx(to_np(U), to_np(S), to_np(V))
    assert rel_fro(A, X.astype(np.float64)) < TOL_FP32          # exact tubal rank recovered
    assert rel_fro(A, approx(Ur, Sr, Vr)) < TOL_FP32
    s, sr = sing_vals(to_np(S)), sing_vals(Sr)
    assert rel_fro(s[:r], sr[:r]) < TOL_FP32
    # the sign sketch is a different test matrix but the same exact result
    U2, S2, V2 = tp.tsvd_randomized(dev(X), k, p, q, seed=7)
    assert rel_fro(approx(to_np(U2), to_np(S2), to_np(V2)), A) < TOL_FP32


@pytest.mark.parametrize("precision", [tp.TP_FP32, tp.TP_BF16X3])
@pytest.mark.parametrize("n1,n2,n3,r,k,p,q,sizes", [
    (48, 40, 10, 6, 6, 4, 1, [10, 3, 6, 8, 1, 7]),
    (40, 48, 7, 5, 4, 4, 2, [2, 8, 5, 4]),
    (300, 40, 4, 3, 4, 3, 1, [7, 2, 4]),          # CholeskyQR2 (more than 256 rows)
])
def test_per_frequency_sketch_sizes_match_oracle(n1, n2, n3, r, k, p, q, sizes, precision):
    # slice f sketches with the first l_f columns of the same Philox test
    # matrix on both sides; l_f below the tubal rank gives a (deterministic)
    # approximation, l_f at or above it the exact slice
    import torch
    X = synth.lowrank_np(n1, n2, n3, r, seed=n1 + n2 + r)
    h = n3 // 2 + 1
    sz = np.array(sizes, dtype=np.int32)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    U, S, V = tp.tsvd_randomized(dev(X), k, p, q, seed=11, status=st, precision=precision,
                                 sketch_sizes=torch.from_numpy(sz).cuda())
    assert int(st.item()) == 0
    Om = philox_ref.sketch_signs(n2, k + p, h, n3, 11)
    Ur, Sr, Vr = decomp_ref.tsvd_randomized(X.astype(np.float64), k, p, q, Om, sketch_sizes=sz)
    s, sr = sing_vals(to_np(S)), sing_vals(Sr)
    assert rel_fro(s, sr) < TOL_FP32
    for f in range(h):            # min(k, l_f) triplets, zeros after (up to the round trip)
        kf = min(k, int(sz[f]))
        assert np.all(np.abs(s[kf:, f]) <= 1e-6 * s.max())
    assert rel_fro(approx(to_np(U), to_np(S), to_np(V)), approx(Ur, Sr, Vr)) < TOL_FP32
    # sizes of k + p everywhere are the plain call, bit for bit
    full = torch.full((h,), k + p, dtype=torch.int32, device="cuda")
    U1, S1, V1 = tp.tsvd_randomized(dev(X), k, p, q, seed=11, precision=precision,
                                    sketch_sizes=full)
    U0, S0, V0 = tp.tsvd_randomized(dev(X), k, p, q, seed=11, precision=precision)
    assert torch.equal(U1, U0) and torch.equal(S1, S0) and torch.equal(V1, V0)


def test_core_iteration_cap_is_flagged():
    """The core eigensolver's QL takes at most max_sweeps chases per
    eigenvalue: a cap of one on a generic tensor must raise the device
    non-convergence bit (its off-diagonals are dropped, nothing hangs) and
    still give finite factors."""
    import torch
    X = synth.lowrank_np(48, 40, 6, 12, seed=31, noise=1e-2)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    U, S, V = tp.tsvd_randomized(dev(X), 8, 4, 1, seed=0, status=st, max_sweeps=1)
    torch.cuda.synchronize()
    assert int(st.item()) & 0x1
    assert bool(torch.isfinite(U).all()) and bool(torch.isfinite(S).all())
    st.zero_()
    tp.tsvd_randomized(dev(X), 8, 4, 1, seed=0, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
