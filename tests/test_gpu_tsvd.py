"""GPU parity of the t-SVD (Theorem 2.6 via Eq. circ1) against the float64
oracle, through the C ABI.  Singular vectors are unique only up to a phase
per column, so U and V are compared through invariants: per-frequency
singular values, the reconstruction U * S * V^T, orthogonality U^T * U = I,
and |<u_j, u_j_ref>| for well separated singular values."""
import numpy as np
import pytest

import paper_1704_04362_gb300 as tp
from paper_1704_04362_gb300 import synth
from oracle import decomp_ref, tensor_ref
from tests.util import TOL_FP32, rel_fro, to_np

pytestmark = pytest.mark.gpu


def dev(x):
    return tp.as_tprod_layout(x)


SHAPES = [(64, 48, 16), (48, 64, 16), (5, 3, 4), (3, 5, 5), (7, 7, 1), (130, 40, 17),
          (1, 1, 1), (2, 9, 2), (200, 100, 8),
          # the re-orthonormalised path's limit (4096 entries, 256 rows) and the
          # float64 sweeps beyond it
          (256, 16, 3), (64, 64, 2), (256, 96, 3), (96, 256, 2), (257, 40, 2),
          # fewer slices than SMs and >= 32 columns: cluster-per-slice sweeps;
          # block pairs too large for shared memory in float64 (1700 rows) and
          # in both precisions (3300 rows, transposed)
          (1700, 64, 2), (64, 3300, 2)]


@pytest.mark.parametrize("n1,n2,n3", SHAPES)
def test_tsvd_matches_oracle(n1, n2, n3):
    import torch
    X = synth.iid_normal((n1, n2, n3), seed=0)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    U, S, V = tp.tsvd(dev(X), status=st)
    assert int(st.item()) == 0
    U, S, V = to_np(U), to_np(S), to_np(V)
    m = min(n1, n2)
    X64 = X.astype(np.float64)
    # reconstruction through the block-circulant definition route
    Xr = tensor_ref.tprod(tensor_ref.tprod(U, S), tensor_ref.ttranspose(V))
    assert rel_fro(Xr, X64) < TOL_FP32
    # orthogonality
    I = tensor_ref.identity(m, n3)
    assert np.linalg.norm(tensor_ref.tprod(tensor_ref.ttranspose(U), U) - I) / np.sqrt(m) < 2e-5
    assert np.linalg.norm(tensor_ref.tprod(tensor_ref.ttranspose(V), V) - I) / np.sqrt(m) < 2e-5
    # singular values per frequency
    Uh_ref, s_ref, Vh_ref = decomp_ref.tsvd_hat(X64)
    Sh = tensor_ref.half_spectrum(tensor_ref.fft3(S))
    s_gpu = np.stack([np.diag(Sh[:, :, k]).real for k in range(Sh.shape[2])], axis=1)
    assert rel_fro(s_gpu, s_ref) < TOL_FP32
    off = Sh - np.stack([np.diag(np.diag(Sh[:, :, k])) for k in range(Sh.shape[2])], axis=2)
    assert np.abs(off).max() < 1e-5 * max(1.0, s_ref.max())
    # left singular vectors of well separated singular values, up to phase
    Uh = tensor_ref.half_spectrum(tensor_ref.fft3(U))
    for k in range(Uh.shape[2]):
        s = s_ref[:, k]
        for j in range(m):
            gap = min([abs(s[j] - s[l]) for l in range(m) if l != j] + [np.inf])
            if s[j] > 1e-3 * s[0] and gap > 1e-2 * s[0]:
                ov = abs(np.vdot(Uh_ref[:, j, k], Uh[:, j, k]))
                assert ov > 1 - 1e-4, (k, j, ov)


def test_tsvd_exact_workload_and_sweep_cap_flag():
    """The exact-product workload's A (64 x 48 x 16, iid N(0,1), seed 0); a
    sweep cap of 1 must raise the device non-convergence bit instead of
    looping."""
    import torch
    X = synth.iid_normal((64, 48, 16), seed=0)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    tp.tsvd(dev(X), status=st, max_sweeps=1)
    torch.cuda.synchronize()
    assert int(st.item()) & 0x1


def test_cluster_float64_sweep_cap_flag():
    """A slice pair of 257 x 40 takes the float64 sweeps (over 4096 entries)
    on the cluster-per-slice path; a cap of 1 sweep must raise the device
    non-convergence bit there."""
    import torch
    X = synth.iid_normal((257, 40, 2), seed=1)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    tp.tsvd(dev(X), status=st, max_sweeps=1)
    torch.cuda.synchronize()
    assert int(st.item()) & 0x1


def test_tsvd_low_rank_and_zero():
    import torch
    X = synth.lowrank_np(30, 20, 6, 3, seed=3)
    U, S, V = tp.tsvd(dev(X))
    Sh = tensor_ref.half_spectrum(tensor_ref.fft3(to_np(S)))
    s = np.stack([np.diag(Sh[:, :, k]).real for k in range(Sh.shape[2])], axis=1)
    assert np.all(s[3:] < 1e-4 * s[0])     # tubal rank 3
    Xr = tensor_ref.tprod(tensor_ref.tprod(to_np(U), to_np(S)), tensor_ref.ttranspose(to_np(V)))
    assert rel_fro(Xr, X.astype(np.float64)) < TOL_FP32
    Z = np.zeros((4, 3, 2), dtype=np.float32)
    U, S, V = tp.tsvd(dev(Z))
    assert float(S.abs().max()) == 0.0


def test_sync_status_reports_the_device_status_word():
    import torch
    X = synth.iid_normal((40, 30, 6), seed=8)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    tp.tsvd(dev(X), status=st)
    assert tp.sync_status(st) == 0 and tp.sync_status() == 0
    tp.tsvd(dev(X), status=st, max_sweeps=1)
    assert tp.sync_status(st) & 0x1          # TP_DEV_NOCONV


def test_hand_worked_singular_tube():
    # tests/golden/tube_1x1x3_by_hand.txt: the singular tube of (1, 2, 3)
    from tests.util import golden
    t = golden("tube_1x1x3_by_hand.txt")
    a = np.array([1, 2, 3], dtype=np.float32).reshape(1, 1, 3)
    U, S, V = tp.tsvd(dev(a))
    np.testing.assert_allclose(to_np(S).ravel(), t["svd_s"][0], rtol=1e-6)
