"""GPU parity of the tensor-completion ADMM (Algorithm 7, completion form of
problem tlow6) with tensor singular-value thresholding, against the float64
oracle, through the C ABI."""
import numpy as np
import pytest

import paper_1704_04362_gb300 as tp
from paper_1704_04362_gb300 import synth
from oracle import completion_ref
from tests.util import TOL_FP32, rel_fro, to_np, tol_for

pytestmark = pytest.mark.gpu


def dev(x, dtype=None):
    return tp.as_tprod_layout(x, dtype)


def state_on_device(X, mask, L, E, Y, mu):
    import torch
    return (dev(X), dev(mask.astype(np.uint8), torch.uint8), dev(L), dev(E), dev(Y),
            torch.tensor([mu], dtype=torch.float64, device="cuda"))


# the last five slices exceed the shared-memory Jacobi: in a batch they take
# the blocked one (128 columns in 8 blocks; 150 columns, transposed, with a
# ragged block; then 128, 300 and 400 rows: the register form's row counts
# up to 128, 384 and 512), alone (fewer slices than SMs, >= 32 columns) the
# cluster-per-slice sweeps
@pytest.mark.parametrize("form", ["alone", "batch"])
@pytest.mark.parametrize("precision", [tp.TP_FP32, tp.TP_TF32X3, tp.TP_BF16X3])
@pytest.mark.parametrize("n1,n2,n3", [(20, 16, 6), (12, 30, 5), (24, 24, 1), (33, 17, 8),
                                      (160, 128, 4), (150, 200, 5), (120, 128, 3),
                                      (300, 130, 3), (100, 400, 2)])
def test_one_iteration_matches_oracle(n1, n2, n3, precision, form):
    """One iteration in each form: FP32, and the SVT's three GEMMs on the
    tensor cores with the 3xTF32 or BF16x3 split (held to that split's
    tolerance); through tcomplete_svt and as a batch of one tensor."""
    import torch
    g = np.random.default_rng(n1 * n2 + n3)
    X = synth.lowrank_np(n1, n2, n3, 3, seed=n3, noise=0.01)
    X = X / np.sqrt(np.mean(X.astype(np.float64) ** 2))
    mask = g.random(X.shape) < 0.6
    E = np.where(mask, 0, g.standard_normal(X.shape)).astype(np.float32)
    Y = (0.1 * g.standard_normal(X.shape)).astype(np.float32)
    L0 = np.zeros_like(X)
    # tau = 1/mu inside the range of the slice singular values
    mu = 0.08
    Xd, Md, Ld, Ed, Yd, mud = state_on_device(X, mask, L0, E, Y, mu)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    if form == "alone":
        tp.tcomplete_svt(Xd, Md, 1, L=Ld, E=Ed, Y=Yd, mu=mud, status=st, precision=precision)
    else:
        tp.tcomplete_svt_batched([(Xd, Md, Ld, Ed, Yd, mud)], 1, status=st, precision=precision)
    assert int(st.item()) == 0
    Xo = np.where(mask, X.astype(np.float64), 0.0)
    Lr, Er, Yr, mur = completion_ref.admm_step(Xo, mask, L0.astype(np.float64),
                                               E.astype(np.float64), Y.astype(np.float64), mu)
    assert np.linalg.norm(Lr) > 0          # the threshold keeps part of the spectrum
    tol = tol_for(precision)
    assert rel_fro(to_np(Ld), Lr) < tol
    assert rel_fro(to_np(Ed), Er) < tol
    # Y <- Y + mu (L + E - X) (Algorithm 7) inherits mu times L's error: Y is
    # held to the float32 bound on the scale of that update
    dY = np.linalg.norm(to_np(Yd) - Yr)
    assert dY < tol * (np.linalg.norm(Yr) + mu * np.linalg.norm(Lr))
    assert abs(float(mud.item()) - mur) <= 1e-15 * mur
    assert np.all(to_np(Ed)[mask] == 0)


def test_many_iterations_track_oracle_and_resume():
    import torch
    X = synth.lowrank_np(20, 20, 6, 2, seed=60)
    X = X / np.sqrt(np.mean(X.astype(np.float64) ** 2))
    mask = np.random.default_rng(61).random(X.shape) < 0.6
    Z = np.zeros_like(X)
    Xd, Md, Ld, Ed, Yd, mud = state_on_device(X, mask, Z, Z, Z, 1e-3)
    tp.tcomplete_svt(Xd, Md, 60, L=Ld, E=Ed, Y=Yd, mu=mud)
    Lr, Er, Yr, mur = completion_ref.tcomplete_svt(X.astype(np.float64), mask, 60)
    # float32 state carried over 60 iterations: looser bound than one step
    assert rel_fro(to_np(Ld), Lr) < 1e-4
    assert abs(float(mud.item()) / mur - 1) < 1e-12
    # resuming from the returned state (L, E, Y, mu) equals one longer run up
    # to float32 rounding carried over the iterations (the bound held against
    # the oracle above): the only state not carried over is the slice
    # Jacobi's starting rotations (warm within a call, the identity at a
    # call's start)
    Xd2, Md2, La, Ea, Ya, mua = state_on_device(X, mask, Z, Z, Z, 1e-3)
    tp.tcomplete_svt(Xd2, Md2, 25, L=La, E=Ea, Y=Ya, mu=mua)
    tp.tcomplete_svt(Xd2, Md2, 35, L=La, E=Ea, Y=Ya, mu=mua)
    assert rel_fro(to_np(La), to_np(Ld)) < 1e-4
    assert rel_fro(to_np(Ya), to_np(Yd)) < 1e-4
    assert rel_fro(to_np(Ea), to_np(Ed)) < 1e-4
    assert float(mua.item()) == float(mud.item())
    # and a repeated call is deterministic
    Xd3, Md3, Lb, Eb, Yb, mub = state_on_device(X, mask, Z, Z, Z, 1e-3)
    tp.tcomplete_svt(Xd3, Md3, 60, L=Lb, E=Eb, Y=Yb, mu=mub)
    assert torch.equal(Lb, Ld) and torch.equal(Yb, Yd) and torch.equal(Eb, Ed)


def test_recovers_low_rank_video():
    """A small video-shaped tensor (tubal rank 3, unit RMS, sigma = 0.01 noise,
    50% observed): after 150 iterations the relative error to the clean
    tensor is at the noise level."""
    truth, noisy, mask = synth.video_np(40, 36, 12, r=3, seed=4, sigma=0.01, observed=0.5)
    Z = np.zeros_like(noisy)
    Xd, Md, Ld, Ed, Yd, mud = state_on_device(noisy, mask.astype(bool), Z, Z, Z, 1e-3)
    tp.tcomplete_svt(Xd, Md, 150, L=Ld, E=Ed, Y=Yd, mu=mud)
    rse = rel_fro(to_np(Ld), truth.astype(np.float64))
    assert rse < 0.05


@pytest.mark.parametrize("precision", [tp.TP_FP32, tp.TP_BF16X3])
def test_batched_equals_separate_calls_and_oracle(precision):
    """tcomplete_svt_batched over tensors of uneven sizes (one per side
    stream and a shared side stream for the rest, graph replay after the
    first iteration) gives exactly the results of separate tcomplete_svt
    calls, in the FP32 and the BF16x3 form; the first tensor also tracks the
    oracle."""
    import torch
    sizes = [(20, 16, 6), (12, 30, 5), (33, 17, 8), (24, 24, 1), (16, 40, 7), (9, 11, 4),
             (30, 22, 3), (18, 18, 9), (40, 12, 6), (14, 26, 5)]
    iters = 12
    batch, single = [], []
    for i, (n1, n2, n3) in enumerate(sizes):
        X = synth.lowrank_np(n1, n2, n3, 3, seed=70 + i, noise=0.01)
        X = X / np.sqrt(np.mean(X.astype(np.float64) ** 2))
        mask = np.random.default_rng(80 + i).random(X.shape) < 0.6
        Z = np.zeros_like(X)
        batch.append(state_on_device(X, mask, Z, Z, Z, 1e-3))
        single.append(state_on_device(X, mask, Z, Z, Z, 1e-3))
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    tp.tcomplete_svt_batched(batch, iters, status=st, precision=precision)
    assert int(st.item()) == 0
    for (Xd, Md, L, E, Y, mu) in single:
        tp.tcomplete_svt(Xd, Md, iters, L=L, E=E, Y=Y, mu=mu, precision=precision)
    for b, s in zip(batch, single):
        for x, y in zip(b[2:], s[2:]):
            assert torch.equal(x, y)
    # the oracle on the first tensor
    n1, n2, n3 = sizes[0]
    X = synth.lowrank_np(n1, n2, n3, 3, seed=70, noise=0.01)
    X = X / np.sqrt(np.mean(X.astype(np.float64) ** 2))
    mask = np.random.default_rng(80).random(X.shape) < 0.6
    Lr, _, _, mur = completion_ref.tcomplete_svt(X.astype(np.float64), mask, iters)
    assert rel_fro(to_np(batch[0][2]), Lr) < (1e-4 if precision == tp.TP_FP32 else 5e-4)
    assert abs(float(batch[0][5].item()) / mur - 1) < 1e-12


def test_robust_form_one_iteration_matches_oracle():
    """Algorithm 7 as printed (problem tlow7): the E-step soft-thresholds every
    entry at lambda/mu."""
    import torch
    g = np.random.default_rng(50)
    X = synth.lowrank_np(22, 18, 6, 3, seed=51, noise=0.01)
    X = (X / np.sqrt(np.mean(X.astype(np.float64) ** 2))).astype(np.float32)
    E = (0.3 * g.standard_normal(X.shape)).astype(np.float32)
    Y = (0.1 * g.standard_normal(X.shape)).astype(np.float32)
    mu, lam = 0.08, 0.15
    Ld, Ed, Yd = dev(np.zeros_like(X)), dev(E), dev(Y)
    mud = torch.tensor([mu], dtype=torch.float64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    tp.trpca_admm(dev(X), 1, lam=lam, L=Ld, E=Ed, Y=Yd, mu=mud, status=st)
    assert int(st.item()) == 0
    Lr, Er, Yr, mur = completion_ref.admm_robust_step(X.astype(np.float64), 0.0, E.astype(np.float64),
                                                      Y.astype(np.float64), mu, lam)
    assert rel_fro(to_np(Ld), Lr) < TOL_FP32
    assert rel_fro(to_np(Ed), Er) < TOL_FP32
    assert rel_fro(to_np(Yd), Yr) < TOL_FP32
    assert abs(float(mud.item()) - mur) <= 1e-15 * mur


def test_robust_form_recovers_low_rank_plus_sparse_and_tracks_oracle():
    L0 = synth.lowrank_np(30, 30, 6, 2, seed=41).astype(np.float64)
    L0 /= np.sqrt(np.mean(L0 ** 2))
    g = np.random.default_rng(42)
    S0 = np.where(g.random(L0.shape) < 0.05, 10.0 * g.standard_normal(L0.shape), 0.0)
    X = (L0 + S0).astype(np.float32)
    L, E, Y, mu = tp.trpca_admm(dev(X), 60)
    Lr, Er, Yr, mur = completion_ref.trpca(X.astype(np.float64), 60)
    assert rel_fro(to_np(L), Lr) < 1e-4                 # float32 state over 60 iterations
    assert abs(float(mu.item()) / mur - 1) < 1e-12
    L2, E2, _, _ = tp.trpca_admm(dev(X), 120)
    assert rel_fro(to_np(L2), L0) < 1e-3 and rel_fro(to_np(E2), S0) < 1e-3


@pytest.mark.parametrize("form", ["alone", "batch"])
def test_blocked_jacobi_slices_track_oracle_over_iterations(form):
    # 160 x 128 slices, warm-started every iteration: in a batch the blocked
    # Jacobi, alone the cluster-per-slice sweeps
    import torch
    X = synth.lowrank_np(160, 128, 4, 3, seed=62, noise=0.01)
    X = X / np.sqrt(np.mean(X.astype(np.float64) ** 2))
    mask = np.random.default_rng(63).random(X.shape) < 0.6
    Z = np.zeros_like(X)
    Xd, Md, Ld, Ed, Yd, mud = state_on_device(X, mask, Z, Z, Z, 1e-3)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    if form == "alone":
        tp.tcomplete_svt(Xd, Md, 30, L=Ld, E=Ed, Y=Yd, mu=mud, status=st)
    else:
        tp.tcomplete_svt_batched([(Xd, Md, Ld, Ed, Yd, mud)], 30, status=st)
    assert int(st.item()) == 0
    Lr, Er, Yr, mur = completion_ref.tcomplete_svt(X.astype(np.float64), mask, 30)
    assert rel_fro(to_np(Ld), Lr) < 1e-4                 # float32 state over 30 iterations
    assert abs(float(mud.item()) / mur - 1) < 1e-12
