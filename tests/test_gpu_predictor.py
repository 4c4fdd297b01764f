"""The learned sketch-size predictor end to end on the GPU: trained by the
library's own kernels on tensors the plain method decomposes, it must (a)
lower its loss, (b) never do worse than the plain method in truncation error
on held-out tensors (the plain rule judges every result and falls back to the
full sketch when a rank reaches its cap), and (c) choose smaller sketches
than the plain method's 50 columns where the spectra decay fast."""
import numpy as np
import pytest

import paper_1704_04362_gb300 as tp
from paper_1704_04362_gb300 import predictor as P
from paper_1704_04362_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trained():
    x, t = P.training_set(60, seed0=100)
    theta, w16, losses = P.train(x, t, steps=1500, lr=2e-3, seed=1)
    return w16, losses, x, t


def test_training_lowers_the_loss(trained):
    _, losses, x, t = trained
    assert x.shape[1] == 16 and t.shape[1] == 2 and x.shape[0] == t.shape[0] > 500
    first, last = losses[0][1], losses[-1][1]
    assert last < 0.2 * first, losses


SHAPES = {16: (144, 128), 64: (96, 96), 128: (80, 64), 256: (64, 64)}


@pytest.mark.parametrize("n3", [16, 64, 128, 256])
@pytest.mark.parametrize("alpha", [1.5, 2.5, 3.5])
def test_learned_matches_plain_error_with_smaller_sketches(trained, alpha, n3):
    w16 = trained[0]
    n1, n2 = SHAPES[n3]
    sizes, errs_l, errs_p = [], [], []
    for s in range(4 if n3 == 16 else 2):
        X, spec = synth.spectral_torch(n1, n2, n3, alpha, 0.3,
                                       9000 + 10 * s + int(10 * alpha) + 1000 * n3)
        r_plain, _, _ = P.decompose(X, None, seed=s)
        r_learn, l, fell_back = P.decompose(X, w16, seed=s)
        e_plain = P.truncation_error(spec, r_plain, n3)
        e_learn = P.truncation_error(spec, r_learn, n3)
        sizes.append(l)
        errs_p.append(e_plain)
        errs_l.append(e_learn)
        # the rule as arbiter: never a worse truncation than the plain method (beyond the
        # sketch's own resolution of the tail)
        assert e_learn <= 1.05 * e_plain + 2e-3, (alpha, n3, s, e_learn, e_plain, l, fell_back)
    if alpha >= 2.5:
        assert np.mean(sizes) < 40, sizes       # fast decay: smaller sketches than 50


@pytest.mark.parametrize("per_frequency", [False, True])
def test_multi_rank_factorisation_reaches_the_rule_error(trained, per_frequency):
    # U * S * V^T with every frequency truncated to the predicted-and-judged
    # rank: its error is the per-frequency truncation error of those ranks
    # (up to the sketch's resolution of the tail), with one sketch size for
    # all frequencies or each frequency's own predicted l_f = r_f + p_f
    import torch
    w16 = trained[0]
    X, spec = synth.spectral_torch(144, 128, 16, 3.0, 0.3, 9100)
    U, S, V, r, l = P.factorize(X, w16, seed=1, per_frequency=per_frequency)
    if per_frequency:
        sizes = P.sketch_sizes(w16, X, r, l, seed=1)
        assert bool((sizes >= r.int() + 2).all()) and int(sizes.max()) <= l
        assert int(sizes.min()) < l            # some frequency sketches with fewer columns
    assert U.shape[1] == int(r.max().item()) and l <= 50
    # t-product U * S * V^T through the library's own exact t-product
    Vt = torch.flip(V.permute(1, 0, 2), dims=[2])
    Vt = torch.roll(Vt, 1, dims=2)                     # (V^T): transpose slices, reverse 2..n3
    US = tp.tprod(tp.as_tprod_layout(U), tp.as_tprod_layout(S))
    R = tp.tprod(US, tp.as_tprod_layout(Vt.contiguous()))
    err = float(torch.linalg.vector_norm(R - X) / torch.linalg.vector_norm(X))
    want = P.truncation_error(spec, r, 16)
    assert want * (1 - 1e-4) <= err <= 1.05 * want + 2e-3, (err, want)
