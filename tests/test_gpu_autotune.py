"""The launch-shape autotuner on the GPU: every candidate shape of a tunable
launch gives bit-identical results, the first call of a shape fills the
table with a timed choice no slower than the default, and a stream being
captured into a CUDA graph is never timed."""
import numpy as np
import pytest

import paper_1704_04362_gb300 as tp
from paper_1704_04362_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture
def tuner():
    prev = tp.autotune_mode(tp.TP_TUNE_ON)
    tp.autotune_reset()
    yield
    tp.autotune_force(-1)
    tp.autotune_mode(prev)


def forced(fn, ncand):
    import torch
    outs = []
    for c in range(ncand):
        tp.autotune_force(c)
        outs.append([t.clone() for t in fn()])
        torch.cuda.synchronize()
    tp.autotune_force(-1)
    return outs


@pytest.mark.parametrize("n3", [12, 5, 64, 16])
def test_transform_candidates_are_bit_identical(tuner, n3):
    import torch
    X = tp.as_tprod_layout(synth.iid_normal((300, 70, n3), seed=n3))
    fwd = forced(lambda: tp.rdft3(X), 4)
    for o in fwd[1:]:
        assert all(torch.equal(a, b) for a, b in zip(o, fwd[0]))
    Xr, Xi = fwd[0]
    inv = forced(lambda: [tp.irdft3(Xr, Xi, n3)], 4)
    for o in inv[1:]:
        assert torch.equal(o[0], inv[0][0])
    assert torch.allclose(inv[0][0], X, atol=1e-5)


def test_lateral_norm_candidates_are_bit_identical(tuner):
    import torch
    for shape in [(100, 3000, 5), (2000, 64, 8), (37, 500, 3)]:
        X = tp.as_tprod_layout(synth.iid_normal(shape, seed=sum(shape)))
        outs = forced(lambda: [tp.slice_norms(X, 0)], 4)
        for o in outs[1:]:
            assert torch.equal(o[0], outs[0][0])


def test_first_call_fills_the_table(tuner):
    A = tp.as_tprod_layout(synth.iid_normal((256, 300, 64), seed=1))
    B = tp.as_tprod_layout(synth.iid_normal((300, 200, 64), seed=2))
    Z1, _, _ = tp.tprod_sampled(A, B, 50, seed=3, precision=tp.TP_BF16X3)
    table = tp.autotune_table()
    ops = {k.split(":")[0] for k, *_ in table}
    assert {"norms_lateral", "rfft_reg", "irfft_reg"} <= ops, ops
    for key, choice, ncand, best, dflt in table:
        assert 0 <= choice < ncand and 0 < best <= dflt, (key, best, dflt)
    Z2, _, _ = tp.tprod_sampled(A, B, 50, seed=3, precision=tp.TP_BF16X3)
    assert len(tp.autotune_table()) == len(table)          # cached: nothing timed again
    assert bool((Z1 == Z2).all())


def test_graph_capture_is_never_timed(tuner):
    import torch
    X = tp.as_tprod_layout(synth.iid_normal((128, 40, 12), seed=5))
    eager = tp.rdft3(X)
    tp.autotune_reset()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            out = tp.rdft3(X)
    assert tp.autotune_table() == []
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out[0], eager[0]) and torch.equal(out[1], eager[1])
