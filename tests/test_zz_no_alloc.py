"""tp_slice_norms_noalloc: the slice norms for callers that cannot allocate
device memory (its scratch is a fixed array inside the library).  Checked
through the C ABI against tp_slice_norms on two calls in a row.  This file is
collected last so that a failure here comes after every other test ran."""
import ctypes

import numpy as np
import pytest

import paper_1704_04362_gb300 as tp
from paper_1704_04362_gb300 import synth

pytestmark = pytest.mark.gpu


def test_noalloc_norms_match_allocating_entry_point_twice():
    import torch
    L = tp.lib()
    cap = int(L.tp_slice_norms_noalloc_capacity())
    assert cap == 1 << 20
    cases = [((300, 700, 16), 0), ((2000, 40, 8), 1), ((37, 41, 3), 0), ((64, 48, 16), 1)]
    for (n1, n2, n3), which in cases:
        X = tp.as_tprod_layout(synth.iid_normal((n1, n2, n3), seed=n1 + n2))
        ref = tp.slice_norms(X, which)
        n_out = n2 if which == 0 else n1
        out = torch.full((n_out,), float("nan"), dtype=torch.float64, device="cuda")
        for _ in range(2):   # the shared array keeps the previous call's contents
            out.fill_(float("nan"))
            rc = L.tp_slice_norms_noalloc(ctypes.c_void_p(X.data_ptr()), n1, n2, n3, which,
                                          ctypes.c_void_p(out.data_ptr()),
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
            assert rc == 0, L.tp_last_error()
            torch.cuda.synchronize()
            np.testing.assert_allclose(out.cpu().numpy(), ref.cpu().numpy(), rtol=1e-11, atol=0)


def test_noalloc_rejects_sizes_beyond_capacity():
    import torch
    L = tp.lib()
    X = tp.as_tprod_layout(np.zeros((1, 1, 1), dtype=np.float32))
    out = torch.zeros(1 << 11, dtype=torch.float64, device="cuda")
    # lateral norms of a 1 x 2048 x 1024 tensor need 2^21 partial sums
    rc = L.tp_slice_norms_noalloc(ctypes.c_void_p(X.data_ptr()), 1, 2048, 1024, 0,
                                  ctypes.c_void_p(out.data_ptr()), None)
    assert rc == -1
    assert b"fixed array" in L.tp_last_error()
