"""C-ABI checks that need no GPU: the library loads, exports every function
include/tprod.h declares, and rejects bad arguments before touching CUDA."""
import ctypes
import os
import re

import pytest

import paper_1704_04362_gb300 as tp

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "tprod.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*([a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(tp.lib_path()):
        pytest.skip("libtprod.so not built (run __graft_entry__.build())")
    return tp.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("tprod", "tprod_sampled", "tsvd", "tsvd_randomized", "tcomplete_svt"):
        assert must in names
    assert set(names) == set(tp.exported_symbols())


def test_library_exports_every_declared_symbol(L):
    for name in declared_functions():
        assert hasattr(L, name), name
    assert L.tp_version() >= 1
    assert L.tp_status_string(0) == b"TP_OK"
    assert b"workspace" in L.tp_status_string(-9)


def test_null_and_size_errors_need_no_gpu(L):
    nul = None
    assert L.tprod(nul, nul, nul, 2, 2, 2, 2, nul, nul) == -2
    assert b"NULL" in L.tp_last_error()
    p = ctypes.c_void_p(16)  # never dereferenced: validation fails first
    assert L.tprod(p, p, p, 0, 2, 2, 2, nul, nul) == -1
    assert L.tprod(p, p, p, 2, -1, 2, 2, nul, nul) == -1
    assert L.tprod_sampled(p, p, p, 2, 2, 2, 2, 0, 0, 0, 0, nul, nul, nul, nul, nul) == -1  # c = 0
    assert L.tprod_sampled(p, p, p, 2, 2, 2, 2, 1, 0, 7, 0, nul, nul, nul, nul, nul) == -1  # mode
    assert L.tprod_sampled(p, p, p, 2, 2, 2, 2, 1, 0, 2, 0, nul, nul, nul, nul, nul) == -2  # p_given
    assert L.tprod_sampled(p, p, p, 2, 2, 2, 2, 1, 0, 0, 5, nul, nul, nul, nul, nul) == -1  # sample
    assert L.tprod_sampled(p, p, p, 2, 2, 2, 2, 3, 0, 0, 1, nul, nul, nul, nul, nul) == -1  # c > n2
    assert L.tp_sample_draw(nul, nul, 4, 1, 0, 0, 0, 0, nul, nul, nul, nul, nul) == -2
    assert L.tp_sample_draw(p, nul, 4, 1, 0, 1, 2, 0, p, nul, p, nul, nul) == -1     # sample
    assert L.tp_slice_norms(p, 2, 2, 2, 5, p, nul, nul) == -1
    t = [nul] * 8
    assert L.tcur(nul, 2, 2, 2, 1, 1, 0, 0, 1, nul, nul, p, *t) == -2      # A
    assert L.tcur(p, 2, 2, 2, 1, 0, 0, 0, 1, nul, nul, p, *t) == -1        # l = 0
    assert L.tcur(p, 2, 2, 2, 1, 1, -1, 0, 1, nul, nul, p, *t) == -1       # rank < 0
    assert L.tcur(p, 2, 2, 2, 1, 1, 0, 0, 0, nul, nul, p, *t) == -1        # mode AB
    assert L.tcur(p, 2, 2, 2, 1, 1, 0, 0, 2, nul, nul, p, *t) == -2        # p_cols
    assert L.tcur(p, 600, 600, 2, 1, 1, 0, 0, 1, nul, nul, p, *t) == -10   # min(n1, n2) > 512
    d = ctypes.c_double
    k = [d(1e-3), d(1.1), d(1e10), d(1e-4), p, nul, nul] + [nul] * 7
    assert L.cur_tnn(nul, nul, 2, 2, 2, 1, 1, 0, 0, 1, nul, nul, 5, d(0), *k) == -2   # X
    assert L.cur_tnn(p, nul, 2, 2, 2, 1, 1, 0, 0, 1, nul, nul, -1, d(0), *k) == -1    # iters
    assert L.cur_tnn(p, nul, 2, 2, 2, 1, 1, 0, 0, 1, nul, nul, 5, d(-1), *k) == -1    # lambda
    assert L.cur_tnn(p, nul, 2, 2, 2, 1, 1, 0, 0, 2, nul, nul, 5, d(0), *k) == -2     # p_cols
    k[0] = d(0.0)
    assert L.cur_tnn(p, nul, 2, 2, 2, 1, 1, 0, 0, 1, nul, nul, 5, d(0), *k) == -1     # mu0
    # randomized t-SVD: unknown sketch mode, and k + p beyond min(n1, n2)
    assert L.tsvd_randomized(p, 8, 8, 4, 2, 2, 1, 0, 7, nul, nul, p, p, p, nul, nul) == -1
    assert L.tsvd_randomized(p, 8, 8, 4, 6, 4, 1, 0, 0, nul, nul, p, p, p, nul, nul) == -1
    # a status word without a host destination
    assert L.tp_sync_status(nul, p, nul) == -2
    # with-replacement draws need c <= n
    assert L.tp_sample_draw(p, nul, 4, 5, 0, 2, 1, 0, p, nul, p, nul, nul) == -1


def test_workspace_query_is_monotone(L):
    def q(op, dims):
        d = (ctypes.c_int64 * len(dims))(*dims)
        return L.tp_workspace_query(op, ctypes.cast(d, ctypes.c_void_p), len(dims), None)
    small = q(tp.binding.TP_OP_TPROD, [4, 4, 4, 4])
    big = q(tp.binding.TP_OP_TPROD, [64, 48, 32, 16])
    assert 0 < small < big
    # cfg2-sized sampled product: capacity for every slice, a few GB at most
    s = q(tp.binding.TP_OP_TPROD_SAMPLED, [2000, 4000, 1500, 64])
    assert 1 << 30 < s < 16 << 30


def test_no_cpu_fallback_without_cuda():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(tp.TprodError):
        tp.empty_tensor(2, 2, 2)


def test_autotune_table_round_trip_needs_no_gpu(L, tmp_path):
    prev = L.tp_autotune_mode(-1)
    assert prev in (0, 1)
    assert L.tp_autotune_mode(0) == prev and L.tp_autotune_mode(-1) == 0
    L.tp_autotune_mode(prev)
    tp.autotune_reset()
    f = tmp_path / "tune.txt"
    f.write_text("rdft:64,2000,4000,2,1,1,1 2\nnorms_lateral:2000,256000,1 1\n")
    tp.autotune_load(f)
    table = tp.autotune_table()
    assert [(k, c) for k, c, *_ in table] == [("norms_lateral:2000,256000,1", 1),
                                               ("rdft:64,2000,4000,2,1,1,1", 2)]
    assert all(best == -1.0 and d == -1.0 for *_, best, d in table)   # loaded, not timed
    g = tmp_path / "again.txt"
    tp.autotune_save(g)
    assert sorted(g.read_text().splitlines()) == sorted(f.read_text().splitlines())
    (tmp_path / "bad.txt").write_text("rdft:1 x\n")
    with pytest.raises(tp.TprodError):
        tp.autotune_load(tmp_path / "bad.txt")
    tp.autotune_reset()
    assert tp.autotune_table() == []
    assert tp.autotune_force(3) == -1 and tp.autotune_force(-1) == 3
