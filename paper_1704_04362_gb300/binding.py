"""ctypes binding of libtprod.so (declared in include/tprod.h).

Argument marshalling only: every step of every path runs in the library's
CUDA kernels.  Tensors are torch CUDA tensors of logical shape (n1, n2, n3)
stored column-major (strides (1, n1, n1*n2)), as produced by
``empty_tensor`` / ``as_tprod_layout``.  The library's scratch memory is a
torch-allocated buffer passed through tp_opts, so the library itself does
not allocate when called from here.  There is no CPU fallback: a missing
library or a CUDA-less process raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

__all__ = [
    "TP_FP32", "TP_TF32X3", "TP_BF16X3", "TP_PROB_AB", "TP_PROB_A2", "TP_PROB_GIVEN",
    "TP_SAMPLE_BERNOULLI", "TP_SAMPLE_IID", "TP_SKETCH_SIGNS", "TP_SKETCH_SLICES",
    "TprodError", "lib", "lib_path", "empty_tensor", "as_tprod_layout",
    "tprod", "tprod_sampled", "tsvd", "tsvd_randomized", "tcomplete_svt", "tcx",
    "rdft3", "irdft3", "slice_norms", "sample_draw", "launch_count", "exported_symbols",
    "profile_start", "profile_stop", "slice_norms_noalloc", "tcomplete_svt_batched",
    "sketch_spectrum", "rank_rule", "rank_features", "mlp_param_count", "mlp_round",
    "mlp_forward", "mlp_train_step", "trpca_admm", "tcur", "cur_tnn",
    "TP_TUNE_OFF", "TP_TUNE_ON", "autotune_mode", "autotune_force", "autotune_table",
    "autotune_save", "autotune_load", "autotune_reset", "sync_status", "philox4x32_10",
]

TP_FP32, TP_TF32X3, TP_BF16X3 = 0, 1, 2
TP_PROB_AB, TP_PROB_A2, TP_PROB_GIVEN = 0, 1, 2
TP_SAMPLE_BERNOULLI, TP_SAMPLE_IID = 0, 1
TP_SKETCH_SIGNS, TP_SKETCH_SLICES = 0, 1
TP_OP_TPROD, TP_OP_TPROD_SAMPLED, TP_OP_TSVD, TP_OP_TSVD_RANDOMIZED, TP_OP_TCOMPLETE_SVT, \
    TP_OP_SLICE_NORMS, TP_OP_TCX, TP_OP_TCOMPLETE_SVT_BATCHED, TP_OP_SKETCH_SPECTRUM, \
    TP_OP_MLP_TRAIN, TP_OP_TRPCA, TP_OP_TCUR, TP_OP_CUR_TNN = \
    1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13

_HERE = os.path.dirname(os.path.abspath(__file__))
_c_i64, _c_u64, _c_int, _c_u32 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32
_vp, _dbl = ctypes.c_void_p, ctypes.c_double


class TprodError(RuntimeError):
    pass


class TpOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("max_sweeps", ctypes.c_int),
                ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_size_t),
                ("status", ctypes.c_void_p), ("pipeline_wait_limit", ctypes.c_int64)]


class TpTensorDesc(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("mask", ctypes.c_void_p), ("L", ctypes.c_void_p),
                ("E", ctypes.c_void_p), ("Y", ctypes.c_void_p), ("mu", ctypes.c_void_p),
                ("n1", ctypes.c_int64), ("n2", ctypes.c_int64), ("n3", ctypes.c_int64)]


# Every symbol include/tprod.h declares, with its ctypes signature.
_SIGS = {
    "tprod": (_c_int, [_vp, _vp, _vp, _c_i64, _c_i64, _c_i64, _c_i64, _vp, _vp]),
    "tprod_sampled": (_c_int, [_vp, _vp, _vp, _c_i64, _c_i64, _c_i64, _c_i64, _c_i64, _c_u64,
                               _c_int, _c_int, _vp, _vp, _vp, _vp, _vp]),
    "tsvd": (_c_int, [_vp, _c_i64, _c_i64, _c_i64, _vp, _vp, _vp, _vp, _vp]),
    "tsvd_randomized": (_c_int, [_vp, _c_i64, _c_i64, _c_i64, _c_int, _c_int, _c_int, _c_u64,
                                 _c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "tcomplete_svt": (_c_int, [_vp, _vp, _c_i64, _c_i64, _c_i64, _c_int, _dbl, _dbl,
                               _vp, _vp, _vp, _vp, _vp, _vp]),
    "tcx": (_c_int, [_vp, _c_i64, _c_i64, _c_i64, _c_i64, _c_u64, _c_int, _vp, _vp, _vp, _vp,
                     _vp, _vp]),
    "tcur": (_c_int, [_vp, _c_i64, _c_i64, _c_i64, _c_i64, _c_i64, _c_int, _c_u64, _c_int, _vp,
                      _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "cur_tnn": (_c_int, [_vp, _vp, _c_i64, _c_i64, _c_i64, _c_i64, _c_i64, _c_int, _c_u64, _c_int,
                         _vp, _vp, _c_int, _dbl, _dbl, _dbl, _dbl, _dbl, _vp, _vp, _vp, _vp, _vp,
                         _vp, _vp, _vp, _vp, _vp]),
    "tcomplete_svt_batched": (_c_int, [_c_int, _vp, _c_int, _dbl, _dbl, _vp, _vp]),
    "trpca_admm": (_c_int, [_vp, _c_i64, _c_i64, _c_i64, _c_int, _dbl, _dbl, _dbl, _vp, _vp, _vp,
                            _vp, _vp, _vp]),
    "tp_sketch_spectrum": (_c_int, [_vp, _c_i64, _c_i64, _c_i64, _c_int, _c_int, _c_u64, _vp,
                                    _vp, _vp]),
    "tp_rank_rule": (_c_int, [_vp, _c_i64, _c_int, _c_int, _dbl, _vp, _vp]),
    "tp_rank_features": (_c_int, [_vp, _c_i64, _c_int, _vp, _vp]),
    "tp_mlp_param_count": (_c_int, []),
    "tp_mlp_round": (_c_int, [_vp, _vp, _vp]),
    "tp_mlp_forward": (_c_int, [_vp, _vp, _c_i64, _vp, _vp]),
    "tp_mlp_train_step": (_c_int, [_vp, _vp, _vp, _vp, _c_int, ctypes.c_float, _vp, _vp, _c_i64,
                                   _vp, _vp, _vp]),
    "tp_rdft3": (_c_int, [_vp, _c_i64, _c_i64, _vp, _vp, _vp]),
    "tp_irdft3": (_c_int, [_vp, _vp, _c_i64, _c_i64, _vp, _vp]),
    "tp_slice_norms": (_c_int, [_vp, _c_i64, _c_i64, _c_i64, _c_int, _vp, _vp, _vp]),
    "tp_sample_draw": (_c_int, [_vp, _vp, _c_i64, _c_i64, _c_u64, _c_int, _c_int, _c_u32, _vp,
                                _vp, _vp, _vp, _vp]),
    "tp_workspace_query": (ctypes.c_size_t, [_c_int, _vp, _c_int, _vp]),
    "tp_status_string": (ctypes.c_char_p, [_c_int]),
    "tp_last_error": (ctypes.c_char_p, []),
    "tp_release": (_c_int, []),
    "tp_sync_status": (_c_int, [_vp, _vp, _vp]),
    "tp_autotune_mode": (_c_int, [_c_int]),
    "tp_autotune_force": (_c_int, [_c_int]),
    "tp_autotune_count": (_c_int, []),
    "tp_autotune_entry": (_c_int, [_c_int, _vp, _c_int, _vp, _vp, _vp, _vp]),
    "tp_autotune_save": (_c_int, [ctypes.c_char_p]),
    "tp_autotune_load": (_c_int, [ctypes.c_char_p]),
    "tp_autotune_reset": (_c_int, []),
    "tp_launch_count": (_c_u64, []),
    "tp_version": (_c_int, []),
    "tp_profile_start": (_c_int, []),
    "tp_profile_stop": (_c_int, []),
    "tp_profile_entry": (_c_int, [_c_int, ctypes.c_char_p, _c_int, _vp, _vp]),
    "tp_profile_reset": (_c_int, []),
    "tp_slice_norms_noalloc": (_c_int, [_vp, _c_i64, _c_i64, _c_i64, _c_int, _vp, _vp]),
    "tp_slice_norms_noalloc_capacity": (ctypes.c_size_t, []),
    "tp_philox4x32_10": (_c_int, [_vp, _c_u32, _c_u32, _c_i64, _vp, _vp]),
}

_LIB = None
_LOCK = threading.Lock()


def lib_path() -> str:
    return os.environ.get("TPROD_LIB", os.path.join(_HERE, "libtprod.so"))


def lib():
    """The loaded library; raises if it has not been built."""
    global _LIB
    if _LIB is not None:
        return _LIB
    with _LOCK:
        if _LIB is None:
            path = lib_path()
            if not os.path.exists(path):
                raise TprodError(f"{path} is missing: build it with "
                                 "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _LIB = L
    return _LIB


def exported_symbols():
    return list(_SIGS)


TP_TUNE_OFF, TP_TUNE_ON = 0, 1


def autotune_mode(mode=-1) -> int:
    """Sets the autotuner mode (TP_TUNE_OFF / TP_TUNE_ON); returns the previous
    one (any other value only queries)."""
    return int(lib().tp_autotune_mode(int(mode)))


def autotune_force(candidate=-1) -> int:
    """Forces every tunable launch to one candidate (-1: stop forcing)."""
    return int(lib().tp_autotune_force(int(candidate)))


def autotune_table() -> list:
    """[(key, choice, candidates, best ms, default ms)] of the tuned launches."""
    L = lib()
    out = []
    buf = ctypes.create_string_buffer(512)
    for i in range(int(L.tp_autotune_count())):
        ch, nc = ctypes.c_int(), ctypes.c_int()
        best, dflt = ctypes.c_double(), ctypes.c_double()
        rc = L.tp_autotune_entry(i, ctypes.cast(buf, ctypes.c_void_p), 512,
                                 ctypes.cast(ctypes.byref(ch), ctypes.c_void_p),
                                 ctypes.cast(ctypes.byref(nc), ctypes.c_void_p),
                                 ctypes.cast(ctypes.byref(best), ctypes.c_void_p),
                                 ctypes.cast(ctypes.byref(dflt), ctypes.c_void_p))
        _check(rc, "tp_autotune_entry")
        out.append((buf.value.decode(), ch.value, nc.value, best.value, dflt.value))
    return out


def autotune_save(path):
    _check(lib().tp_autotune_save(str(path).encode()), "tp_autotune_save")


def autotune_load(path):
    _check(lib().tp_autotune_load(str(path).encode()), "tp_autotune_load")


def autotune_reset():
    _check(lib().tp_autotune_reset(), "tp_autotune_reset")


def sync_status(status=None) -> int:
    """Waits for the current stream; raises on an asynchronous CUDA error and
    returns the TP_DEV_* bits of the device status word `status` (0 without)."""
    torch = _torch()
    out = ctypes.c_int32(0)
    sd = _tensor_arg(status, "status", torch.int32) if status is not None else None
    rc = lib().tp_sync_status(_stream(), sd, ctypes.cast(ctypes.byref(out), ctypes.c_void_p)
                              if status is not None else None)
    _check(rc, "tp_sync_status")
    return int(out.value)


def launch_count() -> int:
    return int(lib().tp_launch_count())


def profile_start():
    L = lib()
    L.tp_profile_reset()
    _check(L.tp_profile_start(), "tp_profile_start")


def profile_stop() -> dict:
    """Stops timing; returns {kernel name: (total ms, launches)}."""
    L = lib()
    _check(L.tp_profile_stop(), "tp_profile_stop")
    out = {}
    i = 0
    buf = ctypes.create_string_buffer(128)
    while True:
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        if L.tp_profile_entry(i, buf, 128, ctypes.cast(ctypes.byref(ms), ctypes.c_void_p),
                              ctypes.cast(ctypes.byref(n), ctypes.c_void_p)) != 0:
            break
        out[buf.value.decode()] = (ms.value, n.value)
        i += 1
    return out


def _check(rc: int, what: str):
    if rc != 0:
        L = lib()
        raise TprodError(f"{what}: {L.tp_status_string(rc).decode()}: "
                         f"{L.tp_last_error().decode()}")


# ---------------------------------------------------------------- torch plumbing

def _torch():
    import torch
    if not torch.cuda.is_available():
        raise TprodError("libtprod needs a CUDA device; there is no CPU path")
    return torch


def empty_tensor(n1, n2, n3, dtype=None, device=None):
    """Uninitialised column-major tensor of logical shape (n1, n2, n3)."""
    torch = _torch()
    dtype = dtype or torch.float32
    device = device or torch.device("cuda", torch.cuda.current_device())
    return torch.empty((n3, n2, n1), dtype=dtype, device=device).permute(2, 1, 0)


def as_tprod_layout(x, dtype=None):
    """Column-major device copy of a (n1, n2, n3) array or tensor (no copy when
    it already is one)."""
    torch = _torch()
    dtype = dtype or torch.float32
    if isinstance(x, np.ndarray):
        x = torch.from_numpy(np.ascontiguousarray(np.transpose(x, (2, 1, 0))))
        x = x.to(device="cuda", dtype=dtype).permute(2, 1, 0)
        return x
    x = x.to(device="cuda", dtype=dtype)
    if _is_colmajor(x):
        return x
    return x.permute(2, 1, 0).contiguous().permute(2, 1, 0)


def _is_colmajor(x) -> bool:
    if x.dim() != 3:
        return False
    n1, n2, n3 = x.shape
    want = (1, n1, n1 * n2)
    return all(s == w or d == 1 for s, w, d in zip(x.stride(), want, x.shape))


def _tensor_arg(x, name, dtype=None):
    torch = _torch()
    dtype = dtype or torch.float32
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise TprodError(f"{name} must be a CUDA torch tensor")
    if x.dtype != dtype:
        raise TprodError(f"{name} must be {dtype}, got {x.dtype}")
    if x.dim() == 3 and not _is_colmajor(x):
        raise TprodError(f"{name} must be column-major (use as_tprod_layout)")
    if x.dim() != 3 and not x.is_contiguous():
        raise TprodError(f"{name} must be contiguous")
    return ctypes.c_void_p(x.data_ptr())


def _stream():
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


_WS = {}


def _opts(op, dims, precision=TP_FP32, status=None, max_sweeps=0, wait_limit=0):
    """tp_opts with a torch-allocated workspace large enough for this call."""
    torch = _torch()
    L = lib()
    d = (ctypes.c_int64 * len(dims))(*[int(v) for v in dims])
    o = TpOpts(int(precision), int(max_sweeps), None, 0, None, int(wait_limit))
    need = int(L.tp_workspace_query(op, ctypes.cast(d, ctypes.c_void_p), len(dims), ctypes.byref(o)))
    dev = torch.cuda.current_device()
    buf = _WS.get(dev)
    if need > 0 and (buf is None or buf.numel() < need):
        _WS[dev] = buf = torch.empty(max(need, 1 << 20), dtype=torch.uint8, device="cuda")
    if buf is not None and need > 0:
        o.workspace = buf.data_ptr()
        o.workspace_bytes = buf.numel()
    if status is not None:
        o.status = status.data_ptr()
    return o


# ---------------------------------------------------------------- entry points

def tprod(A, B, C=None, precision=TP_FP32, status=None, wait_limit=0):
    """C = A * B (Def. 2.1 / Algorithm 1).  ``status``: optional device int32
    tensor that receives TP_DEV_* bits.  ``wait_limit``: tp_opts'
    pipeline_wait_limit (a failure-detection test hook; 0 = default)."""
    n1, n2, n3 = A.shape
    n2b, n4, n3b = B.shape
    if n2b != n2 or n3b != n3:
        raise TprodError(f"tprod: shapes {tuple(A.shape)} and {tuple(B.shape)} do not chain")
    if C is None:
        C = empty_tensor(n1, n4, n3, device=A.device)
    o = _opts(TP_OP_TPROD, (n1, n2, n4, n3), precision, status, wait_limit=wait_limit)
    rc = lib().tprod(_tensor_arg(A, "A"), _tensor_arg(B, "B"), _tensor_arg(C, "C"),
                     n1, n2, n4, n3, ctypes.byref(o), _stream())
    _check(rc, "tprod")
    return C


def tprod_sampled(A, B, c, seed=0, prob_mode=TP_PROB_AB, p_given=None, precision=TP_FP32,
                  Z=None, idx=None, count=None, status=None, sample_mode=TP_SAMPLE_BERNOULLI):
    """rt-product (Algorithm 2).  Returns (Z, idx int32[n2], count int64[1]);
    idx[:count] are the kept slice indices, ascending (Bernoulli) or in draw
    order (TP_SAMPLE_IID)."""
    torch = _torch()
    n1, n2, n3 = A.shape
    n2b, n4, n3b = B.shape
    if n2b != n2 or n3b != n3:
        raise TprodError("tprod_sampled: shapes do not chain")
    if Z is None:
        Z = empty_tensor(n1, n4, n3, device=A.device)
    if idx is None:
        idx = torch.empty(n2, dtype=torch.int32, device=A.device)
    if count is None:
        count = torch.empty(1, dtype=torch.int64, device=A.device)
    pg = None
    if prob_mode == TP_PROB_GIVEN:
        if p_given is None or p_given.numel() != n2:
            raise TprodError("tprod_sampled: TP_PROB_GIVEN needs p_given of length n2")
        pg = _tensor_arg(p_given, "p_given", torch.float64)
    o = _opts(TP_OP_TPROD_SAMPLED, (n1, n2, n4, n3), precision, status)
    rc = lib().tprod_sampled(_tensor_arg(A, "A"), _tensor_arg(B, "B"), _tensor_arg(Z, "Z"),
                             n1, n2, n4, n3, int(c), int(seed) & ((1 << 64) - 1), int(prob_mode),
                             int(sample_mode), pg, _tensor_arg(idx, "idx", torch.int32),
                             _tensor_arg(count, "count", torch.int64), ctypes.byref(o), _stream())
    _check(rc, "tprod_sampled")
    return Z, idx, count


def tsvd(X, max_sweeps=0, status=None):
    """Economy t-SVD (Theorem 2.6): returns (U, S, V)."""
    n1, n2, n3 = X.shape
    m = min(n1, n2)
    U = empty_tensor(n1, m, n3, device=X.device)
    S = empty_tensor(m, m, n3, device=X.device)
    V = empty_tensor(n2, m, n3, device=X.device)
    o = _opts(TP_OP_TSVD, (n1, n2, n3), TP_FP32, status, max_sweeps)
    rc = lib().tsvd(_tensor_arg(X, "X"), n1, n2, n3, _tensor_arg(U, "U"), _tensor_arg(S, "S"),
                    _tensor_arg(V, "V"), ctypes.byref(o), _stream())
    _check(rc, "tsvd")
    return U, S, V


def tsvd_randomized(X, k, p=10, q=2, seed=0, status=None, max_sweeps=0, ranks=None,
                    sketch=0, precision=TP_FP32, sketch_sizes=None):
    """Randomized tubal-rank-k t-SVD: returns (U, S, V).  ranks: optional
    device int32[n3 // 2 + 1] per-frequency ranks (each at most k);
    sketch_sizes: optional device int32[n3 // 2 + 1] per-frequency sketch
    sizes (each at most k + p); sketch: TP_SKETCH_SIGNS (0) or
    TP_SKETCH_SLICES (1, picked lateral slices); precision: TP_FP32 (products
    on the CUDA cores) or TP_TF32X3 / TP_BF16X3 (the products with X_hat on
    the tensor cores, split operands)."""
    torch = _torch()
    n1, n2, n3 = X.shape
    rk = sz = None
    if ranks is not None:
        if ranks.numel() != n3 // 2 + 1:
            raise TprodError("tsvd_randomized: ranks needs n3 // 2 + 1 entries")
        rk = _tensor_arg(ranks, "ranks", torch.int32)
    if sketch_sizes is not None:
        if sketch_sizes.numel() != n3 // 2 + 1:
            raise TprodError("tsvd_randomized: sketch_sizes needs n3 // 2 + 1 entries")
        sz = _tensor_arg(sketch_sizes, "sketch_sizes", torch.int32)
    U = empty_tensor(n1, k, n3, device=X.device)
    S = empty_tensor(k, k, n3, device=X.device)
    V = empty_tensor(n2, k, n3, device=X.device)
    o = _opts(TP_OP_TSVD_RANDOMIZED, (n1, n2, n3, k, p), precision, status, max_sweeps)
    rc = lib().tsvd_randomized(_tensor_arg(X, "X"), n1, n2, n3, int(k), int(p), int(q),
                               int(seed) & ((1 << 64) - 1), int(sketch), rk, sz,
                               _tensor_arg(U, "U"),
                               _tensor_arg(S, "S"), _tensor_arg(V, "V"), ctypes.byref(o),
                               _stream())
    _check(rc, "tsvd_randomized")
    return U, S, V


def tcomplete_svt(X, mask, iters, L=None, E=None, Y=None, mu=None, mu0=1e-3, rho=1.1,
                  mu_max=1e10, status=None, max_sweeps=0, precision=TP_FP32):
    """ADMM completion (Algorithm 7, problem tlow6).  State (L, E, Y, mu) is
    updated in place and returned.  precision: TP_FP32, or TP_TF32X3 /
    TP_BF16X3 for the SVT's three GEMMs on the tensor cores."""
    torch = _torch()
    n1, n2, n3 = X.shape
    if L is None:
        L = torch.zeros_like(X)
        E = torch.zeros_like(X)
        Y = torch.zeros_like(X)
    if mu is None:
        mu = torch.full((1,), float(mu0), dtype=torch.float64, device=X.device)
    o = _opts(TP_OP_TCOMPLETE_SVT, (n1, n2, n3), precision, status, max_sweeps)
    rc = lib().tcomplete_svt(_tensor_arg(X, "X"), _tensor_arg(mask, "mask", torch.uint8),
                             n1, n2, n3, int(iters), float(rho), float(mu_max),
                             _tensor_arg(L, "L"), _tensor_arg(E, "E"), _tensor_arg(Y, "Y"),
                             _tensor_arg(mu, "mu", torch.float64), ctypes.byref(o), _stream())
    _check(rc, "tcomplete_svt")
    return L, E, Y, mu


def trpca_admm(X, iters, lam=0.0, L=None, E=None, Y=None, mu=None, mu0=1e-3, rho=1.1,
               mu_max=1e10, status=None, max_sweeps=0, precision=TP_FP32):
    """Robust TNN (Algorithm 7, problem tlow7); lam <= 0 takes the default
    1/sqrt(max(n1, n2) n3).  State (L, E, Y, mu) updated in place and returned."""
    torch = _torch()
    n1, n2, n3 = X.shape
    if L is None:
        L = torch.zeros_like(X)
        E = torch.zeros_like(X)
        Y = torch.zeros_like(X)
    if mu is None:
        mu = torch.full((1,), float(mu0), dtype=torch.float64, device=X.device)
    o = _opts(TP_OP_TRPCA, (n1, n2, n3), precision, status, max_sweeps)
    rc = lib().trpca_admm(_tensor_arg(X, "X"), n1, n2, n3, int(iters), float(lam), float(rho),
                          float(mu_max), _tensor_arg(L, "L"), _tensor_arg(E, "E"),
                          _tensor_arg(Y, "Y"), _tensor_arg(mu, "mu", torch.float64),
                          ctypes.byref(o), _stream())
    _check(rc, "trpca_admm")
    return L, E, Y, mu


def tcomplete_svt_batched(tensors, iters, rho=1.1, mu_max=1e10, status=None, max_sweeps=0,
                          precision=TP_FP32):
    """tcomplete_svt over a list of independent tensors of possibly different
    sizes: each item is a tuple (X, mask, L, E, Y, mu) of device tensors
    (column-major layout, mask uint8, mu a float64 1-element tensor), updated
    in place.  Returns the list."""
    torch = _torch()
    descs = (TpTensorDesc * len(tensors))()
    dims = []
    for i, (X, mask, L, E, Y, mu) in enumerate(tensors):
        n1, n2, n3 = X.shape
        descs[i] = TpTensorDesc(_tensor_arg(X, "X").value,
                                _tensor_arg(mask, "mask", torch.uint8).value,
                                _tensor_arg(L, "L").value, _tensor_arg(E, "E").value,
                                _tensor_arg(Y, "Y").value,
                                _tensor_arg(mu, "mu", torch.float64).value, n1, n2, n3)
        dims += [n1, n2, n3]
    o = _opts(TP_OP_TCOMPLETE_SVT_BATCHED, dims, precision, status, max_sweeps)
    rc = lib().tcomplete_svt_batched(len(tensors), ctypes.cast(descs, ctypes.c_void_p), int(iters),
                                     float(rho), float(mu_max), ctypes.byref(o), _stream())
    _check(rc, "tcomplete_svt_batched")
    return tensors


def sketch_spectrum(X, l, q=2, seed=0, status=None):
    """Singular values of the randomized sketch of every half-spectrum
    frequency: (h, l) float32 device tensor, rows descending."""
    torch = _torch()
    n1, n2, n3 = X.shape
    sig = torch.empty((n3 // 2 + 1, l), dtype=torch.float32, device=X.device)
    o = _opts(TP_OP_SKETCH_SPECTRUM, (n1, n2, n3, l), TP_FP32, status)
    rc = lib().tp_sketch_spectrum(_tensor_arg(X, "X"), n1, n2, n3, int(l), int(q), int(seed),
                                  _tensor_arg(sig, "sig"), ctypes.byref(o), _stream())
    _check(rc, "tp_sketch_spectrum")
    return sig


def rank_rule(sig, cap, tol=1e-2):
    """Per-frequency ranks (int32 device tensor) from (h, l) spectra."""
    torch = _torch()
    h, l = sig.shape
    out = torch.empty(h, dtype=torch.int32, device=sig.device)
    rc = lib().tp_rank_rule(_tensor_arg(sig, "sig"), h, l, int(cap), float(tol),
                            _tensor_arg(out, "rank", torch.int32), _stream())
    _check(rc, "tp_rank_rule")
    return out


def rank_features(sig):
    """(h, 16) float16 predictor features from (h, >= 17) spectra."""
    torch = _torch()
    h, l = sig.shape
    out = torch.empty((h, 16), dtype=torch.float16, device=sig.device)
    rc = lib().tp_rank_features(_tensor_arg(sig, "sig"), h, l,
                                _tensor_arg(out, "features", torch.float16), _stream())
    _check(rc, "tp_rank_features")
    return out


def mlp_param_count():
    return int(lib().tp_mlp_param_count())


def mlp_round(theta, w16=None):
    """float16 copy of the float32 master parameters."""
    torch = _torch()
    if w16 is None:
        w16 = torch.empty(theta.shape, dtype=torch.float16, device=theta.device)
    rc = lib().tp_mlp_round(_tensor_arg(theta, "theta"), _tensor_arg(w16, "w16", torch.float16),
                            _stream())
    _check(rc, "tp_mlp_round")
    return w16


def mlp_forward(w16, x16):
    torch = _torch()
    B = x16.shape[0]
    y = torch.empty((B, 2), dtype=torch.float32, device=x16.device)
    rc = lib().tp_mlp_forward(_tensor_arg(w16, "w16", torch.float16),
                              _tensor_arg(x16, "x", torch.float16), B, _tensor_arg(y, "y"),
                              _stream())
    _check(rc, "tp_mlp_forward")
    return y


def mlp_train_step(theta, w16, m, v, step, lr, x16, target, grad=None):
    """Gradient and loss at w16 on the batch (returned: float32 tensor of
    param_count + 1, the last the loss), then one Adam step if lr > 0."""
    torch = _torch()
    B = x16.shape[0]
    if grad is None:
        grad = torch.empty(mlp_param_count() + 1, dtype=torch.float32, device=x16.device)
    o = _opts(TP_OP_MLP_TRAIN, (B,))
    rc = lib().tp_mlp_train_step(_tensor_arg(theta, "theta"), _tensor_arg(w16, "w16", torch.float16),
                                 _tensor_arg(m, "m"), _tensor_arg(v, "v"), int(step), float(lr),
                                 _tensor_arg(x16, "x", torch.float16), _tensor_arg(target, "target"),
                                 B, _tensor_arg(grad, "grad"), ctypes.byref(o), _stream())
    _check(rc, "tp_mlp_train_step")
    return grad


def tcx(A, c, seed=0, prob_mode=TP_PROB_A2, p_given=None, status=None):
    """t-CX (Algorithm 4): returns (Z = C * C^dagger * A, idx, count)."""
    torch = _torch()
    n1, n2, n3 = A.shape
    Z = empty_tensor(n1, n2, n3, device=A.device)
    idx = torch.empty(n2, dtype=torch.int32, device=A.device)
    count = torch.empty(1, dtype=torch.int64, device=A.device)
    pg = _tensor_arg(p_given, "p_given", torch.float64) if prob_mode == TP_PROB_GIVEN else None
    o = _opts(TP_OP_TCX, (n1, n2, n3), TP_FP32, status)
    rc = lib().tcx(_tensor_arg(A, "A"), n1, n2, n3, int(c), int(seed) & ((1 << 64) - 1),
                   int(prob_mode), pg, _tensor_arg(Z, "Z"), _tensor_arg(idx, "idx", torch.int32),
                   _tensor_arg(count, "count", torch.int64), ctypes.byref(o), _stream())
    _check(rc, "tcx")
    return Z, idx, count


def tcur(A, c, l, seed=0, prob_mode=TP_PROB_A2, p_cols=None, p_rows=None, rank=0, status=None):
    """t-CUR (Algorithm 5): returns (Z, col_idx, col_count, row_idx, row_count,
    row_prob); row_prob is the (top-rank) row leverage of C unless p_rows is
    given."""
    torch = _torch()
    n1, n2, n3 = A.shape
    Z = empty_tensor(n1, n2, n3, device=A.device)
    cidx = torch.empty(n2, dtype=torch.int32, device=A.device)
    ccnt = torch.empty(1, dtype=torch.int64, device=A.device)
    ridx = torch.empty(n1, dtype=torch.int32, device=A.device)
    rcnt = torch.empty(1, dtype=torch.int64, device=A.device)
    prob = torch.empty(n1, dtype=torch.float64, device=A.device)
    pc = _tensor_arg(p_cols, "p_cols", torch.float64) if prob_mode == TP_PROB_GIVEN else None
    pr = _tensor_arg(p_rows, "p_rows", torch.float64) if p_rows is not None else None
    o = _opts(TP_OP_TCUR, (n1, n2, n3), TP_FP32, status)
    rc = lib().tcur(_tensor_arg(A, "A"), n1, n2, n3, int(c), int(l), int(rank),
                    int(seed) & ((1 << 64) - 1),
                    int(prob_mode), pc, pr, _tensor_arg(Z, "Z"),
                    _tensor_arg(cidx, "col_idx", torch.int32),
                    _tensor_arg(ccnt, "col_count", torch.int64),
                    _tensor_arg(ridx, "row_idx", torch.int32),
                    _tensor_arg(rcnt, "row_count", torch.int64),
                    _tensor_arg(prob, "row_prob", torch.float64), ctypes.byref(o), _stream())
    _check(rc, "tcur")
    return Z, cidx, ccnt, ridx, rcnt, prob


def cur_tnn(X, c, l, iters, seed=0, rank=0, mask=None, lam=0.0, prob_mode=TP_PROB_A2,
            p_cols=None, p_rows=None, pinv_rtol=1e-4, mu0=1e-3, rho=1.1, mu_max=1e10,
            status=None, max_sweeps=0):
    """CUR t-NN (Algorithm 6): returns (L, Ct, Rt, col_idx, col_count, row_idx,
    row_count, row_prob); Ct and Rt are the ADMM solutions on the picked
    lateral (n1 x c' x n3) and horizontal (l' x n2 x n3) slices, as
    column-major tensors."""
    torch = _torch()
    n1, n2, n3 = X.shape
    dev = X.device
    L = empty_tensor(n1, n2, n3, device=dev)
    ct = torch.empty(n1 * n2 * n3, dtype=torch.float32, device=dev)
    rt = torch.empty(n1 * n2 * n3, dtype=torch.float32, device=dev)
    cidx = torch.empty(n2, dtype=torch.int32, device=dev)
    ccnt = torch.empty(1, dtype=torch.int64, device=dev)
    ridx = torch.empty(n1, dtype=torch.int32, device=dev)
    rcnt = torch.empty(1, dtype=torch.int64, device=dev)
    prob = torch.empty(n1, dtype=torch.float64, device=dev)
    mk = _tensor_arg(mask, "mask", torch.uint8) if mask is not None else None
    pc = _tensor_arg(p_cols, "p_cols", torch.float64) if prob_mode == TP_PROB_GIVEN else None
    pr = _tensor_arg(p_rows, "p_rows", torch.float64) if p_rows is not None else None
    o = _opts(TP_OP_CUR_TNN, (n1, n2, n3), TP_FP32, status, max_sweeps)
    rc = lib().cur_tnn(_tensor_arg(X, "X"), mk, n1, n2, n3, int(c), int(l), int(rank),
                       int(seed) & ((1 << 64) - 1), int(prob_mode), pc, pr, int(iters),
                       float(lam), float(mu0), float(rho), float(mu_max), float(pinv_rtol),
                       _tensor_arg(L, "L"), _tensor_arg(ct, "Ct"), _tensor_arg(rt, "Rt"),
                       _tensor_arg(cidx, "col_idx", torch.int32),
                       _tensor_arg(ccnt, "col_count", torch.int64),
                       _tensor_arg(ridx, "row_idx", torch.int32),
                       _tensor_arg(rcnt, "row_count", torch.int64),
                       _tensor_arg(prob, "row_prob", torch.float64), ctypes.byref(o), _stream())
    _check(rc, "cur_tnn")
    cp, lp = int(ccnt.item()), int(rcnt.item())
    Ct = ct[: n1 * cp * n3].view(n3, cp, n1).permute(2, 1, 0)
    Rt = rt[: lp * n2 * n3].view(n3, n2, lp).permute(2, 1, 0)
    return L, Ct, Rt, cidx, ccnt, ridx, rcnt, prob


def rdft3(X):
    """Half-spectrum DFT along mode 3: returns (Xr, Xi), each (n1, n2, h)."""
    n1, n2, n3 = X.shape
    h = n3 // 2 + 1
    Xr = empty_tensor(n1, n2, h, device=X.device)
    Xi = empty_tensor(n1, n2, h, device=X.device)
    rc = lib().tp_rdft3(_tensor_arg(X, "X"), n1 * n2, n3, _tensor_arg(Xr, "Xr"),
                        _tensor_arg(Xi, "Xi"), _stream())
    _check(rc, "tp_rdft3")
    return Xr, Xi


def irdft3(Xr, Xi, n3):
    n1, n2, h = Xr.shape
    if h != n3 // 2 + 1:
        raise TprodError("irdft3: spectrum length does not match n3")
    out = empty_tensor(n1, n2, n3, device=Xr.device)
    rc = lib().tp_irdft3(_tensor_arg(Xr, "Xr"), _tensor_arg(Xi, "Xi"), n1 * n2, n3,
                         _tensor_arg(out, "out"), _stream())
    _check(rc, "tp_irdft3")
    return out


def slice_norms(X, which):
    """Squared Frobenius norms: which=0 lateral (n2 values), 1 horizontal (n1)."""
    torch = _torch()
    n1, n2, n3 = X.shape
    out = torch.empty(n2 if which == 0 else n1, dtype=torch.float64, device=X.device)
    o = _opts(TP_OP_SLICE_NORMS, (n1, n2, n3))
    rc = lib().tp_slice_norms(_tensor_arg(X, "X"), n1, n2, n3, int(which),
                              _tensor_arg(out, "out", torch.float64), ctypes.byref(o), _stream())
    _check(rc, "tp_slice_norms")
    return out


def slice_norms_noalloc(X, which, out=None):
    """Slice norms through tp_slice_norms_noalloc: the library allocates
    nothing (its scratch is a fixed device array), for callers that cannot
    allocate; ``out`` may be passed in so that this call allocates nothing
    either."""
    torch = _torch()
    n1, n2, n3 = X.shape
    if out is None:
        out = torch.empty(n2 if which == 0 else n1, dtype=torch.float64, device=X.device)
    rc = lib().tp_slice_norms_noalloc(_tensor_arg(X, "X"), n1, n2, n3, int(which),
                                      _tensor_arg(out, "out", torch.float64), _stream())
    _check(rc, "tp_slice_norms_noalloc")
    return out


def philox4x32_10(counters, k0, k1):
    """Philox4x32-10 words of the counters (an (n, 4) array of uint32 values,
    word 0 first) under key (k0, k1); returns an (n, 4) numpy uint32 array."""
    torch = _torch()
    ctr = np.ascontiguousarray(np.asarray(counters, dtype=np.uint32).reshape(-1, 4))
    n = ctr.shape[0]
    c_dev = torch.from_numpy(ctr.view(np.int32)).to("cuda")
    out = torch.empty((n, 4), dtype=torch.int32, device="cuda")
    _check(lib().tp_philox4x32_10(c_dev.data_ptr(), int(k0) & 0xFFFFFFFF, int(k1) & 0xFFFFFFFF,
                                  n, out.data_ptr(), _stream()), "tp_philox4x32_10")
    return out.cpu().numpy().view(np.uint32)


def sample_draw(w, w2, c, seed, prob_mode, stream_id=0, sample_mode=TP_SAMPLE_BERNOULLI):
    """Picking loop of Algorithm 2.  Returns (idx, scale, count, q)."""
    torch = _torch()
    n = w.numel()
    idx = torch.empty(n, dtype=torch.int32, device=w.device)
    scale = torch.empty(n, dtype=torch.float32, device=w.device)
    count = torch.empty(1, dtype=torch.int64, device=w.device)
    q = torch.empty(n, dtype=torch.float64, device=w.device)
    rc = lib().tp_sample_draw(_tensor_arg(w, "w", torch.float64),
                              _tensor_arg(w2, "w2", torch.float64) if w2 is not None else None,
                              n, int(c), int(seed) & ((1 << 64) - 1), int(prob_mode),
                              int(sample_mode), int(stream_id),
                              _tensor_arg(idx, "idx", torch.int32),
                              _tensor_arg(scale, "scale", torch.float32),
                              _tensor_arg(count, "count", torch.int64),
                              _tensor_arg(q, "q", torch.float64), _stream())
    _check(rc, "tp_sample_draw")
    return idx, scale, count, q
