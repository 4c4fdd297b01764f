#!/usr/bin/env python
"""Throughput of the sampled t-product hot path (Algorithm 2) on one GB300.

Workload (synthetic, seeded): A 2000 x 4000 x 64 and B 4000 x 1500 x 64, each
the t-product of N(0,1) factors at tubal rank 20 plus Gaussian noise of 1% of
its RMS; c = 400, probabilities proportional to ||A(:,j,:)|| ||B(j,:,:)||,
Philox seed 0.  One step = one tprod_sampled call: slice norms of A and B,
probabilities and Bernoulli picks, rescaled gathers fused into the mode-3
DFTs, facewise complex GEMMs of the 33 half-spectrum slices, inverse DFT.
The timed form (--precision, default bf16x3) runs the facewise GEMMs on the
tensor cores with each operand split into a bf16 hi + lo pair and float32
accumulation; the 3xTF32 split and the plain FP32 form are timed beside it
(--compare).  All three are held to relative error 1e-5 against the float64
oracle at this workload by tests/test_gpu_fullsize.py.

metric  "t-product TFLOP/s": nominal facewise-GEMM flops of the step
        (8 n1 c' n4 per complex slice, 2 n1 c' n4 per real slice) divided by
        the step time; inputs (3.6 GB) are larger than L2 and are streamed
        every step.
e2e     the same metric through the C entry point with host buffers: every
        step's A and B copied from pinned host memory and its Z copied back
        inside the timed region (steps pipelined over two device buffer sets).
Multi-GPU: every rank runs its own replica (weak scaling, no collective).
--impl reference times the float64 oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N1, N2, N4, N3, RANK_T, NOISE, C_SAMPLES, SEED = 2000, 4000, 1500, 64, 20, 0.01, 400, 0
CPU_SAMPLE = 1000  # rows of A and columns of B the CPU baseline sample keeps


def use_small_case():
    """--small: a 600 x 1600 x 64 * 1600 x 500 x 64 case (each input still
    larger than L2, under 2 GB on the device with workspace) for profiler
    captures only; never a bench number."""
    global N1, N2, N4, CPU_SAMPLE
    N1, N2, N4, CPU_SAMPLE = 600, 1600, 500, 200


def gemm_flops(n1, cprime, n4, n3):
    h = n3 // 2 + 1
    real = 2 if n3 % 2 == 0 else 1
    return 8.0 * n1 * cprime * n4 * (h - real) + 2.0 * n1 * cprime * n4 * real


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "sm_max_mhz": float(d.get("sm_max_mhz", 2070.0)), "src": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0, "src": "fallback"}


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        # samples under load: the upper half by power draw
        order = sorted(range(len(sm)), key=lambda i: power[i])
        loaded = [sm[i] for i in order[len(order) // 2:]] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power)}


def host_array(x):
    """Column-major torch tensor (n1, n2, n3) -> float64 numpy (n1, n2, n3)."""
    return x.permute(2, 1, 0).contiguous().cpu().numpy().astype(np.float64).transpose(2, 1, 0)


def run_oracle_sample(A, B, seed, keep_output=False):
    """Times the float64 oracle on the bounded sample A[:S], B[:, :S] (same
    inner dimension n2 = 4000, n3 = 64, c = 400).  Returns (seconds, flops)
    or, with keep_output, (seconds, flops, Z, picked indices)."""
    from oracle import sampling_ref
    S = CPU_SAMPLE
    As = host_array(A[:S])
    Bs = host_array(B[:, :S])
    t0 = time.perf_counter()
    Z, idx, _ = sampling_ref.tprod_sampled(As, Bs, C_SAMPLES, seed)
    dt = time.perf_counter() - t0
    if keep_output:
        return dt, gemm_flops(S, len(idx), S, N3), Z, np.asarray(idx)
    return dt, gemm_flops(S, len(idx), S, N3)


def sample_errors(tp, torch, A, B, Zref, idx_ref, precisions):
    """Relative Frobenius error of each GPU form against the float64 oracle's
    output on the CPU-baseline sample (A[:S], B[:, :S]: the same n2 = 4000
    inner dimension, n3 = 64 and c = 400 as the timed workload, so the same
    number of picked slices enters every sum), and whether the picks agree."""
    S = CPU_SAMPLE
    As = tp.as_tprod_layout(A[:S])
    Bs = tp.as_tprod_layout(B[:, :S])
    ref = torch.from_numpy(np.ascontiguousarray(Zref.transpose(2, 1, 0)))   # (n3, n4, n1)
    den = float(torch.linalg.vector_norm(ref))
    out = {}
    for name, pr in precisions.items():
        Z, idx, cnt = tp.tprod_sampled(As, Bs, C_SAMPLES, seed=SEED, precision=pr)
        got = Z.permute(2, 1, 0).double().cpu()
        picks_equal = bool(np.array_equal(idx[: int(cnt.item())].cpu().numpy(), idx_ref))
        out[name] = {"rel_err": float(torch.linalg.vector_norm(got - ref)) / den,
                     "picks_equal": picks_equal}
        del Z, got
    return out


RSVD_K, RSVD_P, RSVD_Q = 40, 10, 2


def reduce_max(value, dist, device):
    """Largest value over the ranks (the job's time is its slowest rank)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def time_gpu(fn, reps, torch):
    """Mean milliseconds of fn() over reps calls, CUDA events on the current stream."""
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fn()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def bench_rows(tp, torch, with_cpu):
    """The other rows of the hot path, each timed on the GPU through the C ABI
    with the float64 oracle timed beside it on the host cores:
      tsvd   t-SVD (Theorem 2.6) of the 64 x 48 x 16 iid N(0,1) tensor
      tcx    t-CX (Algorithm 4), 256 x 512 x 32 tubal rank 10 + 1% noise, c = 64
      tcur   t-CUR (Algorithm 5), the same tensor, c = 64, l = 64, leverage rows
      svt    completion ADMM (Algorithm 7), one 144 x 256 x 80 video (tubal rank
             10, sigma 0.01, 50% observed; the paper's video shape), 10 iterations
      trpca  robust ADMM (Algorithm 7 as printed), 192 x 168 x 64, 30 iterations
      cur_tnn  CUR t-NN (Algorithm 6) on a face-stack-shaped 192 x 1140 x 168
             tensor (tubal rank 10, 10% spikes), c = 228, l = 96, rank 10, 30
             ADMM iterations, beside the full robust ADMM on the same tensor"""
    from paper_1704_04362_gb300 import synth
    rows = {}
    X = synth.iid_normal((64, 48, 16), seed=0)
    Xd = tp.as_tprod_layout(X)
    ms = time_gpu(lambda: tp.tsvd(Xd), 20, torch)
    rows["tsvd"] = {"workload": "64x48x16 iid N(0,1)", "gpu_ms": ms}
    A = synth.lowrank_np(256, 512, 32, 10, seed=3, noise=0.01)
    Ad = tp.as_tprod_layout(A)
    ms = time_gpu(lambda: tp.tcx(Ad, 64, seed=0), 10, torch)
    rows["tcx"] = {"workload": "256x512x32 tubal rank 10 + 1% noise, c = 64", "gpu_ms": ms}
    ms = time_gpu(lambda: tp.tcur(Ad, 64, 64, seed=0), 10, torch)
    Zc = tp.tcur(Ad, 64, 64, seed=0)[0]
    Adn = torch.linalg.vector_norm(Ad)
    rows["tcur"] = {"workload": "256x512x32 tubal rank 10 + 1% noise, c = 64, l = 64",
                    "gpu_ms": ms,
                    "relative_error": float(torch.linalg.vector_norm(Zc - Ad) / Adn)}
    truth, noisy, mask = synth.video_np(144, 256, 80, r=10, seed=0)
    Xv = tp.as_tprod_layout(noisy)
    Mv = tp.as_tprod_layout(mask, torch.uint8)
    iters = 10

    def run_svt():
        tp.tcomplete_svt(Xv, Mv, iters)
    ms = time_gpu(run_svt, 2, torch)
    rows["svt"] = {"workload": "144x256x80 video, tubal rank 10, 50% observed", "iterations": iters,
                   "gpu_ms": ms, "gpu_iterations_per_s": iters / (ms * 1e-3)}
    # robust TNN (Algorithm 7 as printed): a face-stack-shaped tensor, 192 x 168
    # pixels x 64 images, tubal rank 10, 10% of the entries corrupted by spikes
    L0 = synth.lowrank_np(192, 168, 64, 10, seed=12)
    L0 = L0 / np.sqrt(np.mean(L0.astype(np.float64) ** 2))
    gsp = np.random.default_rng(13)
    Xr_np = (L0 + np.where(gsp.random(L0.shape) < 0.1, 5.0 * gsp.standard_normal(L0.shape),
                           0.0)).astype(np.float32)
    Xrd = tp.as_tprod_layout(Xr_np)
    r_iters = 30

    def run_rpca():
        tp.trpca_admm(Xrd, r_iters)
    ms = time_gpu(run_rpca, 2, torch)
    Lr_gpu = tp.trpca_admm(Xrd, r_iters)[0]
    L0d = tp.as_tprod_layout(L0.astype(np.float32))
    rows["trpca"] = {"workload": "192x168x64 tubal rank 10 + 10% spikes (scale 5)",
                     "iterations": r_iters, "gpu_ms": ms,
                     "gpu_iterations_per_s": r_iters / (ms * 1e-3),
                     "relative_error_to_low_rank": float(torch.linalg.vector_norm(Lr_gpu - L0d) /
                                                         torch.linalg.vector_norm(L0d))}
    # CUR t-NN against the full robust ADMM on the same tensor (the shape of
    # the paper's face experiment: 192 x 168 pixels as 192 rows x (38 people x
    # 30 images) lateral slices, n3 = 168 columns)
    F0 = synth.lowrank_np(192, 1140, 168, 10, seed=14)
    F0 = F0 / np.sqrt(np.mean(F0.astype(np.float64) ** 2))
    gsf = np.random.default_rng(15)
    Xf = (F0 + np.where(gsf.random(F0.shape) < 0.1, 5.0 * gsf.standard_normal(F0.shape),
                        0.0)).astype(np.float32)
    Xfd = tp.as_tprod_layout(Xf)
    F0d = tp.as_tprod_layout(F0.astype(np.float32))
    f_iters = 30
    ms = time_gpu(lambda: tp.cur_tnn(Xfd, 228, 96, f_iters, seed=0, rank=10), 2, torch)
    out = tp.cur_tnn(Xfd, 228, 96, f_iters, seed=0, rank=10)
    ms_full = time_gpu(lambda: tp.trpca_admm(Xfd, f_iters), 1, torch)
    Lfull = tp.trpca_admm(Xfd, f_iters)[0]
    F0n = torch.linalg.vector_norm(F0d)
    rows["cur_tnn"] = {"workload": "192x1140x168 tubal rank 10 + 10% spikes (scale 5), "
                                   "c = 228, l = 96, rank 10",
                       "iterations": f_iters, "gpu_ms": ms,
                       "picked": [int(out[4].item()), int(out[6].item())],
                       "relative_error_to_low_rank": float(torch.linalg.vector_norm(out[0] - F0d) / F0n),
                       "full_admm_gpu_ms": ms_full,
                       "full_admm_relative_error": float(torch.linalg.vector_norm(Lfull - F0d) / F0n)}
    del out, Lfull
    if with_cpu:
        from oracle import completion_ref, decomp_ref
        t0 = time.perf_counter()
        decomp_ref.tsvd(X.astype(np.float64))
        rows["tsvd"]["oracle_ms"] = (time.perf_counter() - t0) * 1e3
        t0 = time.perf_counter()
        decomp_ref.tcx(A.astype(np.float64), 64, 0)
        rows["tcx"]["oracle_ms"] = (time.perf_counter() - t0) * 1e3
        t0 = time.perf_counter()
        decomp_ref.tcur(A.astype(np.float64), 64, 64, 0)
        rows["tcur"]["oracle_ms"] = (time.perf_counter() - t0) * 1e3
        t0 = time.perf_counter()
        completion_ref.tcomplete_svt(noisy.astype(np.float64), mask.astype(bool), 2)
        per_iter = (time.perf_counter() - t0) / 2
        rows["svt"]["oracle_ms"] = per_iter * iters * 1e3
        rows["svt"]["oracle_sample"] = "2 oracle iterations timed, scaled to 10"
        t0 = time.perf_counter()
        completion_ref.trpca(Xr_np.astype(np.float64), 2)
        rows["trpca"]["oracle_ms"] = (time.perf_counter() - t0) / 2 * r_iters * 1e3
        rows["trpca"]["oracle_sample"] = "2 oracle iterations timed, scaled to 30"
        # CUR t-NN: the whole oracle with 2 ADMM iterations, plus 28 more
        # iterations of its two ADMM runs timed one by one
        t0 = time.perf_counter()
        _, Ct2, Rt2, *_ = decomp_ref.cur_tnn(Xf.astype(np.float64), 228, 96, 0, 2, r=10)
        t2 = time.perf_counter() - t0
        t0 = time.perf_counter()
        completion_ref.trpca(Xf.astype(np.float64)[:, :Ct2.shape[1], :], 1)
        completion_ref.trpca(Xf.astype(np.float64)[:Rt2.shape[0], :, :], 1)
        t1 = time.perf_counter() - t0
        rows["cur_tnn"]["oracle_ms"] = (t2 + (f_iters - 2) * t1) * 1e3
        rows["cur_tnn"]["oracle_sample"] = ("the oracle with 2 ADMM iterations, plus 28 x one "
                                            "iteration of each ADMM run on same-sized slices")
    for r in rows.values():
        if "oracle_ms" in r:
            r["speedup_vs_oracle"] = r["oracle_ms"] / r["gpu_ms"]
    return rows


def bench_svt_batched(tp, torch, count=256, iters=100, precision="fp32", sizes=None):
    """The batched completion workload: `count` videos of uneven size (H, W, T
    drawn uniformly from 64..480 x 64..360 x 16..120, PCG64 seed 0), each
    tubal rank 10 (N(0,1) factors) at unit RMS plus sigma = 0.01 noise, 50%
    observed uniformly at random; tcomplete_svt_batched from L = E = Y = 0,
    mu0 = 1e-3, `iters` iterations in one call.  The first iteration runs
    directly (cold slice Jacobi), the later ones replay one captured CUDA
    graph of an iteration over all tensors; the library's profiler times the
    replays as one region on the launch stream (CUDA events), so the warm
    iteration time is that region over iters - 1 and the first iteration is
    the call's time minus it.  After one untimed 1-iteration call (the
    autotuner times its candidate launch shapes on first use)."""
    from paper_1704_04362_gb300 import synth
    sizes = sizes or synth.video_sizes(count, seed=0)
    data, truths = [], []
    for i, (H, W, T) in enumerate(sizes):
        truth = synth.lowrank_torch(H, W, T, 10, seed=5000 + i)
        rms = (torch.linalg.vector_norm(truth, dtype=torch.float64) / truth.numel() ** 0.5).item()
        truth.mul_(1.0 / rms)
        g = torch.Generator(device="cuda")
        g.manual_seed(9000 + i)
        noise = torch.randn((T, W, H), generator=g, device="cuda").permute(2, 1, 0)
        noisy = tp.as_tprod_layout(truth + 0.01 * noise)
        keep = (torch.rand((T, W, H), generator=g, device="cuda") < 0.5).permute(2, 1, 0)
        mask = tp.as_tprod_layout(keep.to(torch.uint8), torch.uint8)
        data.append([noisy, mask, torch.zeros_like(noisy), torch.zeros_like(noisy),
                     torch.zeros_like(noisy), torch.full((1,), 1e-3, dtype=torch.float64,
                                                         device="cuda")])
        truths.append(truth)
        del noise, keep

    def run(n):
        for d in data:
            d[2].zero_()
            d[3].zero_()
            d[4].zero_()
            d[5].fill_(1e-3)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tp.profile_start()
        e0.record()
        tp.tcomplete_svt_batched(data, n, precision={"fp32": tp.TP_FP32, "tf32x3": tp.TP_TF32X3,
                                                     "bf16x3": tp.TP_BF16X3}[precision])
        e1.record()
        torch.cuda.synchronize()
        prof = tp.profile_stop()
        return e0.elapsed_time(e1), prof

    run(1)
    n0 = tp.launch_count()
    total_ms, prof = run(iters)
    launches = tp.launch_count() - n0
    replay_ms = prof.get("svt_graph_replays", (0.0, 0))[0]
    warm_ms = replay_ms / max(1, iters - 1)
    num = sum(float(torch.linalg.vector_norm((d[2] - t).double()) ** 2) for d, t in zip(data, truths))
    den = sum(float(torch.linalg.vector_norm(t.double()) ** 2) for t in truths)
    elems = sum(a * b * c for a, b, c in sizes)
    slices = sum(c // 2 + 1 for _, _, c in sizes)
    first = {k: v[0] for k, v in prof.items() if k != "svt_graph_replays"}
    del data, truths
    return {"workload": f"{count} videos of uneven size (64..480 x 64..360 x 16..120), "
                        f"{elems} elements, {slices} half-spectrum slices per iteration, "
                        "tubal rank 10 + sigma 0.01, 50% observed",
            "precision": precision,
            "iterations": iters, "total_ms": total_ms,
            "first_iteration_ms": total_ms - replay_ms, "warm_iteration_ms": warm_ms,
            "warm_iterations_per_s": 1e3 / warm_ms if warm_ms > 0 else None,
            "relative_error_to_truth": (num / den) ** 0.5, "gpu_launches": launches,
            "first_iteration_kernels_ms": first,
            "note": "iterations after the first replay one captured CUDA graph over all "
                    "tensors (8 side streams), timed as one profiled region"}


def orthonormal_tube_tensor(torch, n1, r, n3, seed):
    """U (n1 x r x n3, float32) with U^T * U = I, distributed as the top-r
    left singular tensor of a dense N(0, 1) tensor: per Fourier slice the Q
    factor of a Gaussian matrix (a uniformly random r-dimensional subspace),
    real at the real slices, conjugate-symmetric elsewhere."""
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    h = n3 // 2 + 1
    Uh = torch.zeros(n3, n1, r, dtype=torch.complex128, device="cuda")
    for f in range(h):
        real = f == 0 or (n3 % 2 == 0 and f == n3 // 2)
        G = torch.randn(n1, r, device="cuda", generator=g, dtype=torch.float64)
        if not real:
            G = torch.complex(G, torch.randn(n1, r, device="cuda", generator=g,
                                             dtype=torch.float64))
        Q, _ = torch.linalg.qr(G)
        Uh[f] = Q.to(torch.complex128)
        if 0 < f < n3 - f:
            Uh[n3 - f] = Q.conj()
    U = torch.fft.ifft(Uh, dim=0).real                       # fft(U) slice f = Q_f
    return U.permute(1, 2, 0).float()                        # logical (n1, r, n3)


def bench_table1(tp, torch, configs=((100, 460), (200, 1000), (300, 1700), (400, 2500),
                                      (500, 3100)), n1=100000, n3=5):
    """The shape of the paper's tensor-multiplication experiment (its Table
    1): U_r^T * U_r for an orthonormal n1 x r x n3 tensor U_r (n1 = 10^5,
    n3 = 5; the left singular tensor of dense N(0, 1) data), exactly (tprod)
    and by the rt-product with l picked slices under the norm probabilities
    of Section 3.1 (the leverage of U_r's rows) and uniform ones.
    RFE = ||I - U~^T U~||_F / ||U_r||_F^2 and RSE = ||I - U~^T U~||_2 /
    ||U_r||_2^2 (the spectral norm of a tensor is the largest over its
    Fourier slices; the slices of U~^T U~ are Hermitian, so it is the largest
    eigenvalue modulus, taken on the host), averaged over 10 seeds."""
    out = []
    for (r, l) in configs:
        t_setup = time.perf_counter()
        U = orthonormal_tube_tensor(torch, n1, r, n3, seed=r)
        Ut = U.permute(1, 0, 2)                                     # slices transposed
        Ut = torch.roll(torch.flip(Ut, dims=[2]), 1, dims=2)        # slices 2..n3 reversed
        Ut = tp.as_tprod_layout(Ut.contiguous())
        Ud = tp.as_tprod_layout(U)
        I = torch.zeros(r, r, n3, device="cuda")
        I[:, :, 0] = torch.eye(r, device="cuda")
        unif = torch.full((n1,), 1.0 / n1, dtype=torch.float64, device="cuda")

        def errs(Z):
            D = (Z - I).permute(2, 0, 1).double()
            Dh = torch.fft.fft(D, dim=0)[: n3 // 2 + 1].cpu().numpy()
            rfe = float(torch.linalg.vector_norm(D)) / r
            rse = max(float(np.abs(np.linalg.eigvalsh(0.5 * (M + M.conj().T))).max()) for M in Dh)
            return rfe, rse
        setup_s = time.perf_counter() - t_setup
        t_exact = time_gpu(lambda: tp.tprod(Ut, Ud, precision=tp.TP_BF16X3), 3, torch)
        exact_err = errs(tp.tprod(Ut, Ud, precision=tp.TP_BF16X3))
        row = {"r": r, "l": l, "tprod_ms": t_exact, "tprod_rfe": exact_err[0], "setup_s": setup_s}
        for name, kw in (("nonuniform", {"prob_mode": tp.TP_PROB_AB}),
                         ("uniform", {"prob_mode": tp.TP_PROB_GIVEN, "p_given": unif})):
            t = time_gpu(lambda: tp.tprod_sampled(Ut, Ud, l, seed=0, precision=tp.TP_BF16X3,
                                                  **kw), 3, torch)
            e = [errs(tp.tprod_sampled(Ut, Ud, l, seed=s, precision=tp.TP_BF16X3, **kw)[0])
                 for s in range(10)]
            row[name] = {"ms": t, "rfe": float(np.mean([x[0] for x in e])),
                         "rse": float(np.mean([x[1] for x in e]))}
        out.append(row)
        del U, Ut, Ud
        torch.cuda.empty_cache()
    return {"workload": f"U_r^T * U_r, U_r {n1} x r x {n3} orthonormal (heavy-tailed row "
                        "leverage), BF16x3, errors averaged over 10 seeds",
            "cases": out}


def bench_learned(torch, train_count=192, eval_n3=(64, 128, 256), eval_n12=(1024, 1024),
                  alphas=(1.5, 2.0, 2.5, 3.0, 3.5, 4.0)):
    """The learned sketch-size predictor against the plain adaptive method
    (rank rule on a 50-column sketch, q = 2) on tensors shaped like the
    1024 x 1024 x n3 rank-predictor workload with per-frequency spectra
    i^(-a_k) (a_k = alpha +- 0.3).  Both methods' per-frequency ranks come
    from a sketch's spectrum and the plain rule; the learned one chooses the
    sketch size from a 17-column sketch, is judged by the rule and falls
    back to 50 columns when a rank reaches its cap.  Times cover the whole
    rank pipeline of each (the learned one includes its cheap pass, the
    network and any fallback); errors are the exact relative truncation
    errors from the known spectra."""
    from paper_1704_04362_gb300 import predictor as P
    from paper_1704_04362_gb300 import synth
    t0 = time.perf_counter()
    x, t = P.training_set(train_count, seed0=100)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    _, w16, losses = P.train(x, t, steps=3000, lr=2e-3, seed=1)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    n1, n2 = eval_n12
    cases = []
    for n3 in eval_n3:
        for i, a in enumerate(alphas if n3 == eval_n3[0] else alphas[::2]):
            X, spec = synth.spectral_torch(n1, n2, n3, a, 0.3, 77000 + i + 100 * n3)
            r_p, _, _ = P.decompose(X, None, seed=i)
            r_l, l, fb = P.decompose(X, w16, seed=i)
            ms_p = P.time_call(lambda: P.decompose(X, None, seed=i), reps=2)
            ms_l = P.time_call(lambda: P.decompose(X, w16, seed=i), reps=2)
            case = {"n3": n3, "alpha": a, "sketch_columns": l, "fell_back": bool(fb),
                    "plain_ms": ms_p, "learned_ms": ms_l, "speedup": ms_p / ms_l,
                    "plain_error": P.truncation_error(spec, r_p, n3),
                    "learned_error": P.truncation_error(spec, r_l, n3),
                    "ranks_equal_fraction": float((r_p == r_l).float().mean().item())}
            if i == 1:
                # the whole multi-rank factorisation U * S * V^T: plain (50
                # columns everywhere) against the predictor's per-frequency
                # sketch sizes l_f = r_f + p_f in one call
                fac = {}
                for name, w in (("plain", None), ("learned", w16)):
                    U, S, V, r, lc = P.factorize(X, w, seed=i)
                    fac[name + "_ms"] = P.time_call(lambda: P.factorize(X, w, seed=i), reps=2)
                    fac[name + "_error"] = _factor_error(tp_mod(), X, U, S, V)
                    if w is not None:
                        sz = P.sketch_sizes(w, X, r, lc, seed=i)
                        fac["learned_sketch_sizes_mean"] = float(sz.float().mean().item())
                    del U, S, V
                fac["optimal_error"] = P.truncation_error(spec, r_l, n3)
                case["factorisation"] = fac
            cases.append(case)
            del X, spec
            torch.cuda.empty_cache()
    return {"workload": f"{n1}x{n2}x{{{','.join(str(v) for v in eval_n3)}}} tensors, "
                        "per-frequency spectra i^-a, a = alpha +- 0.3; trained on "
                        f"{train_count} tensors of 64..160 x 64..128 x 16..256",
            "training_samples": int(x.shape[0]), "data_s": t_data, "train_s": t_train,
            "loss_first_last": [losses[0][1], losses[-1][1]],
            "total_plain_ms": sum(c["plain_ms"] for c in cases),
            "total_learned_ms": sum(c["learned_ms"] for c in cases),
            "cases": cases}


def tp_mod():
    import paper_1704_04362_gb300 as tp
    return tp


def _factor_error(tp, X, U, S, V):
    """||X - U * S * V^T||_F / ||X||_F through the library's t-product (V^T:
    each frontal slice transposed, slices 2..n3 in reverse order)."""
    import torch
    Vt = torch.roll(torch.flip(V.permute(1, 0, 2), dims=[2]), 1, dims=2).contiguous()
    US = tp.tprod(tp.as_tprod_layout(U), tp.as_tprod_layout(S))
    R = tp.tprod(US, tp.as_tprod_layout(Vt))
    err = float(torch.linalg.vector_norm(R - X) / torch.linalg.vector_norm(X))
    del US, R, Vt
    return err


def bench_rsvd(args, tp, torch, with_cpu, forms=("bf16x3", "fp32", "tf32x3")):
    """Randomized low-tubal-rank t-SVD on the mass-spectrometry-shaped
    workload (128 x 128 pixels x 2000 channels, Gamma factors at tubal rank
    15, spikes, 0.5% noise; k = 40, p = 10, q = 2): tensors per second of the
    split tensor-core form (first of `forms`) and of the plain FP32 form.
    With the CPU baseline the float64 oracle decomposes the same tensor once
    (same test matrix) and every form's top-k singular values (all 1001
    frequencies) are compared with it (relative Frobenius error)."""
    from paper_1704_04362_gb300 import synth
    PREC = {"fp32": tp.TP_FP32, "tf32x3": tp.TP_TF32X3, "bf16x3": tp.TP_BF16X3}
    X = synth.msi_like_np()
    Xd = tp.as_tprod_layout(X)
    steps = max(3, min(20, args.steps // 5))
    stream = torch.cuda.current_stream()
    res = {}
    outs = {}
    prof_main = None
    for name in forms:
        pr = PREC[name]
        for _ in range(2):
            outs[name] = tp.tsvd_randomized(Xd, RSVD_K, RSVD_P, RSVD_Q, seed=0, precision=pr)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tp.profile_start()
        e0.record(stream)
        for _ in range(steps):
            tp.tsvd_randomized(Xd, RSVD_K, RSVD_P, RSVD_Q, seed=0, precision=pr)
        e1.record(stream)
        torch.cuda.synchronize()
        prof = tp.profile_stop()
        if prof_main is None:
            prof_main = prof
        res[name] = e0.elapsed_time(e1) / steps
    main = forms[0]
    ms = res[main]
    out = {"metric": "randomized t-SVD tensors/s", "value": 1e3 / ms, "unit": "tensors/s",
           "ms_per_tensor": ms, "steps": steps, "precision": main,
           "dtype": "f32 data; products %s; f32 Householder QR" % main,
           "workload": "128x128x2000 MSI-shaped, tubal rank 15 + spikes + 0.5% noise, "
                       "k=40 p=10 q=2",
           "forms_ms": res,
           "kernels": {k: {"ms_per_launch": v[0] / max(1, v[1]), "launches": v[1]}
                       for k, v in prof_main.items()}}
    cmp = {"fp32_tensors_per_s": 1e3 / res["fp32"]} if "fp32" in res else {}
    if with_cpu:
        from oracle import decomp_ref, philox_ref
        X64 = X.astype(np.float64)
        Om = philox_ref.sketch_signs(128, RSVD_K + RSVD_P, 1001, 2000, 0)
        t0 = time.perf_counter()
        _, Sr, _ = decomp_ref.tsvd_randomized(X64, RSVD_K, RSVD_P, RSVD_Q, Om)
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": 1.0 / dt, "unit": "tensors/s", "cores": os.cpu_count(),
                               "kind": "oracle", "sample": f"one full tensor, {dt:.1f} s"}
        # singular values of every half-spectrum slice (diagonal of S_hat)
        sr = np.stack([np.diag(M).real for M in np.moveaxis(
            np.fft.fft(Sr, axis=2)[:, :, :1001], 2, 0)])
        den = np.linalg.norm(sr)
        for name, (_, S, _) in outs.items():
            Sh = torch.fft.fft(S.permute(2, 0, 1).double(), dim=0)[:1001]
            s = torch.diagonal(Sh, dim1=1, dim2=2).real.cpu().numpy()
            e = float(np.linalg.norm(s - sr) / den)
            out.setdefault("rel_err_singular_values", {})[name] = e
            cmp[("" if name == main else name + "_") + "rel_err"] = sig(e, 3)
    out["compare"] = {k: sig(v) for k, v in cmp.items()}
    return out


def make_inputs(device):
    from paper_1704_04362_gb300 import synth
    A = synth.lowrank_torch(N1, N2, N3, RANK_T, seed=1000, noise=NOISE, device=device)
    B = synth.lowrank_torch(N2, N4, N3, RANK_T, seed=2000, noise=NOISE, device=device)
    return A, B


def gpu_uuid(torch, dev):
    try:
        return "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        return str(dev)


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one
# single-pass ncu capture of the full-size workload; valid only for the kernel
# version it was taken on (profiles/cgemm_tc_2000x4000x1500x64_traffic.md).
MEASURED_TRAFFIC = {"cgemm_tc:bf16x3": 475354624 + 739854080}


def kernel_bytes(name, cprime, precision):
    """Algorithmic DRAM bytes per launch of the HBM-bound kernels of one step
    (inputs read once, outputs written once; the picked-index dimension of the
    transform outputs is padded to 32 with zeros for the tensor-core tiles)."""
    h = N3 // 2 + 1
    kp = (cprime + 31) // 32 * 32
    split = {"fp32": 8.0, "tf32x3": 16.0, "bf16x3": 8.0}[precision]   # bytes per complex output
    if precision == "fp32":
        kp = cprime
    return {
        "norms_lateral": 4.0 * N1 * N2 * N3,
        "norms_horizontal": 4.0 * N2 * N4 * N3,
        "rdft_t": 4.0 * N1 * cprime * N3 + split * N1 * kp * h,
        "rdft": 4.0 * cprime * N4 * N3 + split * kp * N4 * h,
        "irdft": 8.0 * N1 * N4 * h + 4.0 * N1 * N4 * N3,
    }.get(name)


def roofline_for(name, ms_avg, cprime, peaks, sm_mhz, precision="tf32x3"):
    """Algorithmic work per launch of the named kernel and its roofline."""
    h = N3 // 2 + 1
    fl = gemm_flops(N1, cprime, N4, N3)
    if name == "cgemm_fp32":
        # FP32 SIMT: 152 SMs x 128 lanes x 2 flops per FMA x clock
        peak = 152 * 128 * 2 * peaks["sm_max_mhz"] * 1e6 / 1e12
        ach = fl / (ms_avg * 1e-3) / 1e12
        return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": None,
                "peak_src": "derived: 152 SM x 128 FP32 lanes x 2 x sm_max_mhz"}
    if name == "cgemm_tc":
        bf16 = precision == "bf16x3"
        # tf32 dense = bf16 / 2 (nominal ratio); the BF16x3 split runs at the bf16 rate
        peak = peaks["bf16_tflops"] / (1.0 if bf16 else 2.0)
        ach = fl / (ms_avg * 1e-3) / 1e12
        kblk = 32 if bf16 else 16
        kp = (cprime + kblk - 1) // kblk * kblk
        esz = 2.0 if bf16 else 4.0
        alg = 4 * esz * (N1 + N4) * kp * h + 8.0 * N1 * N4 * h
        return {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "pipe_frac": 3 * ach / peak,
                "traffic": MEASURED_TRAFFIC.get("cgemm_tc:" + precision),
                "algorithmic_bytes": alg,
                "peak_src": peaks["src"] + (" bf16 burst" if bf16
                                            else " bf16 burst x 1/2 (tf32 nominal ratio)"),
                "work": "achieved: the nominal 8 n1 c' n4 flops per complex slice; pipe_frac: "
                        "the 3 %s products executed per real product" % ("bf16" if bf16 else "tf32")}
    bytes_per = kernel_bytes(name, cprime, precision)
    if bytes_per is None:
        return None
    ach = bytes_per / (ms_avg * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": ach / peaks["hbm_gbs"], "traffic": None, "peak_src": peaks["src"],
            "algorithmic_bytes": bytes_per}


def sig(x, digits=4):
    """x rounded to `digits` significant digits (None and non-numbers kept)."""
    if isinstance(x, (bool, int)) or not isinstance(x, float):
        return x
    if x == 0 or x != x:
        return x
    return float(f"{x:.{digits}g}")


def step_bytes(cprime):
    """Algorithmic DRAM bytes of one rt-product step with every stage fused:
    A and B read once by the norm passes, the picked slices read once by the
    gathers, Z written once (the Fourier-domain intermediates never leave
    the chip)."""
    return (4.0 * N1 * N2 * N3 + 4.0 * N2 * N4 * N3 + 4.0 * N1 * cprime * N3
            + 4.0 * cprime * N4 * N3 + 4.0 * N1 * N4 * N3)


def write_detail(path, detail):
    """Every measured row, the per-kernel table and the autotuner's choices,
    as one JSON document (the headline line stays short)."""
    if not path:
        return
    try:
        d = os.path.dirname(os.path.abspath(path))
        os.makedirs(d, exist_ok=True)
        with open(path, "w") as f:
            json.dump(detail, f, indent=1, default=str)
    except OSError as e:
        print(f"bench: could not write {path}: {e}", file=sys.stderr)


def row_summaries(rows, rsvd):
    """One short dict per measured row (printed before the headline)."""
    out = {}
    if rsvd:
        out["tsvd_randomized"] = {k: sig(rsvd.get(k)) for k in
                                  ("value", "unit", "ms_per_tensor", "workload")}
        if rsvd.get("cpu_baseline"):
            out["tsvd_randomized"]["oracle_tensors_per_s"] = sig(rsvd["cpu_baseline"]["value"])
        if rsvd.get("compare"):
            out["tsvd_randomized"]["compare"] = rsvd["compare"]
    for name, r in (rows or {}).items():
        if not isinstance(r, dict):
            continue
        keep = {k: sig(v) for k, v in r.items()
                if isinstance(v, (int, float, str, bool)) and k != "note"}
        if "cases" in r:
            keep["cases"] = len(r["cases"])
        out[name] = keep
    return out


def bind_to_gpu_local_cpus(dev):
    """Restricts this process to the allowed CPUs local to GPU `dev` (the
    sysfs local_cpulist of its PCI function, bus id from nvidia-smi); returns
    a short note of what was done."""
    try:
        bus = subprocess.run(["nvidia-smi", "-i", str(dev), "--query-gpu=pci.bus_id",
                              "--format=csv,noheader"], capture_output=True, text=True,
                             timeout=30).stdout.strip()
        dom, rest = bus.split(":", 1)
        path = f"/sys/bus/pci/devices/{dom[-4:].lower()}:{rest.lower()}/local_cpulist"
        cpus = set()
        with open(path) as fh:
            for part in fh.read().strip().split(","):
                a, _, b = part.partition("-")
                if a:
                    cpus.update(range(int(a), int(b or a) + 1))
        allowed = os.sched_getaffinity(0)
        use = cpus & allowed
        if use and use != allowed:
            os.sched_setaffinity(0, use)
            return f"bound to {len(use)} of {len(allowed)} allowed cpus (GPU-local)"
        return "unchanged: " + ("every allowed cpu is GPU-local" if use else
                                "no GPU-local cpu is allowed")
    except Exception as exc:   # no nvidia-smi, no sysfs entry, no affinity call
        return f"unchanged ({type(exc).__name__})"


def headline(args, world, value, ms, cprime, launches, roof, kernels, cpu, e2e, clocks,
             compare, errors, rsvd, rows, peaks):
    """The one JSON line the benchmark contract asks for, kept under 2 KB."""
    sb = step_bytes(cprime)
    roof_c = None
    if roof:
        roof_c = {k: sig(roof.get(k)) for k in ("bound", "achieved", "peak", "unit", "frac",
                                                  "traffic", "kernel")}
        if "pipe_frac" in roof:
            # frac: nominal 8mnk complex flops; pipe_frac: the three split
            # products the tensor cores execute per real product
            roof_c["pipe_frac"] = sig(roof["pipe_frac"])
        roof_c["peak_src"] = "measured bf16 burst" if roof.get("unit") == "TFLOP/s" and \
            str(roof.get("peak_src", "")).startswith("measured") else roof.get("peak_src")
    forms = {args.precision: {"tflops": sig(value), "ms": sig(ms)}}
    for cm in compare:
        forms[cm["precision"]] = {"tflops": sig(cm["value"]), "ms": sig(cm["ms_per_step"])}
    for name, e in (errors or {}).items():
        forms.setdefault(name, {})["rel_err"] = sig(e["rel_err"], 3)
    if errors:
        # relative Frobenius error of each form against the float64 oracle
        # on the CPU-baseline sample, and whether all forms drew its picks
        forms["picks_equal"] = all(e["picks_equal"] for e in errors.values())
    sec = {}
    if rsvd:
        r = {"tensors_per_s": sig(rsvd["value"]), "ms": sig(rsvd["ms_per_tensor"])}
        r.update(rsvd.get("compare") or {})
        if rsvd.get("cpu_baseline"):
            r["oracle_tensors_per_s"] = sig(rsvd["cpu_baseline"]["value"], 3)
        sec["tsvd_randomized"] = r
    # batched completion: [warm iteration ms, iterations, relative error to the truth]
    for key, name in (("completion_batched", "completion_fp32"),
                      ("completion_batched_bf16x3", "completion_bf16x3")):
        cb = (rows or {}).get(key)
        if cb:
            sec[name] = [sig(cb.get("warm_iteration_ms")), cb.get("iterations"),
                         sig(cb.get("relative_error_to_truth"), 3)]
    line = {
        "metric": "t-product TFLOP/s & randomized t-SVD tensors/s vs plain FP32 at equal rel. error",
        "value": sig(value), "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sig(ms), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "tf32x3": "tf32x3 (f32 accumulate)",
                  "bf16x3": "bf16x3 (f32 accumulate)"}[args.precision],
        "data": "synthetic",
        "config": {"workload": "rt-product (Alg. 2) A 2000x4000x64 * B 4000x1500x64, tubal "
                               "rank 20 + 1% noise, c=400, norm-product probabilities",
                   "c_prime": cprime, "precision": args.precision,
                   "l2": "inputs 3.58 GB > L2, streamed",
                   "parallelism": f"replicas x{world}"},
        "roofline": roof_c,
        # the whole step against its fused minimum (A, B read once, picks
        # gathered once, Z written once)
        "step_hbm": {"bytes": sig(sb), "frac": sig(sb / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"], 3)},
        "kernels_ms": {k.split("<")[0][:24]: [sig(v["ms_per_launch"], 3), sig(v["share"], 3)]
                       for k, v in sorted(kernels.items(), key=lambda kv: -kv[1]["share"])[:6]},
        "forms": forms,
        "e2e": None if e2e is None else {k: sig(e2e[k]) for k in
                                         ("value", "unit", "ms_per_step", "h2d_bytes_per_step",
                                          "d2h_bytes_per_step")},
        "gpu_launches": launches,
        "cpu_baseline": None if cpu is None else {
            "value": sig(cpu.get("value")), "unit": cpu.get("unit"), "cores": cpu.get("cores"),
            "kind": cpu.get("kind"), "sample": str(cpu.get("sample"))[:100]},
        "clocks": {k: sig(clocks.get(k)) for k in ("sm_mhz", "sm_max_mhz", "reasons")},
        "secondary": sec or None,
        "detail_file": args.detail_file,
    }
    # keep the line short: drop the least important parts first
    for drop in ("detail_file", "kernels_ms", "secondary"):
        if len(json.dumps(line)) < 2000:
            break
        line.pop(drop, None)
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16x3", choices=["fp32", "tf32x3", "bf16x3"])
    ap.add_argument("--compare", default="tf32x3,fp32",
                    help="comma-separated precisions also timed (the 3xTF32 split and the plain "
                         "FP32 form), or 'none'")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=6)
    ap.add_argument("--small", action="store_true", help="profiling case, not a bench number")
    ap.add_argument("--detail-file", default="bench_detail.json",
                    help="where every row, the per-kernel table and the autotuner's choices "
                         "are written (the stdout headline stays under 2 KB)")
    ap.add_argument("--no-rsvd", action="store_true", help="skip the randomized t-SVD line")
    ap.add_argument("--no-rows", action="store_true", help="skip the t-SVD / t-CX / ADMM rows")
    ap.add_argument("--svt-iters", type=int, default=100,
                    help="iterations of the batched completion row (256 videos)")
    ap.add_argument("--only", default=None,
                    help="comma-separated rows to run instead of the headline step "
                         "(rsvd, svt_batched, svt_batched_bf16x3, svt_video, learned, tcx): "
                         "profiling and "
                         "tuning runs, no headline line")
    ap.add_argument("--tune-file", default=None,
                    help="autotuner table: loaded before the run when the file exists, "
                         "written after it (so that a profiled run reuses the plain run's "
                         "launch shapes instead of timing them under the profiler)")
    args = ap.parse_args()
    if args.small:
        use_small_case()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    import torch
    if args.impl == "reference":
        return reference_arm(args, rank, world)

    import paper_1704_04362_gb300 as tp
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    PREC = {"fp32": tp.TP_FP32, "tf32x3": tp.TP_TF32X3, "bf16x3": tp.TP_BF16X3}
    prec = PREC[args.precision]
    peaks = load_peaks()
    if args.tune_file and os.path.exists(args.tune_file):
        tp.autotune_load(args.tune_file)

    if args.only:
        # single rows for profiling and tuning: printed one per line, no headline
        for name in args.only.split(","):
            if name == "rsvd":
                out = bench_rsvd(args, tp, torch, with_cpu=False)
            elif name == "svt_batched":
                out = bench_svt_batched(tp, torch, iters=args.svt_iters)
            elif name == "svt_batched_bf16x3":
                out = bench_svt_batched(tp, torch, iters=args.svt_iters, precision="bf16x3")
            elif name == "learned":
                out = bench_learned(torch)
            elif name == "tcx":
                # the t-CX row alone (its two Jacobi launches dominate)
                from paper_1704_04362_gb300 import synth
                Ad = tp.as_tprod_layout(synth.lowrank_np(256, 512, 32, 10, seed=3, noise=0.01))
                out = {"workload": "256x512x32 tubal rank 10 + 1% noise, c = 64",
                       "gpu_ms": time_gpu(lambda: tp.tcx(Ad, 64, seed=0), args.steps, torch)}
            elif name == "svt_video":
                # one 480 x 360 x 120 video (the largest of the batch): a
                # single-tensor profiling case a few GB in size
                out = bench_svt_batched(tp, torch, count=1, iters=args.svt_iters,
                                        sizes=[(480, 360, 120)])
            else:
                raise SystemExit(f"bench: unknown row {name!r}")
            print(json.dumps({"row": name, **out}, default=str))
        return

    A, B = make_inputs("cuda")
    Z = tp.empty_tensor(N1, N4, N3)
    idx = torch.empty(N2, dtype=torch.int32, device="cuda")
    cnt = torch.empty(1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(pr, Zout):
        """W warm-up steps, then K steps between CUDA events with per-kernel
        event timing; returns (ms per step, profile, launches)."""
        def step():
            tp.tprod_sampled(A, B, C_SAMPLES, seed=SEED, precision=pr, Z=Zout, idx=idx, count=cnt)
        for _ in range(max(3, args.warmup)):
            step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        n0 = tp.launch_count()
        tp.profile_start()
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
        pf = tp.profile_stop()
        nl = tp.launch_count() - n0
        if dist:
            dist.barrier()
        t_ms = reduce_max(ev0.elapsed_time(ev1) / args.steps, dist, "cuda")
        return t_ms, pf, nl

    compare = []
    for cp in [c for c in args.compare.split(",") if c and c != "none" and c != args.precision]:
        Zc = tp.empty_tensor(N1, N4, N3)
        c_ms, c_prof, _ = timed(PREC[cp], Zc)
        compare.append({"precision": cp, "ms_per_step": c_ms, "Z": Zc,
                        "kernels": {k: v[0] / max(1, v[1]) for k, v in c_prof.items()}})

    sampler = ClockSampler(gpu_uuid(torch, local_rank))
    sampler.start()
    ms, prof, launches = timed(prec, Z)
    clocks = sampler.stop()
    cprime = int(cnt.item())
    flops = gemm_flops(N1, cprime, N4, N3)
    value = world * flops / (ms * 1e-3) / 1e12
    for cm in compare:
        cm["value"] = world * flops / (cm["ms_per_step"] * 1e-3) / 1e12
        # agreement with the headline form (each form is checked against the
        # float64 oracle in tests/test_gpu_fullsize.py)
        Zc = cm.pop("Z")
        cm["rel_fro_diff"] = float(torch.linalg.vector_norm((Z - Zc).double()) /
                                   torch.linalg.vector_norm(Z.double()))
        del Zc

    # per-kernel breakdown and roofline of the dominant kernel
    kernels = {k: {"ms_per_launch": v[0] / max(1, v[1]), "launches": v[1],
                   "share": v[0] / max(1e-9, sum(x[0] for x in prof.values()))}
               for k, v in prof.items()}
    dom = max(prof, key=lambda k: prof[k][0]) if prof else None
    roof = roofline_for(dom, prof[dom][0] / prof[dom][1], cprime, peaks, clocks.get("sm_mhz"),
                        args.precision) if dom else None
    for k, kv in kernels.items():
        kb = kernel_bytes(k, cprime, args.precision)
        if kb is not None:
            kv["hbm_frac"] = kb / (kv["ms_per_launch"] * 1e-3) / 1e9 / peaks["hbm_gbs"]
    if roof is not None:
        roof["kernel"] = dom

    # end to end through the C entry point with host buffers: every step
    # copies its A and B from pinned host memory and its Z back.  Steps are
    # pipelined over two device buffer sets: step k+1's upload (copy stream)
    # overlaps step k's compute (launch stream) and download (second copy
    # stream); the host link (about 210 GB/s each way on these boxes) bounds it.
    e2e = None
    if args.e2e_steps > 0:
        # pinned buffers allocated while the process runs on the GPU-local
        # CPUs (so that they land on the GPU's NUMA node); the affinity is
        # restored afterwards (the copies are DMA, and the CPU baseline keeps
        # every allowed core)
        allowed = os.sched_getaffinity(0) if hasattr(os, "sched_getaffinity") else None
        numa_note = bind_to_gpu_local_cpus(local_rank)
        Ah = torch.empty((N3, N2, N1), dtype=torch.float32, pin_memory=True)
        Bh = torch.empty((N3, N4, N2), dtype=torch.float32, pin_memory=True)
        Zh = [torch.empty((N3, N4, N1), dtype=torch.float32, pin_memory=True) for _ in range(2)]
        if allowed is not None:
            os.sched_setaffinity(0, allowed)
        Ah.copy_(A.permute(2, 1, 0))
        Bh.copy_(B.permute(2, 1, 0))
        Ad = [tp.empty_tensor(N1, N2, N3) for _ in range(2)]
        Bd = [tp.empty_tensor(N2, N4, N3) for _ in range(2)]
        Zd = [tp.empty_tensor(N1, N4, N3) for _ in range(2)]
        up, down = torch.cuda.Stream(), torch.cuda.Stream()
        uploaded = [torch.cuda.Event() for _ in range(2)]
        computed = [torch.cuda.Event() for _ in range(2)]
        downloaded = [torch.cuda.Event() for _ in range(2)]
        for b in range(2):
            computed[b].record(stream)
            downloaded[b].record(stream)
        torch.cuda.synchronize()

        def e2e_steps(n):
            for k in range(n):
                b = k % 2
                with torch.cuda.stream(up):
                    up.wait_event(computed[b])           # set b's inputs free again
                    Ad[b].permute(2, 1, 0).copy_(Ah, non_blocking=True)
                    Bd[b].permute(2, 1, 0).copy_(Bh, non_blocking=True)
                    uploaded[b].record(up)
                stream.wait_event(uploaded[b])
                stream.wait_event(downloaded[b])         # set b's Z read back
                tp.tprod_sampled(Ad[b], Bd[b], C_SAMPLES, seed=SEED, precision=prec, Z=Zd[b],
                                 idx=idx, count=cnt)
                computed[b].record(stream)
                with torch.cuda.stream(down):
                    down.wait_event(computed[b])
                    Zh[b].copy_(Zd[b].permute(2, 1, 0), non_blocking=True)
                    downloaded[b].record(down)
            stream.wait_event(downloaded[(n - 1) % 2])
            stream.wait_event(downloaded[n % 2])

        e2e_steps(2)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        ev0.record(stream)
        e2e_steps(args.e2e_steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        ems = reduce_max(ev0.elapsed_time(ev1) / args.e2e_steps, dist, "cuda")
        # the link itself: one plain upload of A's pinned buffer
        ev0.record(stream)
        Ad[0].permute(2, 1, 0).copy_(Ah, non_blocking=True)
        ev1.record(stream)
        torch.cuda.synchronize()
        h2d_gbs = Ah.numel() * 4 / (ev0.elapsed_time(ev1) * 1e-3) / 1e9
        e2e = {"value": world * flops / (ems * 1e-3) / 1e12, "unit": "TFLOP/s",
               "ms_per_step": ems,
               "h2d_bytes_per_step": int(Ah.numel() * 4 + Bh.numel() * 4),
               "d2h_bytes_per_step": int(Zh[0].numel() * 4),
               "h2d_gbs_plain_copy": h2d_gbs, "pinned_buffers": numa_note,
               "pipeline": "two buffer sets; upload of step k+1 overlaps compute and "
                           "download of step k"}
        del Ah, Bh, Zh, Ad, Bd, Zd

    cpu = None
    errors = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            dt, fl, Zref, idx_ref = run_oracle_sample(A, B, SEED, keep_output=True)
            cpu = {"value": fl / dt / 1e12, "unit": "TFLOP/s", "cores": os.cpu_count(),
                   "kind": "oracle",
                   "sample": (f"oracle rt-product of A[:{CPU_SAMPLE}], B[:, :{CPU_SAMPLE}] "
                              f"(n2=4000, n3=64, c=400), {dt:.1f} s")}
            forms = {args.precision: prec}
            for cm in compare:
                forms[cm["precision"]] = PREC[cm["precision"]]
            errors = sample_errors(tp, torch, A, B, Zref, idx_ref, forms)
            del Zref
        except Exception as e:  # reported, never fatal
            cpu = {"value": None, "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"failed: {e!r}"}

    rsvd = None
    if not args.no_rsvd and not args.small:
        del A, B
        torch.cuda.empty_cache()
        rsvd = bench_rsvd(args, tp, torch, with_cpu=(rank == 0 and world == 1
                                                      and not args.no_cpu_baseline))
        rsvd["value"] *= world
    rows = None
    if not args.no_rows and not args.small:
        rows = bench_rows(tp, torch, with_cpu=(rank == 0 and world == 1 and not args.no_cpu_baseline))
        rows["completion_batched"] = bench_svt_batched(tp, torch, iters=args.svt_iters)
        # the BF16x3 form (the SVT's three GEMMs on the tensor cores), fewer iterations
        rows["completion_batched_bf16x3"] = bench_svt_batched(
            tp, torch, iters=max(2, args.svt_iters // 4), precision="bf16x3")
        rows["learned_rank"] = bench_learned(torch)
        rows["table1_shape"] = bench_table1(tp, torch)

    if rank == 0:
        detail = {
            "e2e": e2e, "roofline": roof, "kernels": kernels, "cpu_baseline": cpu,
            "clocks": clocks, "compare": compare, "sample_errors": errors,
            "secondary": rsvd, "rows": rows,
            "autotune": [{"key": k, "choice": c, "candidates": n, "ms": b, "default_ms": d}
                         for (k, c, n, b, d) in tp.autotune_table()],
        }
        write_detail(args.detail_file, detail)
        # summaries of the other rows, one short line each, before the headline
        for name, summ in row_summaries(rows, rsvd).items():
            print(json.dumps({"row": name, **summ}))
        line = headline(args, world, value, ms, cprime, launches, roof, kernels, cpu, e2e,
                        clocks, compare, errors, rsvd, rows, peaks)
        sys.stdout.flush()
        print(json.dumps(line), flush=True)
        if args.tune_file:
            tp.autotune_save(args.tune_file)
    if dist:
        dist.destroy_process_group()


def reference_arm(args, rank, world):
    """--impl reference: the float64 oracle on the host cores, per step one
    bounded sample of the same workload.  Rank 0 only."""
    if rank != 0:
        return
    import torch
    torch.cuda.set_device(0)
    A, B = make_inputs("cuda")
    times, fls = [], []
    for i in range(args.warmup + args.steps):
        dt, fl = run_oracle_sample(A, B, SEED)
        if i >= args.warmup:
            times.append(dt)
            fls.append(fl)
    sec = sum(times) / len(times)
    val = (sum(fls) / len(fls)) / sec / 1e12
    line = {
        "impl": "reference", "metric": "t-product TFLOP/s (sampled rt-product, Algorithm 2)",
        "value": val, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "rt-product A 2000x4000x64 * B 4000x1500x64, tubal rank 20 "
                               "+1% noise, c=400, p ~ ||A(:,j,:)|| ||B(j,:,:)||",
                   "parallelism": "host cores"},
        "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": f"float64 oracle on A[:{CPU_SAMPLE}], B[:, :{CPU_SAMPLE}] per step"},
        "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()
