#!/usr/bin/env python
"""Throughput of the compressed CQM-BEM single-layer solve on GB300.

Metric: triangle * frequency / s (M * L per step, L = N + 1 CQM frequencies)
of one full pass of the hot path -- geometry, cluster tree, partition,
Chebyshev bases, MACA of every block, plane-wave data, forward R-scaled DFT,
batched GMRES over the solved frequencies, inverse DFT -- on the 5120-triangle
unit sphere, BDF2, N = 256, dt = 0.1, eta = 1, m = 4, leaf 32, MACA tolerance
1e-9.  Arithmetic: bf16x3 tensor-core far coupling and fp32 near field in the
inner GMRES iterations, float-float residual applies, fp64 MACA, transforms and
Krylov basis; the result meets the FP64 residual target.  Synthetic input:
seeded icosphere and Gaussian plane-wave pulse.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs one independent replica per GPU (the method does not shard across
GPUs here); value = all ranks' units / max over ranks of the timed region.
--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (3 of its solved frequencies) on all host cores (rank 0 only).
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

# MACA tolerance 1e-9: the metric is quoted at a relative error of 1e-6 in
# the time domain.  The inverse transform scales per-frequency errors by up to
# R^-N ~ 1e5 at the last steps; measured against the full FP64 oracle on this
# workload (LU of its H^2-expanded V_l at all 129 solved frequencies), MACA
# tolerances of 1e-7, 1e-8, 1e-9 give time-domain errors of 1.3e-5, 1.6e-6,
# 3.4e-7.
WORKLOAD = dict(name="sphere5120_N256", level=4, N=256, dt=0.1, bdf=2, eta=1.0, cheb_m=4,
                n_min=32, aca_eps=1e-9)
# Other workloads (--workload): the mixed-precision torus (major radius 1, minor
# 0.3, 20480 triangles, n_u = 160, n_v = 64), BDF2, N = 1024, dt = 0.4 times the
# mean edge length (Courant number 0.4); its per-step error is measured against
# the same path with the MACA at 1e-9 (--step-error; 32 rank slots per block
# are what the device holds at this size, and a tighter MACA needs more).
WORKLOADS = {
    "sphere5120_N256": WORKLOAD,
    "torus20480_N1024": dict(name="torus20480_N1024", torus=20480, N=1024, courant=0.4, bdf=2,
                             eta=1.0, cheb_m=4, n_min=32, aca_eps=1e-8, ref_eps=1e-9, ref_cap=32),
}


def workload_mesh(W):
    """Mesh and time step of a workload."""
    from paper_2006_05186_gb300 import synth
    if "torus" in W:
        m = synth.torus_for(W["torus"])
        return m, W["courant"] * synth.mean_edge_length(m)
    return synth.icosphere(W["level"]), W["dt"]
METRIC = "CQM-BEM solve throughput (triangle·freq/s), p50/p99 latency at rel err ≤1e-6"
UNIT = "triangle*freq/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ALU peaks of a GB300 from unit counts and the maximum SM clock: FP32
# 152 SMs x 128 lanes x 2 flops x 2.07 GHz = 80.5 TFLOP/s (an FMA probe measured
# 69); FP64 at the recipe's nominal 1.25 TFLOP/s (the probe measured 1.19).
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
FP64_PEAK_TFLOPS = 1.25
FP32_PEAK_SOURCE = "unit counts x max SM clock (152 SMs x 128 FP32 lanes x 2 x 2.07 GHz)"
# TF32 dense tensor peak: the measured bf16 cuBLAS rate (sustained: the kernel is
# timed inside a seconds-long step) times the nominal tf32 / bf16 ratio 1.1 / 2.25.
TF32_OVER_BF16 = 1.1 / 2.25
# FP32 issue peak (thread instructions): 152 SMs x 128 lanes x 2.07 GHz.
FP32_ISSUE_PEAK_T = 152 * 128 * 2.07e9 / 1e12
# FP32-pipe instructions per float-float kernel evaluation c exp(-s d) of the
# MACA slices and fibres (the table exponential and cis of csrc/ffexp.cuh, the
# two final float-float products and the float-float accumulation), counted
# from the source.
MACA_FF_INSTR_PER_EVAL = 160


# DRAM bytes (read + write) of one launch of the bf16 tensor-core coupling from
# an ncu capture of that kernel on the 1280-triangle sphere at N = 256, with
# the capture's far rank terms and how many of them took the single product
# (None: no capture of the current kernel).  The traffic is the bf16 images
# (hi and lo planes, 32 KB, of a three-product term; the 16 KB hi plane of a
# single-product one) read once, plus d_t, xhat and the partial tiles, which
# grow with the rank terms: the bench counts the workload's image bytes and
# scales the rest per rank term.
TC2_CAPTURE = dict(dram=380.197376e6 + 22.704896e6, terms=13284, single=4914)
TC2_DRAM_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of k_far_coupling_tc2 (1280-triangle "
                   "sphere, N = 256): this workload's image bytes plus the capture's other bytes per rank term")


def tc2_image_bytes(terms, single):
    return 32768.0 * (terms - single) + 16384.0 * single


def tc2_traffic(info):
    """DRAM bytes of one launch of the tensor-core coupling on this workload,
    from the capture (None without one)."""
    c = TC2_CAPTURE
    if not c:
        return None
    rest = (c["dram"] - tc2_image_bytes(c["terms"], c["single"])) / c["terms"]
    terms = info["rank_sum_far"]
    return tc2_image_bytes(terms, info.get("tc_single_terms", 0)) + rest * terms


def tf32_peak():
    pk, src = _peaks()
    bf16 = pk.get("bf16_tflops_sustained", pk["bf16_tflops"])
    return bf16 * TF32_OVER_BF16, (f"{src} bf16 cuBLAS {bf16:.1f} TFLOP/s (sustained) x nominal "
                                   f"tf32/bf16 ratio 1.1/2.25")


def measure_tf32_peak():
    """Dense TF32 tensor rate of this GPU: cuBLAS fp32 GEMM with TF32 math,
    8192^3 (2 n^3 flops), best of 10 after warm-up, CUDA events."""
    import torch
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        n = 8192
        a = torch.randn(n, n, device="cuda")
        b = torch.randn(n, n, device="cuda")
        for _ in range(3):
            torch.matmul(a, b)
        best = float("inf")
        for _ in range(10):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        del a, b
        torch.cuda.empty_cache()
        return 2.0 * n ** 3 / best / 1e12
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


def dist_init(ngpus):
    import torch
    import torch.distributed as dist
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    """Max of a host float over the ranks (NCCL on GPUs, gloo on CPU)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(units_per_step, steps, my_seconds, world):
    """Whole-job throughput: units of all ranks / max over ranks of the timed region."""
    tmax = max_over_ranks(my_seconds, world)
    return world * units_per_step * steps / tmax, tmax


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


def kernel_models(info, Ls, p, tensor_cores, tf32=None, sinfo=None, launches_per_step=None):
    """Algorithmic work per launch of the contraction kernels and the peak
    that bounds each.  Complex multiply-add = 8 flops.  Factored forms:
    coupling sum_far rank * p^2 * Ls, near field sum_near rank * #r#c * Ls
    complex multiply-adds.  The tensor-core coupling is counted by its useful
    flops against the TF32 tensor peak (its three-product split executes three
    times as many).  The float-float kernels issue 48 FP32 instructions per
    complex multiply-add (four exact products with TwoSum accumulation); their
    work is counted in FP32 issue slots, 2 flops each, against the FP32 peak.
    Expanded forms stream their tables once per launch: the FP32 near field
    8 bytes, the float-float near field and far couplings 16 bytes per entry
    and frequency, against the measured HBM bandwidth."""
    cmac_far = info["rank_sum_far"] * p * p * Ls
    cmac_near = info["near_rank_entries"] * Ls
    fp32 = dict(bound="alu", peak=FP32_PEAK_TFLOPS, peak_source=FP32_PEAK_SOURCE, unit="TFLOP/s")
    models = {
        "far_coupling": dict(fp32, work=8.0 * cmac_far, what="FP32 complex MAC, inner operator"),
        "near_apply": dict(fp32, work=8.0 * cmac_near, what="FP32 complex MAC, inner operator"),
        "far_exact": dict(fp32, work=2.0 * 48 * cmac_far, what="float-float complex MAC (FP32 issue)"),
        "near_exact": dict(fp32, work=2.0 * 48 * cmac_near, what="float-float complex MAC (FP32 issue)"),
    }
    if tensor_cores == 2 and p == 64:
        peak, src = tf32_peak() if tf32 is None else (
            tf32, "measured here: cuBLAS TF32 GEMM 8192^3 (torch.matmul, allow_tf32), best of 10")
        models["far_coupling"] = dict(
            bound="tensor", peak=peak, peak_source=src, unit="TFLOP/s", work=8.0 * cmac_far,
            what="complex MAC on tcgen05 TF32 (useful flops; the 3-product split executes 3x)",
            traffic=None)
    elif tensor_cores == 1 and p == 64:
        pk, src = _peaks()
        bf16 = pk.get("bf16_tflops_sustained", pk["bf16_tflops"])
        models["far_coupling"] = dict(
            bound="tensor", peak=bf16, unit="TFLOP/s", work=8.0 * cmac_far,
            peak_source=f"{src} cuBLAS bf16 GEMM, sustained (MEASURED_PEAKS.json bf16_tflops_sustained)",
            what=("complex MAC on tcgen05 bf16 at all Ls frequencies of every apply (useful flops; the "
                  "hi/lo three-product split executes 3x for the leading rank terms and 1x for the "
                  f"{info.get('tc_single_terms', 0)} trailing ones, frequencies are padded to 128-row chunks, "
                  "and converged frequencies are computed with the rest)"),
            traffic=tc2_traffic(info),
            traffic_source=TC2_DRAM_SOURCE)
    pk, src = _peaks()
    hbm = dict(bound="hbm", peak=pk["hbm_gbs"], unit="GB/s",
               peak_source=f"{src} STREAM-style copy, MEASURED_PEAKS.json hbm_gbs")
    # The streaming kernels skip converged frequencies: the inner applies (one
    # per Arnoldi step) read the active ones, the FP64-accurate applies (one
    # per restart after the first) those not converged at an earlier restart.
    f_inner, f_exact, note_i, note_e = Ls, Ls, "", ""
    if sinfo and sinfo.get("iterations") and sinfo.get("arnoldi_freq_steps"):
        f_inner = sinfo["arnoldi_freq_steps"] / sinfo["iterations"]
        note_i = f", {f_inner:.1f} active frequencies per apply on average"
    if sinfo and sinfo.get("restarts") and sinfo.get("restart_freq_applies"):
        f_exact = sinfo["restart_freq_applies"] / sinfo["restarts"]
        note_e = f", {f_exact:.1f} unconverged frequencies per apply on average"
    if info.get("near_expanded"):
        models["near_apply"] = dict(hbm, work=8.0 * info["near_entries"] * f_inner,
                                    what="expanded FP32 near field streamed (8 B per entry and frequency" + note_i + ")")
        models["near_exact"] = dict(hbm, work=16.0 * info["near_entries"] * f_exact,
                                    what="expanded float-float near field streamed (16 B per entry and frequency"
                                    + note_e + ")")
    if info.get("far_expanded"):
        models["far_exact"] = dict(hbm, work=16.0 * info["far_coupling"] * f_exact,
                                   what="expanded float-float far couplings streamed (16 B per entry and frequency"
                                   + note_e + ")")
    lps = launches_per_step or {}
    issue = dict(bound="alu", peak=FP32_ISSUE_PEAK_T, unit="Tinst/s",
                 peak_source="FP32 issue: unit counts x max SM clock (152 SMs x 128 lanes x 2.07 GHz)")
    for k, key in (("maca_slice", "maca_slice_evals"), ("maca_fibre", "maca_fibre_evals")):
        if info.get(key) and lps.get(k):
            models[k] = dict(issue, work=float(info[key]) * MACA_FF_INSTR_PER_EVAL / lps[k],
                             what=(f"float-float kernel evaluations ({info[key]:.3e} per setup) x "
                                   f"{MACA_FF_INSTR_PER_EVAL} FP32 instructions each"))
    if sinfo and sinfo.get("iterations") and sinfo.get("arnoldi_vectors"):
        byts = (4.0 * sinfo["arnoldi_vectors"] + 8.0 * sinfo["arnoldi_freq_steps"]) * info["nt"] * 16.0
        models["arnoldi"] = dict(hbm, work=byts / sinfo["iterations"],
                                 what=("CGS2 Arnoldi step: the basis read four times and w eight times "
                                       "per active frequency (16 B complex entries)"))
    return models


def cqm_R(N):
    """CQM radius (1e-10)^(1/(2L)), L = N + 1."""
    return 1e-10 ** (1.0 / (2 * (N + 1)))


# FP32 instructions of one float-float multiply-add of the march's history
# sums (a complex value times a real one, or the real part of a complex
# product): two products (two_prod + two cross FMAs + fast_two_sum, 6 each)
# and two TwoSum accumulations (8 each), counted from the source.
MOT_FF_INSTR_PER_MAC = 28


def mot_models(info, N, launches_per_step):
    """Work of the marching-on-in-time kernels.  History of step n (eq.
    fastrhs), in float-float on the FP32 pipes: the convolution
    sum_{k<n} dhat_t[n-k] q_k of every rank term (64 entries for a far term,
    the column cluster for a near one, taken as the mean leaf size) and the
    real part of C_t z_t (one multiply-add per entry of C_t), summed over
    the steps and divided by the launches, each multiply-add
    MOT_FF_INSTR_PER_MAC FP32 instructions.  Step: the dense inverse of
    Vhat_0 applied (8 B per entry, streamed)."""
    M = info["nt"]
    leaf = M / max(1, info["n_leaves"])
    lags = N * (N + 1) / 2.0
    per_lag = info["rank_sum_far"] * 64 + info["rank_sum_near"] * leaf
    per_step = info["rank_sum_far"] * 4096 + info["near_rank_entries"]
    lps = launches_per_step or {}
    models = {}
    if lps.get("mot_history"):
        models["mot_history"] = dict(
            bound="alu", peak=FP32_ISSUE_PEAK_T, unit="Tinst/s",
            peak_source="FP32 issue: unit counts x max SM clock (152 SMs x 128 lanes x 2.07 GHz)",
            work=MOT_FF_INSTR_PER_MAC * (per_lag * lags + per_step * N) / lps["mot_history"],
            what="float-float history sums of the march (eq. fastrhs), FP32 instructions")
    if lps.get("mot_step"):
        models["mot_step"] = dict(bound="hbm", peak=_peaks()[0]["hbm_gbs"], unit="GB/s",
                                  work=8.0 * M * M * (N + 1) / lps["mot_step"],
                                  peak_source="measured STREAM-style copy, MEASURED_PEAKS.json hbm_gbs",
                                  what="inverse of Vhat_0 streamed once per step (8 B per entry)")
    return models


def roofline_of(prof, models):
    """Roofline of the dominant modelled kernel (live CUDA-event timings)."""
    timed = [(k, v) for k, v in prof.items() if k in models and v[0]]
    if not timed:
        return None
    name, (n, ms) = max(timed, key=lambda kv: kv[1][1])
    return roofline_entry(name, n, ms, models[name])


def time_weighted_frac(prof, models):
    """Fraction of peak of the modelled contraction kernels, each weighted by
    its share of their summed device time (live CUDA-event timings)."""
    parts = [(prof[k][1], roofline_entry(k, prof[k][0], prof[k][1], models[k])["frac"])
             for k in models if k in prof and prof[k][0]]
    total = sum(ms for ms, _ in parts)
    if total <= 0:
        return None
    return {"frac": sum(ms * f for ms, f in parts) / total, "kernels": [k for k in models if k in prof and prof[k][0]],
            "ms": total}


def roofline_entry(name, n, ms, mdl):
    scale = 1e9 if mdl["unit"] == "GB/s" else 1e12
    achieved = mdl["work"] / (ms / n / 1e3) / scale
    out = {"bound": mdl["bound"], "kernel": name, "what": mdl["what"], "achieved": achieved,
           "peak": mdl["peak"], "unit": mdl["unit"], "frac": achieved / mdl["peak"],
           "traffic": mdl.get("traffic"), "launches": n, "ms_per_launch": ms / n,
           "peak_source": mdl["peak_source"]}
    if mdl.get("traffic_source"):
        out["traffic_source"] = mdl["traffic_source"]
    return out


def run_ours(args):
    import torch
    from paper_2006_05186_gb300 import CqmBem, synth
    rank, world = dist_init(args.gpus)
    W = WORKLOAD
    m, dt = workload_mesh(W)
    pulse = synth.plane_wave_pulse(seed=synth.SEED_BASE + rank)
    N = W["N"]
    L = N + 1
    Ls = L // 2 + 1
    M = m.nt
    params = dict(mode="h2maca", eta=W["eta"], cheb_m=W["cheb_m"], n_min=W["n_min"],
                  aca_eps=W["aca_eps"], profile=1)
    if args.tensor_cores is not None:
        params["tensor_cores"] = args.tensor_cores
    if args.expand_far is not None:
        params["expand_far"] = args.expand_far
    stream = torch.cuda.current_stream()
    rhs = torch.empty((L, M), dtype=torch.float64, device="cuda")
    q = torch.empty((L, M), dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    mot = args.scheme == "mot"
    dirichlet = args.scheme == "dirichlet"
    # Dirichlet data of sound-soft scattering: g = -u_inc on the boundary, as
    # P0 coefficients (the Galerkin data divided by the element areas)
    P = m.xyz[m.tri]
    area = torch.from_numpy(0.5 * np.linalg.norm(np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), axis=1)).cuda()

    def step():
        op = CqmBem(m.xyz, m.tri, dt, N, W["bdf"], **params)
        op.rhs_plane_wave(pulse.direction, pulse.width, pulse.delay, out=rhs)
        if mot:
            op.solve_mot(rhs, out=q)
        elif dirichlet:
            rhs.div_(area).neg_()
            op.solve_dirichlet(rhs, out=q)
        else:
            op.solve(rhs, out=q)
        return op

    for _ in range(args.warmup):
        step().close()
    torch.cuda.synchronize()
    barrier(world)
    times, prof, infos, sinfos = [], {}, [], []
    with ClockSampler(torch.cuda.current_device()) as clk:
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            op = step()
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
            for k, (n, ms) in op.profile_read().items():
                a = prof.setdefault(k, [0, 0.0])
                a[0] += n
                a[1] += ms
            infos.append(dict(op.info(), tensor_cores=int(op.params.tensor_cores)))
            sinfos.append(op.last_solve_info)
            op.close()
    torch.cuda.synchronize()
    barrier(world)
    total = sum(times)
    value, tmax = whole_job_value(M * L, args.steps, total, world)

    # end to end through the public API with host buffers
    rhs_host = torch.empty((L, M), dtype=torch.float64, pin_memory=True)
    rhs_host.copy_(rhs.cpu())
    q_host = torch.empty((L, M), dtype=torch.float64, pin_memory=True)
    e2e_times = []
    barrier(world)
    for _ in range(0 if args.no_e2e else max(1, args.steps)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        op = CqmBem(m.xyz, m.tri, dt, N, W["bdf"], **params)
        if mot:
            op.solve_mot(rhs_host.numpy(), out=q_host.numpy())
        elif dirichlet:
            op.solve_dirichlet(rhs_host.numpy(), out=q_host.numpy())
        else:
            op.solve(rhs_host.numpy(), out=q_host.numpy())
        op.close()
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
    e2e_value = (whole_job_value(M * L, len(e2e_times), sum(e2e_times), world)[0]
                 if e2e_times else None)

    # the workload's per-frequency solution, for the oracle comparison (untimed)
    qhat_gpu = None
    if rank == 0 and not args.no_cpu_baseline and world == 1 and not mot and not dirichlet:
        op = CqmBem(m.xyz, m.tri, dt, N, W["bdf"], **params)
        g = op.forward_transform(rhs)
        qhat_gpu = op.solve_frequencies(g)[0].cpu().numpy()
        op.close()
    tf32_measured = measure_tf32_peak() if rank == 0 else None
    if rank != 0:
        return
    peaks, src = _peaks()
    inf = infos[-1]
    dom = max(prof.items(), key=lambda kv: kv[1][1])
    p = W["cheb_m"] ** 3
    lps = {k: v[0] / args.steps for k, v in prof.items()}
    models = kernel_models(inf, Ls, p, inf["tensor_cores"], tf32_measured, sinfos[-1], lps)
    if mot:
        models.update(mot_models(inf, N, lps))
    lat = sorted(times)
    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": ("mixed: bf16x3 tensor-core far coupling and fp32 near field in the inner GMRES "
                  "iterations, float-float (~48-bit) residual applies and MACA kernel evaluations, "
                  "fp64 MACA pivots and updates, DFTs, preconditioner and Krylov basis"),
        "data": "synthetic",
        "config": {"workload": W["name"], "triangles": M, "N": N, "L": L, "Ls": Ls, "dt": dt,
                   "bdf": 2, "eta": W["eta"], "cheb_m": W["cheb_m"], "leaf": W["n_min"],
                   "aca_eps": W["aca_eps"], "mode": "h2maca", "parallelism": f"replicas{world}",
                   "far_coupling": {1: "tcgen05 bf16 x3", 2: "tcgen05 tf32 x3"}.get(inf["tensor_cores"], "fp32 simt"),
                   "far_single_product_terms": (f"{inf.get('tc_single_terms', 0)} of {inf['rank_sum_far']} "
                                                "(trailing terms <= 1e-3 of the largest far term at every frequency)"),
                   "l2": "256 MB buffer written between timed steps; working set "
                         f"{inf['device_bytes'] / 2**30:.1f} GiB > L2"},
        "latency_ms": {"p50": 1e3 * lat[len(lat) // 2],
                       "p99": 1e3 * lat[min(len(lat) - 1, int(0.99 * len(lat)))]},
        "accuracy": {"gmres_max_rel_residual": max(s["max_rel_residual"] for s in sinfos),
                     "converged_frequencies": min(s["converged"] for s in sinfos), "Ls": Ls},
        "roofline": roofline_of(prof, models),
        "roofline_all": {k: roofline_of({k: prof[k]}, models) for k in models if k in prof and prof[k][0]},
        "roofline_time_weighted": time_weighted_frac(prof, models),
        "dominant_kernel": {"name": dom[0], "launches": dom[1][0], "ms": dom[1][1]},
        "kernel_ms": {k: round(v[1], 3) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1]) if v[0]},
        "gpu_launches": int(sum(v[0] for v in prof.values())),
        "setup": dict({k: inf[k] for k in ("n_nodes", "n_near", "n_far", "rank_sum_near", "rank_sum_far",
                                           "rank_max", "t_tree_ms", "t_bases_ms", "t_assembly_ms",
                                           "near_expanded", "far_expanded")},
                      total_ms=inf["t_geometry_ms"] + inf["t_tree_ms"] + inf["t_bases_ms"] + inf["t_assembly_ms"]),
        "solve": dict({k: sinfos[-1][k] for k in ("iterations", "restarts", "t_gmres_ms", "arnoldi_freq_steps",
                                                 "restart_freq_applies")},
                      total_ms=sinfos[-1]["t_forward_ms"] + sinfos[-1]["t_gmres_ms"] + sinfos[-1]["t_inverse_ms"]),
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(L * M * 8 + m.xyz.nbytes + m.tri.nbytes),
                "d2h_bytes_per_step": int(L * M * 8)},
        "peaks_source": src,
    }
    line["roofline_peaks"] = {"tf32_tflops": tf32_measured}
    if args.step_error:
        try:
            line["step_error"] = step_error(m, dt, pulse, W, params, q)
        except Exception as e:  # the reference did not fit or failed: report it
            line["step_error"] = {"error": str(e)}
    if args.dense_baseline:
        line["dense_fp64_gpu"] = dense_baseline(m, pulse, W, q)
    if mot:
        line["scheme"] = ("marching on in time (Sec. 3.2) with the compressed weights "
                          "(eqs. fastdft, fastrhs)")
        line["dtype"] = ("fp64 weights, Vhat_0 inverse and step solve; float-float (~48-bit) history sums "
                         "and MACA kernel evaluations; fp64 MACA pivots")
        op = CqmBem(m.xyz, m.tri, dt, N, W["bdf"], **dict(params, profile=0))
        qd = op.solve(rhs).cpu().numpy()
        op.close()
        a = q.cpu().numpy()
        line["accuracy"]["mot_vs_decoupled"] = float(
            np.max(np.linalg.norm(a - qd, axis=1)) / np.max(np.linalg.norm(qd, axis=1)))
        line["accuracy"]["note"] = ("the march is exactly causal; the decoupled solve carries the "
                                    f"O(R^L) = {cqm_R(N) ** (N + 1):.1e} aliasing of the CQM transform")
    if dirichlet:
        line["scheme"] = ("direct formulation of sound-soft scattering (Sec. 7.2, eq. cqmdir) decoupled "
                          "in frequency: V qhat = (-1/2 M + K) ghat, g = -u_inc")
    if not args.no_cpu_baseline and world == 1 and not mot and not dirichlet:  # rank 0 at N = 1 only
        cb, qref = cpu_baseline()
        line["cpu_baseline"] = cb
        errs = {int(l): float(np.max(np.abs(qhat_gpu[l] - ref)) / np.max(np.abs(ref)))
                for l, ref in qref.items()}
        line["accuracy"]["rel_err_vs_oracle"] = max(errs.values())
        line["accuracy"]["rel_err_vs_oracle_per_frequency"] = errs
        line["accuracy"]["oracle_note"] = (
            "max_i |qhat_l[i] - ref_l[i]| / max_i |ref_l[i]| at the sampled solved frequencies, "
            "ref = LU of the FP64 oracle's H^2-expanded V_l (same tree and interpolation, no MACA)")
    print(json.dumps(line), flush=True)


def step_error(m, dt, pulse, W, params, q):
    """Error of the timed path per time step against the same solver with the
    MACA at 1e-11 (its residuals are FP64-accurate; the path is pinned to the
    oracle at smaller sizes): max_n and selected steps of
    ||q_n - q_n^ref|| / max_n ||q_n^ref||."""
    import torch
    from paper_2006_05186_gb300 import CqmBem
    N = W["N"]
    kw = dict(params, aca_eps=W.get("ref_eps", 1e-11), rank_cap=W.get("ref_cap", 64), profile=0)
    op = CqmBem(m.xyz, m.tri, dt, N, W["bdf"], **kw)
    rhs = op.rhs_plane_wave(pulse.direction, pulse.width, pulse.delay)
    qr = op.solve(rhs)
    op.close()
    torch.cuda.empty_cache()
    a = q.cpu().numpy()
    e = np.linalg.norm(a - qr, axis=1) / np.max(np.linalg.norm(qr, axis=1))
    picks = sorted(set([0, N // 4, N // 2, 3 * N // 4, N, int(np.argmax(e))]))
    return {"max": float(e.max()), "worst_step": int(np.argmax(e)),
            "steps": {int(n): float(e[n]) for n in picks},
            "reference": f"same path, MACA {kw['aca_eps']:g}, rank_cap {kw['rank_cap']}"}


def dense_baseline(m, pulse, W, q_compressed):
    """One timed pass of the plain dense FP64 GPU path (dense V_l for every
    solved frequency, FP64 GMRES) on the same workload, and the time-domain
    difference of the two solutions (the H^2 interpolation error)."""
    import torch
    from paper_2006_05186_gb300 import CqmBem
    N = W["N"]
    _, dt = workload_mesh(W)
    L, M = N + 1, m.nt
    rhs = torch.empty((L, M), dtype=torch.float64, device="cuda")
    qd = torch.empty((L, M), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    op = CqmBem(m.xyz, m.tri, dt, N, W["bdf"], mode="dense")
    op.rhs_plane_wave(pulse.direction, pulse.width, pulse.delay, out=rhs)
    op.solve(rhs, out=qd)
    e1.record()
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) / 1e3
    info = op.last_solve_info
    op.close()
    a, b = q_compressed.cpu().numpy(), qd.cpu().numpy()
    diff = float(np.max(np.linalg.norm(a - b, axis=1)) / np.max(np.linalg.norm(b, axis=1)))
    return {"value": M * L / sec, "unit": UNIT, "seconds": sec, "steps": 1,
            "gmres_iterations": info["iterations"],
            "rel_diff_compressed_vs_dense": diff,
            "note": "one pass, no warm-up; the difference is the H^2 interpolation error (eta = 1, m = 4)"}


def oracle_frequencies(freqs, workers=None):
    """The FP64 oracle as it stands on solved frequencies `freqs` of the
    benchmark workload: cluster tree and partition, plane-wave data and its
    R-scaled transform, H^2-expanded assembly of V_l (every near-field pair by
    its quadrature rule, every far block as U_r S_b U_c^T) and one LAPACK LU
    per frequency, evaluated over a process pool on the host cores.
    Returns (qhat (len(freqs), M), seconds, workers)."""
    from oracle import cluster, cqm, incident, pool
    from paper_2006_05186_gb300 import synth
    W = WORKLOAD
    workers = workers or pool.default_workers()
    m, dt = workload_mesh(W)
    p = synth.plane_wave_pulse()
    t0 = time.perf_counter()
    t = cluster.build_tree(m.xyz, m.tri, W["n_min"])
    near, far = cluster.partition(t, W["eta"])
    b = incident.rhs_plane_wave(m.xyz, m.tri, W["N"], dt, p.direction, p.width, p.delay)
    g = cqm.forward(b, cqm.default_R(W["N"]))[freqs]
    s = cqm.frequencies(W["N"], dt, W["bdf"])[freqs]
    q = pool.h2_solve_frequencies(m.xyz, m.tri, s, t, near, far, W["cheb_m"], g, workers=workers)
    return q, time.perf_counter() - t0, workers


def cpu_baseline():
    """The oracle on a bounded sample of the workload: one run on the middle
    solved frequency and one on the first and last, each timed whole.  The
    job time a + b Ls is fitted from the two runs (a: tree, data and set-up
    shared by all frequencies; b: assembly and LU of one frequency).  Also
    returns the oracle's qhat at the three frequencies."""
    W = WORKLOAD
    L = W["N"] + 1
    Ls = L // 2 + 1
    M = workload_mesh(W)[0].nt
    f1, f2 = [Ls // 2], [0, Ls - 1]
    q1, t1, workers = oracle_frequencies(f1)
    q2, t2, _ = oracle_frequencies(f2)
    b = t2 - t1 if t2 > t1 else t1
    a = max(0.0, t1 - b)
    est = a + b * Ls
    qref = {f1[0]: q1[0], f2[0]: q2[0], f2[1]: q2[1]}
    return {"value": M * L / est, "unit": UNIT, "cores": workers, "kind": "oracle",
            "sample": (f"the {W['name']} workload on 3 of its {Ls} solved frequencies (l = {f2[0]}, "
                       f"{f1[0]}, {f2[1]}) in two timed runs ({t1:.1f} s for one frequency, {t2:.1f} s "
                       f"for two): the FP64 oracle's H^2-expanded assembly and LU per frequency over "
                       f"a spawn process pool of {workers} workers (one BLAS thread each); job time "
                       f"a + b Ls with a = {a:.1f} s, b = {b:.1f} s per frequency, est. {est:.0f} s")}, qref


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    times = []
    cb = None
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        cb, _ = cpu_baseline()
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    W = WORKLOAD
    M = workload_mesh(W)[0].nt
    L = W["N"] + 1
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / max(1, len(times)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": W["name"], "triangles": M, "N": W["N"], "L": L,
                       "mode": "oracle H^2-expanded + LU (3 sampled frequencies per step)"},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def draw_requests(kind, count, seed0=20060518):
    """Seeded scatterers of the batched and serving workloads.  Draws per
    request, in this order, from numpy.random.default_rng(seed0 + i): shape,
    size, N, semi-axes (ellipsoid), direction (serving), width, delay."""
    from paper_2006_05186_gb300 import synth
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed0 + i)
        if kind == "batch":
            shape = ["sphere", "ellipsoid", "cube"][rng.integers(3)]
            level = [2, 3, 4][rng.integers(3)]
            N = [64, 128, 256, 512][rng.integers(4)]
        else:
            shape = ["sphere", "ellipsoid", "torus"][rng.integers(3)]
            level = [3, 4][rng.integers(2)]
            N = [128, 256, 512][rng.integers(3)]
        axes = rng.uniform(0.5, 2.0, 3)
        if shape == "sphere":
            m = synth.icosphere(level)
        elif shape == "ellipsoid":
            m = synth.ellipsoid(level, axes)
        elif shape == "cube":
            m = synth.rounded_cube(level)
        else:
            m = synth.torus_for(20 * 4 ** level)
        if kind == "batch":
            d = np.array([0.0, 0.0, 1.0])
            w = 0.5
        else:
            d = rng.standard_normal(3)
            d /= np.linalg.norm(d)
            w = float(rng.uniform(0.2, 1.0))
        size = float(np.max(np.linalg.norm(m.xyz, axis=1)))
        delay = size + 4.0 * w + float(rng.uniform(0.0, w))
        out.append(dict(shape=shape, m=m, N=N, dt=0.4 * synth.mean_edge_length(m), dir=d, width=w,
                        delay=delay))
    return out


def serve_requests(reqs, workers, arrivals=None):
    """Runs the requests through a server; returns per-request infos and the
    wall time from the first submit to the last result."""
    from paper_2006_05186_gb300 import Server
    srv = Server(workers=workers)
    t0 = time.perf_counter()
    tickets = []
    for k, r in enumerate(reqs):
        if arrivals is not None:
            wait = t0 + arrivals[k] - time.perf_counter()
            if wait > 0:
                time.sleep(wait)
        tickets.append(srv.submit(r["m"].xyz, r["m"].tri, r["dt"], r["N"], direction=r["dir"],
                                  width=r["width"], delay=r["delay"], aca_eps=1e-9, expand_far=0))
    infos = []
    for t in tickets:
        code, _, info = srv.poll(t)
        if code != 0:
            raise RuntimeError(f"request {t} failed with status {code}")
        infos.append(info)
    wall = time.perf_counter() - t0
    srv.close()
    return infos, wall


def run_many(args):
    """Batched (64 seeded scatterers, all submitted at once) or serving
    (a Poisson stream of seeded requests, mean 20 per second) through the
    request server, against the same requests run one at a time."""
    import torch
    torch.cuda.set_device(0)
    kind = "batch" if args.workload == "batch64" else "serve"
    count = 64 if kind == "batch" else args.requests
    reqs = draw_requests(kind, count)
    units = sum(r["m"].nt * (r["N"] + 1) for r in reqs)
    arrivals = None
    if kind == "serve":
        gaps = np.random.default_rng(20060518 + 999).exponential(1.0 / 20.0, count)
        arrivals = np.cumsum(gaps) - gaps[0]
    serve_requests(reqs[:2], 1)  # warm-up: module load, pools
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        infos, wall = serve_requests(reqs, args.workers, arrivals)
    seq_infos, seq_wall = serve_requests(reqs, 1, arrivals)
    lat = sorted(i["t_total_ms"] for i in infos)
    slat = sorted(i["t_total_ms"] for i in seq_infos)
    pct = lambda v, q: v[min(len(v) - 1, int(q * len(v)))]
    line = {
        "metric": METRIC, "value": units / wall, "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 1,
        "ms_per_step": 1e3 * wall, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "mixed (as the single-solve line)", "data": "synthetic",
        "config": {"workload": args.workload, "requests": count, "workers": args.workers,
                   "triangles": [r["m"].nt for r in reqs], "N": [r["N"] for r in reqs],
                   "shapes": [r["shape"] for r in reqs], "aca_eps": 1e-9, "expand_far": 0,
                   "arrivals": "Poisson, mean 20/s" if kind == "serve" else "all at t = 0"},
        "latency_ms": {"p50": pct(lat, 0.5), "p99": pct(lat, 0.99)},
        "sequential": {"value": units / seq_wall, "unit": UNIT, "seconds": seq_wall,
                       "latency_ms": {"p50": pct(slat, 0.5), "p99": pct(slat, 0.99)},
                       "note": "the same requests through one worker (one at a time)"},
        "max_rel_residual": max(i["solve"]["max_rel_residual"] for i in infos),
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--dense-baseline", action="store_true",
                    help="also time one pass of the dense FP64 GPU path on the same workload")
    ap.add_argument("--level", type=int, default=None,
                    help="icosphere level override (smaller cases for profiler captures)")
    ap.add_argument("--N", type=int, default=None, help="time-step count override")
    ap.add_argument("--tensor-cores", type=int, choices=[0, 1, 2], default=None,
                    help="far-field coupling on the tensor cores in bf16 (1), TF32 (2), or FP32 SIMT (0)")
    ap.add_argument("--scheme", choices=["decoupled", "mot", "dirichlet"], default="decoupled",
                    help="the decoupled single-layer solve, marching on in time, or the direct "
                         "Dirichlet formulation with the double layer")
    ap.add_argument("--expand-far", type=int, choices=[0, 1], default=None,
                    help="override the expanded far table of the FP64-accurate apply")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["batch64", "serve"],
                    default="sphere5120_N256")
    ap.add_argument("--workers", type=int, default=6, help="server workers (batch64, serve)")
    ap.add_argument("--requests", type=int, default=40, help="requests of the serving stream")
    ap.add_argument("--step-error", action="store_true",
                    help="also solve with the MACA at 1e-11 and report the error per time step")
    args = ap.parse_args()
    if args.workload in ("batch64", "serve"):
        run_many(args)
        return
    if args.workload != "sphere5120_N256":
        WORKLOAD.clear()
        WORKLOAD.update(WORKLOADS[args.workload])
    if args.level is not None:
        WORKLOAD["level"] = args.level
        WORKLOAD["name"] = f"sphere{20 * 4 ** args.level}_N{WORKLOAD['N']}"
    if args.N is not None:
        WORKLOAD["N"] = args.N
        WORKLOAD["name"] = f"sphere{20 * 4 ** WORKLOAD['level']}_N{args.N}"
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
