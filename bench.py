#!/usr/bin/env python
"""FOSB benchmark: one step = one full pass of the FOSB hot path on the mixed-precision
sphere workload -- for every level of a nested icosphere hierarchy (80 .. 20480
triangles, 120 .. 30720 RWG unknowns, k a = 4): EFIE assembly + plane-wave RHS, LU
(complex64 factors) with FP64 iterative refinement, the mean far field at 181 H-plane
angles, and the combination-technique far-field covariance over L0 = 0, L = 4 (blocks
(4,0), (3,1), (2,2), (3,0), (2,1); Gaussian covariance sigma = 0.005, l = 0.3).

Prints one JSON line.  `value` is the device-timed seconds per FOSB step with the
meshes resident on the GPU (lower is better); `e2e` is the same step through the
public API from host arrays (mesh upload, result download).  `--impl reference` times
the FP64 CPU oracle: a complete oracle step one level below the workload's finest,
measured end to end, extended to the workload by a cost model whose error is measured
one level further down.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FOSB covariance time & EFIE entries/s, mixed vs FP64 on one GB300 at 1e-8 rel err"

WORKLOADS = {
    # mixed-precision sphere, levels l = 0..4 are icospheres of T = 80 * 4**l triangles
    "sphere-ka4-ct-L4": dict(mesh="sphere", levels=[0, 1, 2, 3, 4], k=4.0, sigma=0.005, ell=0.3, n_dir=181, L0=0, L=4,
                             d=(0, 0, 1), p=(1, 0, 0), dirs="hplane", kernel="gauss"),
    # smaller cases of the same kernels (profiling captures)
    "sphere-ka4-ct-L3": dict(mesh="sphere", levels=[0, 1, 2, 3], k=4.0, sigma=0.005, ell=0.3, n_dir=181, L0=0, L=3,
                             d=(0, 0, 1), p=(1, 0, 0), dirs="hplane", kernel="gauss"),
    "sphere-ka4-ct-L2": dict(mesh="sphere", levels=[0, 1, 2], k=4.0, sigma=0.005, ell=0.3, n_dir=181, L0=0, L=2,
                             d=(0, 0, 1), p=(1, 0, 0), dirs="hplane", kernel="gauss"),
    # largest: torus R = 1, r = 0.35, levels 1..5 = grids 10x4 .. 160x64 (T = 80 .. 20480), k a = 10,
    # Matern-3/2 (std 0.002, l = 0.2), 361 directions in the z = 0 plane, d = x, p = z
    "torus-ka10-ct-L5": dict(mesh="torus", levels=[1, 2, 3, 4, 5], k=10.0, sigma=0.002, ell=0.2, n_dir=361, L0=1,
                             L=5, d=(1, 0, 0), p=(0, 0, 1), dirs="zplane", kernel="matern32"),
    # batched: 64 seeded ellipsoids (semi-axes U[0.5, 1.5], k U[1, 6], icosphere level 2..4:
    # N = 480 / 1920 / 7680), 16 Fibonacci incident directions each; assembly, complex64 LU
    # with FP64 refinement and the 16 solves of every scatterer
    "batched-ellipsoids-64": dict(kind="batched", n=64, n_dir=16),
    # Monte Carlo: 512 sample surfaces x_p + xi_p n_p, xi ~ N(0, K) (Gaussian sigma = 0.005,
    # l = 0.3), of the 1280-triangle sphere (N = 1920), k = 4, d = +z, p = x, 181 H-plane angles
    "mc-sphere-ka4-N1920-M512": dict(kind="mc", level=3, nsamp=512, k=4.0, sigma=0.005, ell=0.3, n_dir=181,
                                     d=(0, 0, 1), p=(1, 0, 0), seed=230801457),
    # the CT check of Section V-A on the dielectric sphere (k0 = 3, eps_r = 2.1, d = x, p = z,
    # 1801 angles in the z = 0 plane): rank-one tensor right-hand side f (x) f over icosphere
    # levels 0..3 (80 .. 5120 triangles, 2N = 240 .. 15360), L0 = 0, L = 3
    "ct-dielectric-sphere-k3-L3": dict(kind="dect", levels=[0, 1, 2, 3], k=3.0, eps_r=2.1, mu_r=1.0, n_dir=1801,
                                       d=(1, 0, 0), p=(0, 0, 1), L0=0, L=3),
    # Monte Carlo for the dielectric sphere of Section V-A (k0 = 3, eps_r = 2.1, d = x, p = z):
    # 128 sample surfaces of the 1280-triangle sphere (2N = 3840), each solved by the PMCHWT
    # system; Gaussian sigma = 0.005, l = 0.3; 181 angles in the z = 0 plane
    "mc-dielectric-sphere-k3-N3840-M128": dict(kind="mc", level=3, nsamp=128, k=3.0, sigma=0.005, ell=0.3,
                                               n_dir=181, d=(1, 0, 0), p=(0, 0, 1), seed=230801457, eps_r=2.1,
                                               mu_r=1.0, dirs="zplane"),
    # low-rank right-hand side (Section VI): the full tensor of one level (L0 = L = 3: the
    # 5120-triangle sphere, N = 7680, V = 2562), k = 4, Gaussian sigma = 0.005, l = 0.3, 181
    # H-plane angles; the kernel factored by pivoted Cholesky to a relative trace error of
    # 1e-10, timed against the full path (V right-hand sides) on the same problem
    "lowrank-sphere-ka4-full-L3": dict(kind="lowrank", mesh="sphere", levels=[3], k=4.0, sigma=0.005, ell=0.3,
                                       n_dir=181, L0=3, L=3, d=(0, 0, 1), p=(1, 0, 0), dirs="hplane",
                                       kernel="gauss", tol=1e-10),
    # dielectric sphere by the PMCHWT system (Section II-C; Section V-A, Table I: k0 = 3,
    # eps_r = 2.1, mu_r = 1, d = x, p = z, 1801 angles in the z = 0 plane): the icosphere of
    # 5120 triangles, 2N = 15360 unknowns; assembly of both wavenumbers, complex64 LU with
    # FP64-class refinement, far field of the exterior Cauchy data
    "pmchwt-sphere-k3-N15360": dict(kind="pmchwt", level=4, k=3.0, eps_r=2.1, mu_r=1.0, n_dir=1801,
                                    d=(1, 0, 0), p=(0, 0, 1), oracle_level=3),
    # the same kernels one level down (1280 triangles, 2N = 3840; Z 236 MB > L2): profiling captures
    "pmchwt-sphere-k3-N3840": dict(kind="pmchwt", level=3, k=3.0, eps_r=2.1, mu_r=1.0, n_dir=1801,
                                   d=(1, 0, 0), p=(0, 0, 1), oracle_level=2),
}

TF32_PER_BF16 = 1.1 / 2.25  # nominal dense TF32 / BF16 tensor ratio of the part
LU_BLOCK = 256  # column block of the complex64 LU: every trailing update has K = 256
# DRAM bytes (read + write) per complex64 output element of one tcgen05 LU-update launch,
# from the ncu capture summarised in profiles/ (C is read and written once: 16 B algorithmic)
LU_UPDATE_DRAM_BYTES_PER_OUTPUT = (653.6512e6 + 390.073344e6) / 7424.0**2  # 18.94 B


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {}


def _meshes(W):
    import fosb_synth as S

    if W["mesh"] == "torus":
        return S.torus_hierarchy(W["levels"])
    return [S.icosphere(l + 1) for l in W["levels"]]


def _dirs(W):
    import fosb_synth as S

    return S.zplane_directions(W["n_dir"]) if W["dirs"] == "zplane" else S.hplane_directions(W["n_dir"])


def _n_edges(W, l):
    return 120 * 4 ** (l - 1) if W["mesh"] == "torus" else 120 * 4**l


def _problem(F, W, meshes, dirs, prec, arith):
    from paper_2308_01457_gb300.ct import FOSBProblem

    kern = F.COV_MATERN32 if W["kernel"] == "matern32" else F.COV_GAUSS
    return FOSBProblem(meshes, W["k"], W["d"], W["p"], dirs, W["L0"], W["L"], kern, W["sigma"], W["ell"], prec=prec,
                       arith=arith).setup()


def _clock_sampler(gpu_index: int):
    try:
        return subprocess.Popen(
            ["nvidia-smi", "-i", str(gpu_index),
             "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
             "--format=csv,noheader,nounits", "-lms", "200"],
            stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except OSError:
        return None


def _clock_summary(proc):
    if proc is None:
        return None
    proc.terminate()
    try:
        out, _ = proc.communicate(timeout=5)
    except subprocess.TimeoutExpired:
        proc.kill()
        out, _ = proc.communicate()
    sm, smax, reasons = [], 0.0, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in out.strip().splitlines():
        f = [x.strip() for x in line.split(",")]
        if len(f) < 8:
            continue
        try:
            sm.append(float(f[0]))
            smax = max(smax, float(f[1]))
        except ValueError:
            continue
        for n, v in zip(names, f[4:8]):
            if v.lower().startswith("active"):
                reasons.add(n)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _max_over_ranks(value: float, ws: int, device: str = "cuda") -> float:
    """The largest of the ranks' values (the whole job's time per step: every replica has
    finished its step when the slowest has).  One rank: the value itself."""
    if ws <= 1:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------- GPU arm
def run_fosb(args):
    import torch

    import paper_2308_01457_gb300 as F

    F.build.build()
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    W = WORKLOADS[args.workload]
    meshes = _meshes(W)
    dirs = _dirs(W)
    arith = F.ASM_FF if args.arith == "ff" else F.ASM_FP64
    # the library's own throughput microbenchmarks (FP32/FP64 FMA, back-to-back tcgen05 MMAs)
    upeaks = {kd: round(F.peak_microbench(kd), 2) for kd in ("fp32", "fp64", "tf32", "bf16")}
    prob = _problem(F, W, meshes, dirs, F.MIXED, arith)
    L = W["L"]
    N = {l: prob.levels[l].mesh.n_edges for l in prob.levels}

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        prob.run()
        prob.release()
    barrier()
    launches0 = F.lib().fosb_kernel_launches()
    clocks = _clock_sampler(local) if rank == 0 else None
    # the timed region: K steps and one event per step boundary, nothing else recorded
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record()
    for i in range(args.steps):
        out = prob.run()
        prob.release()
        ev[i + 1].record()
    barrier()
    clk = _clock_summary(clocks)
    launches = int(F.lib().fosb_kernel_launches() - launches0)
    step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    ms = _max_over_ranks(ev[0].elapsed_time(ev[-1]) / args.steps, ws, "cuda")
    # after it, a profiled pass of two steps: per-phase and per-kernel-family CUDA events
    import ctypes

    families = ["lu_update", "lu_update64", "lu_panel", "asm_regular", "asm_singular", "gemm_ff", "gemm_oz",
                "trsm_update", "oz_prep", "getrs"]
    for fam in families:  # clear earlier records
        F.lib().fosb_profile_read(fam.encode(), None, None, None)
    timers = {}
    prof_steps = 2
    # sequential levels in the profiled pass: with the two streams of the timed step the
    # events of concurrent families would overlap, and each family's time must be its own
    prob.overlap = False
    F.lib().fosb_profile_enable(1)
    for _ in range(prof_steps):
        prob.run(timers)
        prob.release()
    torch.cuda.synchronize()
    F.lib().fosb_profile_enable(0)
    prob.overlap = True
    fam_stats = {}
    for fam in families:
        ms_c, n_c, w_c = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double()
        F.lib().fosb_profile_read(fam.encode(), ctypes.byref(ms_c), ctypes.byref(n_c), ctypes.byref(w_c))
        fam_stats[fam] = {"ms_per_step": ms_c.value / prof_steps, "launches_per_step": n_c.value / prof_steps,
                          "work_per_step": w_c.value / prof_steps}

    def avg(name):
        v = timers.get(name, [])
        return sum(a.elapsed_time(b) for a, b in v) / max(1, len(v))

    t_asm = avg(f"assemble_l{L}")
    t_fac = avg(f"factor_l{L}")
    t_sol = avg(f"solve_l{L}")
    t_cov = avg("covariance_ct")
    NL = N[L]
    T = prob.levels[L].mesh.nt
    peaks = _peaks()
    # kernels timed inside the long step take the sustained peak: measured bf16 sustained (or
    # the pool's fallback 1.7 PFLOP/s) x the nominal TF32/bf16 ratio for the TF32 contraction
    bf16 = peaks.get("bf16_tflops_sustained", 1700.0)
    bf16_src = "of measured" if "bf16_tflops_sustained" in peaks else "of fallback"
    tf32_peak = bf16 * TF32_PER_BF16
    fp_peak = upeaks["fp32"] if arith == F.ASM_FF else upeaks["fp64"]
    # algorithmic work -> (bound, flops, peak, kernel, note) per family
    fam_model = {
        "lu_update": ("tensor", 1.0, tf32_peak,
                      "cgemm_update_split_kernel (persistent tcgen05 kind::tf32 N = 256, 3xTF32 complex, operands "
                      "split once per block and bulk-copied; the split kernels are timed with it)",
                      f"TF32 dense = bf16 sustained {bf16} ({bf16_src}) x 1.1/2.25; work = useful complex flops "
                      "8MNK; 3xTF32 executes 3x that on the tensor pipe (tensor_pipe_frac: executed TF32 rate / "
                      "the TF32 MMA rate fosb_peak_microbench measures, which is above the nominal-ratio peak)"),
        "lu_update64": ("tensor", 1.0, tf32_peak,
                        "cgemm_update_tc_ws_kernel (the K = 64 updates inside each 256-column block of the LU)",
                        "work = useful complex flops 8MNK"),
        "asm_regular": ("alu", 27.0, fp_peak,
                        "efie_regular_ff_kernel" if arith == F.ASM_FF else "efie_regular_kernel<double>",
                        "27 algorithmic FP ops per point pair; peak = the FP32 (float-float) or FP64 FMA pipe "
                        "measured by fosb_peak_microbench"),
        "gemm_ff": ("alu", 1.0, upeaks["fp32"], "zgemm_ff_kernel (float-float complex128 GEMM)",
                    "work = complex128 flops 8MNK executed as ~48 FP32 instructions per complex MAC; "
                    "peak = measured FP32 FMA pipe"),
        "lu_panel": ("latency", 1.0, None, "tslu_gepp_kernel (tournament-pivoting panel)",
                     "latency-bound: 64 sequential pivot steps per tree level"),
        "gemm_oz": ("tensor", 1.0, bf16, "oz_gemm_kernel (bf16 digit-split tcgen05, FP64-class complex)",
                    "work = complex128 flops 8MNK; executes 112 bf16 MMAs (28 digit pairs x 4) per complex product, "
                    "so frac <= 8/(112 x 2)"),
        "trsm_update": ("tensor", 1.0, tf32_peak, "cgemm_update_tc_ws_kernel in the blocked triangular sweeps (K = 64)",
                        "sweep updates of solves with 16 or more right-hand sides; work = useful complex flops 8MNK"),
        "oz_prep": ("hbm", 1.0, peaks.get("hbm_gbs", 6800.0), "oz_row_exp_kernel + oz_split_a_kernel (digit tiles of Z)",
                    "work = bytes: 16 B read + 28 B of digits written per element of Z"),
        # the whole triangular solve; it contains the trsm_update launches, so it is not a
        # candidate for the dominant family
        "getrs": ("latency", 1.0, None, "getrs (permutation, sweeps, copies)", "container of trsm_update"),
    }
    dom = max((f for f in fam_model if fam_stats[f]["ms_per_step"] > 0 and f != "getrs"),
              key=lambda f: fam_stats[f]["ms_per_step"], default="lu_update")
    bound, wscale, peak, kname, note = fam_model[dom]
    st = fam_stats[dom]
    dom_scale, dom_unit = (1e9, "GB/s") if bound == "hbm" else (1e12, "TFLOP/s")
    achieved = st["work_per_step"] * wscale / (st["ms_per_step"] * 1e-3) / dom_scale if st["ms_per_step"] > 0 else 0.0
    roofline = {"bound": bound, "achieved": round(achieved, 3), "peak": round(peak, 2) if peak else None,
                "unit": dom_unit, "frac": round(achieved / peak, 4) if peak else None,
                "traffic": None, "kernel": kname, "family": dom,
                "ms_per_step": round(st["ms_per_step"], 2), "launches_per_step": st["launches_per_step"],
                "peak_source": note}
    if dom == "lu_update" and st["launches_per_step"] > 0:
        # DRAM bytes per launch from the ncu capture (bytes per output element of C, see
        # profiles/), scaled to the average launch of the timed region: C elements = flops /
        # (8 K) with K = 256, the depth of every trailing update of the 256-column blocking
        avg_outputs = st["work_per_step"] / (8.0 * LU_BLOCK * st["launches_per_step"])
        if LU_UPDATE_DRAM_BYTES_PER_OUTPUT is not None:
            roofline["traffic"] = round(LU_UPDATE_DRAM_BYTES_PER_OUTPUT * avg_outputs)
        roofline["algorithmic_bytes"] = round(16.0 * avg_outputs)
        if upeaks.get("tf32"):
            roofline["tensor_pipe_frac"] = round(3.0 * achieved / upeaks["tf32"], 4)
    secondary = {}
    for f, (b, wsc, pk, kn, _) in fam_model.items():
        s_ = fam_stats[f]
        unit_scale, unit = (1e9, "GB/s") if b == "hbm" else (1e12, "TFLOP/s")
        rate = s_["work_per_step"] * wsc / (s_["ms_per_step"] * 1e-3) / unit_scale if s_["ms_per_step"] > 0 else 0.0
        secondary[f] = {"ms_per_step": round(s_["ms_per_step"], 2), "launches_per_step": s_["launches_per_step"],
                        "rate": round(rate, 3), "unit": unit, "frac": round(rate / pk, 4) if pk else None}
    # IR quality (refined path must reach FP64 backward error)
    berr = max(prob.levels[l].berr for l in prob.levels)
    e2e = run_e2e(args, W, meshes, dirs, arith) if (rank == 0 and not args.no_e2e) else None
    fp64 = run_fp64_compare(W, meshes, dirs, out, ms) if (rank == 0 and not args.no_fp64) else None
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": round(ms / 1e3, 4), "unit": "s per FOSB step", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 2), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None,
        "dtype": "mixed: 3xTF32 tensor-core LU (c64 factors), float-float (f32x2) assembly and FP64-class "
                 "refinement residuals, f64 singular quadrature", "data": "synthetic",
        "config": {"workload": args.workload, "levels": W["levels"], "N_levels": [N[l] for l in sorted(N)],
                   "triangles_finest": T, "k": W["k"], "n_dir": W["n_dir"], "ct": [W["L0"], W["L"]],
                   "assembly": args.arith, "parallelism": f"replicas{ws}",
                   "l2": "inputs larger than L2 (Z at N=30720 is 15 GB)",
                   "profiling": "phase and kernel-family events from a separate 2-step pass after the timed region, with the levels run in sequence"},
        "median_step_ms": round(statistics.median(step_ms), 2),
        "efie_entries_per_s": round(NL * NL / (t_asm * 1e-3), 1),
        "phase_ms": {"assemble_finest": round(t_asm, 2), "factor_finest": round(t_fac, 2),
                     "solve_finest": round(t_sol, 2), "covariance_ct": round(t_cov, 2)},
        "ir_backward_error_max": berr,
        "roofline": roofline, "roofline_calls": secondary,
        "gpu_launches": launches,
        "clocks": clk,
        "e2e": e2e,
        "fp64": fp64,
        "hbm_peak_gbs": peaks.get("hbm_gbs"),
    }
    line["peaks_microbench_tflops"] = upeaks
    if not args.no_cpu_baseline:
        cb, Fo, covo = cpu_baseline(W, with_outputs=True)
        line["cpu_baseline"] = cb
        # the same workload one level down (every kernel and launch configuration of the step,
        # finest N = the oracle's measured step) on the GPU against the oracle's outputs
        W1 = dict(W, levels=W["levels"][:-1], L=W["L"] - 1)
        p1 = _problem(F, W1, meshes[:-1], dirs, F.MIXED, arith)
        F1, cov1 = (t.cpu().numpy() for t in p1.run())
        p1.release()
        line["oracle_parity"] = {
            "levels": [W["L0"], W["L"] - 1], "tolerance": 1e-8,
            "rel_err_mean_farfield": float(np.linalg.norm(F1[:, 0] - Fo) / np.linalg.norm(Fo)),
            "rel_err_ct_covariance": float(np.linalg.norm(cov1 - covo) / np.linalg.norm(covo))}
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def _batched_inputs(W):
    import fosb_synth as S

    table = S.batched_ellipsoid_table(W["n"])
    meshes = [S.ellipsoid(lvl, tuple(ax)) for ax, _, lvl in table]
    ks = [k for _, k, _ in table]
    d = S.fibonacci_directions(W["n_dir"])
    p = np.asarray(S.polarisation_for(d)).reshape(-1, 3)
    return table, meshes, ks, d, p


def run_batched(args):
    """The batched workload: one step = batched assembly (regular pairs of all 64 scatterers in
    one persistent launch, tile shape from the autotuner), then the batched factorisation and
    refined 16-column solve of every scatterer (worker streams, largest first)."""
    import ctypes

    import torch

    import paper_2308_01457_gb300 as F
    from paper_2308_01457_gb300.batched import BatchedProblem

    F.build.build()
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    W = WORKLOADS[args.workload]
    upeaks = {kd: round(F.peak_microbench(kd), 2) for kd in ("fp32", "fp64", "tf32", "bf16")}
    table, meshes, ks, d, p = _batched_inputs(W)
    prob = BatchedProblem(meshes, ks, d, p, workers=args.workers).setup()

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):  # the first warm-up step runs the autotuner
        prob.run(tune=True)
    barrier()
    launches0 = F.lib().fosb_kernel_launches()
    clocks = _clock_sampler(local) if rank == 0 else None
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record()
    for i in range(args.steps):
        prob.run(tune=True)
        ev[i + 1].record()
    barrier()
    clk = _clock_summary(clocks)
    launches = int(F.lib().fosb_kernel_launches() - launches0)
    step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    ms = _max_over_ranks(ev[0].elapsed_time(ev[-1]) / args.steps, ws, "cuda")
    # kernel-family events from a separate 2-step pass after the timed region
    families = ["lu_update", "lu_update64", "lu_panel", "asm_regular", "asm_singular", "gemm_ff", "gemm_oz", "oz_prep",
                "getrs"]
    for f in families:
        F.lib().fosb_profile_read(f.encode(), None, None, None)
    F.lib().fosb_profile_enable(1)
    for _ in range(2):
        prob.run(tune=True)
    torch.cuda.synchronize()
    F.lib().fosb_profile_enable(0)
    fam = {}
    for f in families:
        ms_c, n_c, w_c = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double()
        F.lib().fosb_profile_read(f.encode(), ctypes.byref(ms_c), ctypes.byref(n_c), ctypes.byref(w_c))
        fam[f] = (ms_c.value / 2, n_c.value / 2, w_c.value / 2)
    peaks = _peaks()
    bf16 = peaks.get("bf16_tflops_sustained", 1700.0)
    model = {"lu_update": ("tensor", 1.0, bf16 * TF32_PER_BF16, "cgemm_update_split_kernel"),
             "lu_update64": ("tensor", 1.0, bf16 * TF32_PER_BF16, "cgemm_update_tc_ws_kernel"),
             "asm_regular": ("alu", 27.0, upeaks["fp32"], "efie_regular_ff_batched_kernel (persistent, ticketed tiles)"),
             "lu_panel": ("latency", 1.0, None, "tslu_gepp_kernel"),
             "asm_singular": ("alu", 1.0, None, "efie_singular_batched_kernel"),
             "gemm_oz": ("tensor", 1.0, bf16, "oz_gemm_kernel"), "gemm_ff": ("alu", 1.0, upeaks["fp32"], "zgemm_ff_kernel"),
             "oz_prep": ("hbm", 1.0, peaks.get("hbm_gbs", 6800.0), "oz digit prep")}
    dom = max((f for f in model if fam[f][0] > 0), key=lambda f: fam[f][0])
    bound, wsc, pk, kname = model[dom]
    unit_scale, unit = (1e9, "GB/s") if bound == "hbm" else (1e12, "TFLOP/s")
    ach = fam[dom][2] * wsc / (fam[dom][0] * 1e-3) / unit_scale
    roofline = {"bound": bound, "achieved": round(ach, 3), "peak": round(pk, 2) if pk else None, "unit": unit,
                "frac": round(ach / pk, 4) if pk else None, "traffic": None, "kernel": kname, "family": dom,
                "ms_per_step": round(fam[dom][0], 2), "launches_per_step": fam[dom][1],
                "peak_source": "measured (MEASURED_PEAKS.json bf16 sustained x 1.1/2.25 for TF32; FP32 FMA pipe by "
                               "fosb_peak_microbench); family times overlap across the worker streams"}
    calls = {f: {"ms_per_step": round(v[0], 2), "launches_per_step": v[1]} for f, v in fam.items()}
    N = [h.n_edges for h in prob.handles]
    t_asm = fam["asm_regular"][0] + fam["asm_singular"][0]
    e2e = run_batched_e2e(args, W) if rank == 0 and not args.no_e2e else None
    if rank != 0:
        return
    line = {"metric": METRIC, "value": round(ms / 1e3, 4), "unit": "s per batch step", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 2), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "mixed: float-float (f32x2) regular pairs, f64 singular pairs, 3xTF32 tensor-core LU "
                     "(c64 factors) with FP64-class refinement", "data": "synthetic",
            "config": {"workload": args.workload, "scatterers": len(N),
                       "N_counts": {str(n): N.count(n) for n in sorted(set(N))}, "n_dir": W["n_dir"],
                       "k_range": [round(min(ks), 3), round(max(ks), 3)], "parallelism": f"replicas{ws}",
                       "tile_shape": {"warps": prob.tuning.warps, "ctas_per_sm": prob.tuning.ctas_per_sm,
                                      "tuned_ms": round(prob.tuning.tuned_ms, 3)},
                       "l2": "inputs larger than L2 (the 64 matrices are 16.4 GB)"},
            "median_step_ms": round(statistics.median(step_ms), 2), "solve_workers": args.workers,
            "scatterers_per_s": round(len(N) / (ms * 1e-3), 2),
            "efie_entries_per_s": round(sum(n * n for n in N) / (t_asm * 1e-3), 1) if t_asm > 0 else None,
            "ir_backward_error_max": max(prob.berr), "refinement_iters_max": max(prob.iters),
            "roofline": roofline, "roofline_calls": calls, "gpu_launches": launches, "clocks": clk, "e2e": e2e,
            "peaks_microbench_tflops": upeaks}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_batched(W)
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_batched_e2e(args, W):
    """The batched step through the public API from host arrays: mesh upload of all
    scatterers, assembly, factorisations and solves, and the download of every solution."""
    import torch

    from paper_2308_01457_gb300.batched import BatchedProblem

    _, meshes, ks, d, p = _batched_inputs(W)
    h2d = sum(m.verts.size * 8 + m.tris.size * 4 + m.vnormals.size * 8 for m in meshes)
    times = []
    for i in range(max(1, min(args.steps, 3)) + 1):
        torch.cuda.synchronize()
        t = time.perf_counter()
        prob = BatchedProblem(meshes, ks, d, p, workers=args.workers).setup()
        prob.run(tune=True)
        host = [x.cpu() for x in prob.X]
        torch.cuda.synchronize()
        if i > 0:
            times.append(time.perf_counter() - t)
        d2h = sum(x.numel() * 16 for x in host)
        del prob
    return {"value": round(statistics.median(times), 4), "unit": "s per batch step", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "steps": len(times)}


def run_mc(args):
    """The Monte Carlo workload: one step = the nominal solve, all sample surfaces (chunks of
    128: batched assembly and batched factor + solve), their far fields and the sample moments."""
    import torch

    import fosb_synth as S
    import paper_2308_01457_gb300 as F
    from paper_2308_01457_gb300.montecarlo import MonteCarloProblem

    F.build.build()
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    W = WORKLOADS[args.workload]
    sm = S.icosphere(W["level"])
    dirs = S.zplane_directions(W["n_dir"]) if W.get("dirs") == "zplane" else S.hplane_directions(W["n_dir"])
    z = S.gaussian_field_samples(W["nsamp"], sm.verts.shape[0], seed=W["seed"])
    prob = MonteCarloProblem(sm, W["k"], W["d"], W["p"], dirs, z, F.COV_GAUSS, W["sigma"], W["ell"], 1.0,
                             workers=args.workers, eps_r=W.get("eps_r"), mu_r=W.get("mu_r", 1.0),
                             arith=F.ASM_FF if args.arith == "ff" else F.ASM_FP64).setup()
    for _ in range(args.warmup):
        out = prob.run()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    launches0 = F.lib().fosb_kernel_launches()
    clocks = _clock_sampler(local) if rank == 0 else None
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record()
    for i in range(args.steps):
        out = prob.run()
        ev[i + 1].record()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = _clock_summary(clocks)
    launches = int(F.lib().fosb_kernel_launches() - launches0)
    ms = _max_over_ranks(ev[0].elapsed_time(ev[-1]) / args.steps, ws, "cuda")
    if rank != 0:
        return
    N = prob.base.n_edges
    line = {"metric": METRIC, "value": round(ms / 1e3, 4), "unit": "s per Monte Carlo run", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 2), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "mixed: float-float regular pairs, f64 singular pairs, 3xTF32 LU with FP64-class refinement",
            "data": "synthetic",
            "config": {"workload": args.workload, "N": N, "samples": W["nsamp"], "k": W["k"], "n_dir": W["n_dir"],
                       "sigma": W["sigma"], "ell": W["ell"], "scatterer": "PEC" if W.get("eps_r") is None else
                       f"dielectric eps_r = {W['eps_r']}, mu_r = {W.get('mu_r', 1.0)} (PMCHWT, 2N unknowns)",
                       "parallelism": f"replicas{ws}"},
            "samples_per_s": round(W["nsamp"] / (ms * 1e-3), 1), "gpu_launches": launches, "clocks": clk,
            "variance_far_field_max": float(np.diag(out[2].cpu().numpy()).real.max())}
    if not args.no_cpu_baseline:
        import oracle as O

        O.build()
        om = O.from_synth(sm)
        nsub = 8
        t = time.perf_counter()
        if W.get("eps_r") is None:
            O.monte_carlo(om, W["k"], W["d"], W["p"], dirs, "gauss", W["sigma"], W["ell"], 1.0, z[:nsub])
        else:
            O.monte_carlo_dielectric(om, W["k"], W["eps_r"], W.get("mu_r", 1.0), W["d"], W["p"], dirs, "gauss",
                                     W["sigma"], W["ell"], 1.0, z[:nsub])
        dt = time.perf_counter() - t
        line["cpu_baseline"] = {"value": round(dt / (nsub + 1) * (W["nsamp"] + 1), 2), "unit": "s per Monte Carlo run",
                                "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
                                "sample": f"oracle.monte_carlo on {nsub} of the {W['nsamp']} samples (plus the nominal "
                                          f"surface) in {dt:.1f} s, counted per surface (every surface costs the same)"}
    print(json.dumps(line), flush=True)


def run_lowrank(args):
    """The low-rank workload: one step = the FOSB step of fosb.ct with the kernel factored by
    pivoted Cholesky (fosb_kernel_lowrank) and the covariance formed as Y Y^H
    (fosb_covariance_lowrank, fosb_lowrank_combine).  Outside the timed region the same step
    on the full path (fosb_covariance with V right-hand sides) gives the comparison time and
    the difference of the two covariances."""
    import torch

    import paper_2308_01457_gb300 as F

    F.build.build()
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    W = WORKLOADS[args.workload]
    meshes, dirs = _meshes(W), _dirs(W)
    arith = F.ASM_FF if args.arith == "ff" else F.ASM_FP64

    def problem(tol):
        prob = _problem(F, W, meshes, dirs, F.MIXED, arith)
        prob.pseudo, prob.lowrank_tol = True, tol
        return prob

    def timed(prob, steps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        ev[0].record()
        for i in range(steps):
            out = prob.run()
            prob.release()
            ev[i + 1].record()
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[-1]) / steps, out

    prob = problem(W["tol"])
    for _ in range(args.warmup):
        prob.run()
        prob.release()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    launches0 = F.lib().fosb_kernel_launches()
    clocks = _clock_sampler(local) if rank == 0 else None
    ms, out = timed(prob, args.steps)
    if ws > 1:
        torch.distributed.barrier()
    clk = _clock_summary(clocks)
    launches = int(F.lib().fosb_kernel_launches() - launches0)
    ms = _max_over_ranks(ms, ws, "cuda")
    if rank != 0:
        return
    cov_lr, pcov_lr = out[1].cpu().numpy(), out[2].cpu().numpy()
    # the factorisation alone (it synchronises: host clock around the call)
    t0 = time.perf_counter()
    F.kernel_lowrank([prob.levels[l].mesh for l in sorted(prob.levels)], prob.kernel, prob.sigma, prob.ell, W["tol"],
                     device=prob.levels[W["L"]].Z.device)
    factor_ms = (time.perf_counter() - t0) * 1e3
    full = problem(None)
    full.run()
    full.release()
    ms_full, out_f = timed(full, 1)
    cov_f, pcov_f = out_f[1].cpu().numpy(), out_f[2].cpu().numpy()
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    L = W["L"]
    V = prob.levels[L].mesh.nv
    line = {"metric": METRIC, "value": round(ms / 1e3, 4), "unit": "s per FOSB step", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 2), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "mixed: float-float regular pairs, f64 singular pairs, 3xTF32 LU with FP64-class refinement, "
                     "f64 pivoted Cholesky", "data": "synthetic",
            "config": {"workload": args.workload, "N": prob.levels[L].mesh.n_edges, "V": V, "k": W["k"],
                       "n_dir": W["n_dir"], "sigma": W["sigma"], "ell": W["ell"], "tol": W["tol"],
                       "parallelism": f"replicas{ws}"},
            "rank": prob.rank, "trace_err_rel": prob.trace_err / (V * W["sigma"] ** 2),
            "factor_ms": round(factor_ms, 2),
            "full_path": {"s_per_step": round(ms_full / 1e3, 4), "rhs": V,
                          "rel_diff_cov": rel(cov_lr, cov_f), "rel_diff_pcov": rel(pcov_lr, pcov_f)},
            "speedup_vs_full_path": round(ms_full / ms, 3), "gpu_launches": launches, "clocks": clk}
    if not args.no_cpu_baseline:
        import oracle as O

        O.build()
        t = time.perf_counter()
        lev = {L: O.nominal_level(O.from_synth(meshes[0]), W["k"], W["d"], W["p"], dirs)}
        O.ct_farfield_covariance_lowrank(lev, L, L, W["kernel"], W["sigma"], W["ell"], W["tol"])
        O.ct_farfield_covariance_lowrank(lev, L, L, W["kernel"], W["sigma"], W["ell"], W["tol"], pseudo=True)
        dt = time.perf_counter() - t
        line["cpu_baseline"] = {"value": round(dt, 2), "unit": "s per FOSB step", "cores": len(os.sched_getaffinity(0)),
                                "kind": "oracle",
                                "sample": "the complete step: oracle assembly, LAPACK solve, maps and the low-rank "
                                          "covariance and pseudo-covariance (each with its own pivoted Cholesky)"}
    print(json.dumps(line), flush=True)


# algorithmic FP64 operations per point pair and wavenumber of the PMCHWT regular pairs: the
# EFIO's 27 (distance 8, phase 1, G 2, 8 real-weighted complex moments 16) and the MFIO's 24
# (its kernel exp(ikr)(ikr - 1)/r^3 from G: 10; its scalar and y-weighted moments: 14)
PMCHWT_OPS_PER_POINT_PAIR = 51.0


def run_pmchwt(args):
    """The dielectric workload: one step = fosb_assemble_pmchwt (both wavenumbers and the
    tested incident data), the complex64 LU of the 2N x 2N system (fosb_factor, MIXED), the
    refined solve and the far field at 1801 angles (fosb_farfield_pmchwt)."""
    import ctypes

    import torch

    import fosb_synth as S
    import paper_2308_01457_gb300 as F

    F.build.build()
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    W = WORKLOADS[args.workload]
    dev = f"cuda:{local}"
    sm = S.icosphere(W["level"])
    dirs = S.zplane_directions(W["n_dir"])
    inc = F.incidence([W["d"]], [W["p"]])
    upeaks = {kd: round(F.peak_microbench(kd), 2) for kd in ("fp32", "fp64", "tf32", "bf16")}
    arith = F.ASM_FF if args.arith == "ff" else F.ASM_FP64
    mesh = F.mesh_create(sm.verts, sm.tris, sm.vnormals)
    N = mesh.n_edges
    C128 = torch.complex128
    Z = torch.empty((2 * N, 2 * N), dtype=C128, device=dev)
    b = torch.empty((2 * N, 1), dtype=C128, device=dev)
    out = torch.empty((3 * W["n_dir"], 1), dtype=C128, device=dev)

    def step(m, prec, timers=None):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)] if timers is not None else None
        if ev:
            ev[0].record()
        F.assemble_pmchwt(m, W["k"], W["eps_r"], W["mu_r"], Z, inc=inc, b=b, arith=arith)
        if ev:
            ev[1].record()
        lu = F.factor(Z, prec=prec)
        if ev:
            ev[2].record()
        X, _, berr = F.solve(lu, b)
        if ev:
            ev[3].record()
        F.farfield_pmchwt(m, W["k"], dirs, X, out)
        if ev:
            ev[4].record()
            torch.cuda.synchronize()
            for i, name in enumerate(("assemble", "factor", "solve", "farfield")):
                timers.setdefault(name, []).append(ev[i].elapsed_time(ev[i + 1]))
        del lu
        return berr

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        step(mesh, F.MIXED)
    barrier()
    launches0 = F.lib().fosb_kernel_launches()
    clocks = _clock_sampler(local) if rank == 0 else None
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record()
    for i in range(args.steps):
        berr = step(mesh, F.MIXED)
        ev[i + 1].record()
    barrier()
    clk = _clock_summary(clocks)
    launches = int(F.lib().fosb_kernel_launches() - launches0)
    step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    ms = _max_over_ranks(ev[0].elapsed_time(ev[-1]) / args.steps, ws, "cuda")
    F_mixed = out.cpu().numpy()[:, 0].copy()
    # profiled pass after the timed region: phases and kernel families
    families = ["pmchwt_regular", "pmchwt_singular", "lu_update", "lu_update64", "lu_panel", "gemm_ff", "gemm_oz",
                "trsm_update", "oz_prep", "getrs"]
    for fam in families:
        F.lib().fosb_profile_read(fam.encode(), None, None, None)
    timers = {}
    F.lib().fosb_profile_enable(1)
    for _ in range(2):
        step(mesh, F.MIXED, timers)
    torch.cuda.synchronize()
    F.lib().fosb_profile_enable(0)
    fam_stats = {}
    for fam in families:
        ms_c, n_c, w_c = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double()
        F.lib().fosb_profile_read(fam.encode(), ctypes.byref(ms_c), ctypes.byref(n_c), ctypes.byref(w_c))
        fam_stats[fam] = {"ms_per_step": ms_c.value / 2, "launches_per_step": n_c.value / 2,
                          "work_per_step": w_c.value / 2}
    phase = {k: round(statistics.mean(v), 2) for k, v in timers.items()}
    peaks = _peaks()
    bf16 = peaks.get("bf16_tflops_sustained", 1700.0)
    tf32_peak = bf16 * TF32_PER_BF16
    model = {
        "pmchwt_regular": ("alu", PMCHWT_OPS_PER_POINT_PAIR, upeaks["fp32" if arith == F.ASM_FF else "fp64"],
                           "pmchwt_regular_ff_kernel (float-float)" if arith == F.ASM_FF
                           else "pmchwt_regular_kernel (FP64)",
                           f"{PMCHWT_OPS_PER_POINT_PAIR:.0f} algorithmic FP64-class ops per point pair and "
                           "wavenumber (work = point pairs of both launches); peak = the FP32 (float-float) or FP64 "
                           "FMA pipe measured by fosb_peak_microbench"),
        "lu_update": ("tensor", 1.0, tf32_peak, "cgemm_update_split_kernel (tcgen05 kind::tf32, 3xTF32 complex)",
                      "TF32 dense = measured bf16 sustained x 1.1/2.25; work = useful complex flops 8MNK"),
        "lu_panel": ("latency", 1.0, None, "tslu_gepp_kernel (tournament-pivoting panel)", "latency-bound"),
        "pmchwt_singular": ("alu", 1.0, None, "pmchwt_singular_kernel (FP64 Sauter-Schwab)",
                            "work = touching pairs per launch"),
    }
    dom = max((f for f in model if fam_stats[f]["ms_per_step"] > 0), key=lambda f: fam_stats[f]["ms_per_step"])
    bound, wsc, peak, kname, note = model[dom]
    st = fam_stats[dom]
    achieved = st["work_per_step"] * wsc / (st["ms_per_step"] * 1e-3) / 1e12
    roofline = {"bound": bound, "achieved": round(achieved, 4), "peak": round(peak, 3) if peak else None,
                "unit": "TFLOP/s", "frac": round(achieved / peak, 4) if peak else None, "traffic": None,
                "kernel": kname, "family": dom, "ms_per_step": round(st["ms_per_step"], 2),
                "launches_per_step": st["launches_per_step"], "peak_source": note}
    families_out = {f: {"ms_per_step": round(v["ms_per_step"], 2), "launches_per_step": v["launches_per_step"]}
                    for f, v in fam_stats.items() if v["ms_per_step"] > 0}
    if rank != 0:
        return
    e2e = None
    if not args.no_e2e:
        # the public API from host arrays: mesh upload, the step, the far field downloaded
        h2d = sm.verts.nbytes + sm.tris.nbytes + sm.vnormals.nbytes + inc.nbytes
        ts = []
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            m2 = F.mesh_create(sm.verts, sm.tris, sm.vnormals)
            step(m2, F.MIXED)
            Fh = out.cpu().numpy()
            ts.append(time.perf_counter() - t0)
            del m2
        e2e = {"value": round(statistics.median(ts), 4), "unit": "s per PMCHWT step", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(Fh.nbytes), "steps": 3, "stat": "median"}
    fp64 = None
    if not args.no_fp64:
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        step(mesh, F.FP64)
        e1.record()
        torch.cuda.synchronize()
        F64 = out.cpu().numpy()[:, 0]
        fp64 = {"s_per_step": round(e0.elapsed_time(e1) / 1e3, 3),
                "rel_diff_farfield_mixed_vs_fp64": float(np.linalg.norm(F_mixed - F64) / np.linalg.norm(F64)),
                "speedup_mixed_vs_fp64": round(e0.elapsed_time(e1) / ms, 2)}
    R = np.array([[0, 0, 1.0], [0, -1.0, 0], [1.0, 0, 0]])  # (e_x, e_y, e_z) -> (e_z, -e_y, e_x)
    import oracle.mie as mie

    Fm = (mie.farfield(W["k"], 1.0, dirs @ R, eps_r=W["eps_r"], mu_r=W["mu_r"]) @ R.T).reshape(-1)
    t_asm = phase.get("assemble", 0.0)
    line = {"metric": METRIC, "value": round(ms / 1e3, 4), "unit": "s per PMCHWT step", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 2), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None,
            "dtype": ("mixed: float-float (f32x2) regular pairs, f64 singular pairs" if arith == F.ASM_FF
                      else "mixed: f64 assembly") + ", 3xTF32 tensor-core LU (c64 factors) with FP64-class refinement",
            "data": "synthetic",
            "config": {"workload": args.workload, "triangles": sm.nt, "N": N, "unknowns": 2 * N, "k0": W["k"],
                       "eps_r": W["eps_r"], "mu_r": W["mu_r"], "n_dir": W["n_dir"], "assembly": args.arith,
                       "parallelism": f"replicas{ws}",
                       "l2": "inputs larger than L2 (Z is 3.8 GB)"},
            "median_step_ms": round(statistics.median(step_ms), 2),
            "entries_per_s": round(4.0 * N * N / (t_asm * 1e-3), 1) if t_asm > 0 else None,
            "phase_ms": phase, "families": families_out, "ir_backward_error": berr,
            "rel_err_farfield_vs_mie": float(np.linalg.norm(F_mixed - Fm) / np.linalg.norm(Fm)),
            "roofline": roofline, "peaks_microbench_tflops": upeaks, "gpu_launches": launches, "clocks": clk,
            "e2e": e2e, "fp64": fp64}
    if not args.no_cpu_baseline:
        import oracle as O

        O.build()
        lo = W["oracle_level"]
        om = O.from_synth(S.icosphere(lo))
        t0 = time.perf_counter()
        Zo = O.assemble_pmchwt(om, W["k"], W["eps_r"], W["mu_r"])
        bo = O.rhs_pmchwt(om, W["k"], [W["d"]], [W["p"]])
        t1 = time.perf_counter()
        xo = O.solve(Zo, bo)
        t2 = time.perf_counter()
        O.farfield_matrix_pmchwt(om, W["k"], dirs) @ xo
        t3 = time.perf_counter()
        T_ratio = sm.nt / om.nt
        model_s = (t1 - t0) * T_ratio**2 + (t2 - t1) * T_ratio**3 + (t3 - t2) * T_ratio
        line["cpu_baseline"] = {
            "value": round(model_s, 2), "unit": "s per PMCHWT step", "cores": len(os.sched_getaffinity(0)),
            "kind": "oracle",
            "sample": f"the complete oracle step on the {om.nt}-triangle sphere (2N = {2 * om.n_edges}) measured: "
                      f"assembly {t1 - t0:.2f} s, LAPACK solve {t2 - t1:.2f} s, far field {t3 - t2:.2f} s; scaled "
                      f"to {sm.nt} triangles by the exact operation counts (pairs x{T_ratio**2:.0f}, LU "
                      f"x{T_ratio**3:.0f}, far field x{T_ratio:.0f})",
            "measured_level_s": round(t3 - t0, 2)}
    print(json.dumps(line), flush=True)


def run_dect(args):
    """The dielectric CT workload: one step = every level's PMCHWT solve and far field
    (DielectricCT.farfield) and the CT second moment of the rank-one right-hand side."""
    import torch

    import fosb_synth as S
    import paper_2308_01457_gb300 as F
    from paper_2308_01457_gb300.dielectric import DielectricCT

    F.build.build()
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    W = WORKLOADS[args.workload]
    sms = {l: S.icosphere(l + 1) for l in W["levels"]}
    dirs = S.zplane_directions(W["n_dir"])
    arith = F.ASM_FF if args.arith == "ff" else F.ASM_FP64
    prob = DielectricCT(sms, W["k"], W["eps_r"], W["mu_r"], [W["d"]], [W["p"]], dirs, W["L0"], W["L"], arith=arith,
                        device=f"cuda:{local}").setup()
    for _ in range(args.warmup):
        prob.run()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    launches0 = F.lib().fosb_kernel_launches()
    clocks = _clock_sampler(local) if rank == 0 else None
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record()
    for i in range(args.steps):
        FL, M = prob.run()
        ev[i + 1].record()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = _clock_summary(clocks)
    launches = int(F.lib().fosb_kernel_launches() - launches0)
    ms = _max_over_ranks(ev[0].elapsed_time(ev[-1]) / args.steps, ws, "cuda")
    if rank != 0:
        return
    import oracle.mie as mie

    R = np.array([[0, 0, 1.0], [0, -1.0, 0], [1.0, 0, 0]])  # (e_x, e_y, e_z) -> (e_z, -e_y, e_x)
    Fz = (mie.farfield(W["k"], 1.0, dirs @ R, eps_r=W["eps_r"], mu_r=W["mu_r"]) @ R.T)[:, 2]
    zz = torch.arange(2, 3 * W["n_dir"], 3, device=M.device)
    Mz = M[zz][:, zz].cpu().numpy()
    Mex = np.outer(Fz, Fz.conj())
    FLz = FL.cpu().numpy()[2::3]
    ex = None
    if not args.no_e2e:
        # the public API from host arrays: every level's mesh uploaded, the step, M downloaded
        h2d = sum(sm.verts.nbytes + sm.tris.nbytes + sm.vnormals.nbytes for sm in sms.values())
        ts = []
        for _ in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            p2 = DielectricCT(sms, W["k"], W["eps_r"], W["mu_r"], [W["d"]], [W["p"]], dirs, W["L0"], W["L"],
                              arith=arith, device=f"cuda:{local}").setup()
            _, M2 = p2.run()
            Mh = M2.cpu().numpy()
            ts.append(time.perf_counter() - t0)
            del p2, M2
        ex = {"value": round(statistics.median(ts), 4), "unit": "s per CT step", "h2d_bytes_per_step": int(h2d),
              "d2h_bytes_per_step": int(Mh.nbytes), "steps": 2, "stat": "median"}
    line = {"metric": METRIC, "value": round(ms / 1e3, 4), "unit": "s per CT step", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 2), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "mixed: float-float (f32x2) regular pairs, f64 singular pairs, 3xTF32 tensor-core LU with "
                     "FP64-class refinement", "data": "synthetic",
            "config": {"workload": args.workload, "levels": W["levels"],
                       "unknowns": [2 * prob.meshes[l].n_edges for l in W["levels"]], "k0": W["k"],
                       "eps_r": W["eps_r"], "n_dir": W["n_dir"], "ct": [W["L0"], W["L"]], "assembly": args.arith,
                       "parallelism": f"replicas{ws}"},
            "rel_err_ct_second_moment_zz_vs_mie": float(np.linalg.norm(Mz - Mex) / np.linalg.norm(Mex)),
            "rel_err_full_tensor_zz_vs_mie": float(np.linalg.norm(np.outer(FLz, FLz.conj()) - Mex) /
                                                   np.linalg.norm(Mex)),
            "ir_backward_error_max": max(prob.berr.values()), "gpu_launches": launches, "clocks": clk, "e2e": ex}
    if not args.no_cpu_baseline:
        import oracle as O

        O.build()
        lv = W["levels"]
        t0 = time.perf_counter()
        O.dielectric_ct_second_moment({l: O.from_synth(sms[l]) for l in lv[:-1]}, W["k"], W["eps_r"], W["mu_r"],
                                      [W["d"]], [W["p"]], dirs, W["L0"], W["L"] - 1)
        t_meas = time.perf_counter() - t0
        om = O.from_synth(sms[lv[-2]])
        t1 = time.perf_counter()
        Zo = O.assemble_pmchwt(om, W["k"], W["eps_r"], W["mu_r"])
        bo = O.rhs_pmchwt(om, W["k"], [W["d"]], [W["p"]])
        t2 = time.perf_counter()
        xo = O.solve(Zo, bo)
        t3 = time.perf_counter()
        O.farfield_matrix_pmchwt(om, W["k"], dirs) @ xo
        t4 = time.perf_counter()
        finest = (t2 - t1) * 16 + (t3 - t2) * 64 + (t4 - t3) * 4
        line["cpu_baseline"] = {
            "value": round(t_meas + finest, 2), "unit": "s per CT step", "cores": len(os.sched_getaffinity(0)),
            "kind": "oracle",
            "sample": f"the oracle's CT step over levels {lv[0]}..{lv[-2]} measured end to end ({t_meas:.1f} s), plus "
                      f"level {lv[-1]} from level {lv[-2]}'s measured phases scaled by the exact operation counts "
                      f"(pairs x16, LU x64, far field x4: {finest:.1f} s)"}
    print(json.dumps(line), flush=True)


def cpu_baseline_batched(W):
    """The FP64 CPU oracle, as it stands, on the batched workload: assembly, plane-wave
    right-hand sides and the LAPACK solve of all 16 directions, measured for every
    scatterer with N = 480 and N = 1920 and for the first with N = 7680; each further
    N = 7680 scatterer is counted at that measured time (the oracle's cost depends on N,
    not on k or the semi-axes)."""
    import oracle as O

    O.build()
    table, meshes, ks, d, p = _batched_inputs(W)
    t_begin = time.perf_counter()
    measured, large = 0.0, None
    n_large = 0
    for sm, k in zip(meshes, ks):
        om = O.from_synth(sm)
        if om.n_edges >= 7680:
            n_large += 1
            if large is not None:
                continue
        t = time.perf_counter()
        O.solve(O.assemble_z(om, k), O.rhs_planewave(om, k, d, p))
        dt = time.perf_counter() - t
        if om.n_edges >= 7680:
            large = dt
        else:
            measured += dt
    value = measured + (large or 0.0) * n_large
    return {"value": round(value, 2), "unit": "s per batch step", "cores": len(os.sched_getaffinity(0)),
            "kind": "oracle",
            "sample": f"oracle assembly + RHS + LAPACK solve (16 directions) measured for the {64 - n_large} "
                      f"scatterers with N <= 1920 and one of the {n_large} with N = 7680 ({large:.1f} s), the others "
                      f"counted at that time; sample {time.perf_counter() - t_begin:.1f} s"}


def run_fp64_compare(W, meshes, dirs, out_mixed, ms_mixed):
    """One step of the same workload in plain FP64 (FP64 assembly, complex128 LU on the
    FP64 tensor path, no refinement), outside the timed region: its time, assembly rate
    and the relative difference of the mixed step's mean far field and CT covariance."""
    import torch

    import paper_2308_01457_gb300 as F

    prob = _problem(F, W, meshes, dirs, F.FP64, F.ASM_FP64)
    timers = {}
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    Fm, cov = prob.run(timers)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    L = W["L"]
    NL = prob.levels[L].mesh.n_edges
    t_asm = sum(x.elapsed_time(y) for x, y in timers[f"assemble_l{L}"])

    def rel(x, y):
        return float(torch.linalg.norm(x - y) / torch.linalg.norm(y))

    res = {"s_per_step": round(ms / 1e3, 4), "mixed_speedup": round(ms / ms_mixed, 2),
           "efie_entries_per_s": round(NL * NL / (t_asm * 1e-3), 1),
           "phase_ms": {"assemble_finest": round(t_asm, 2),
                        "factor_finest": round(sum(x.elapsed_time(y) for x, y in timers[f"factor_l{L}"]), 2),
                        "covariance_ct": round(sum(x.elapsed_time(y) for x, y in timers["covariance_ct"]), 2)},
           "rel_diff_mean_farfield": rel(out_mixed[0], Fm), "rel_diff_ct_covariance": rel(out_mixed[1], cov),
           "note": "one step, same workload, FP64 assembly and complex128 LU (DMMA), timed with CUDA events"}
    prob.release()
    del prob
    torch.cuda.empty_cache()
    return res


def run_e2e(args, W, meshes, dirs, arith):
    """Same step through the public API from pinned host arrays: mesh upload (A1),
    the whole path, and the download of the mean far field and the CT covariance."""
    import torch

    import paper_2308_01457_gb300 as F

    pinned = []
    h2d = 0
    for sm in meshes:
        v = torch.from_numpy(np.ascontiguousarray(sm.verts)).pin_memory()
        t = torch.from_numpy(np.ascontiguousarray(sm.tris)).pin_memory()
        n = torch.from_numpy(np.ascontiguousarray(sm.vnormals)).pin_memory()
        pinned.append(type(sm)(v.numpy(), t.numpy(), n.numpy(), sm.name))
        h2d += v.numel() * 8 + t.numel() * 4 + n.numel() * 8
    nd3 = 3 * W["n_dir"]
    F_h = torch.empty((nd3, 1), dtype=torch.complex128).pin_memory()
    C_h = torch.empty((nd3, nd3), dtype=torch.complex128).pin_memory()
    d2h = (F_h.numel() + C_h.numel()) * 16
    steps = max(1, min(args.steps, 3))
    times = []
    for i in range(steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        prob = _problem(F, W, pinned, dirs, F.MIXED, arith)
        Fm, cov = prob.run()
        F_h.copy_(Fm, non_blocking=True)
        C_h.copy_(cov, non_blocking=True)
        torch.cuda.synchronize()
        if i > 0:  # first pass warms the allocator
            times.append(time.perf_counter() - t0)
        prob.release()
        del prob
    return {"value": round(statistics.median(times), 4), "unit": "s per FOSB step", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "steps": len(times)}


# ----------------------------------------------------------------------------- CPU oracle
def _sizes(W, l):
    """(N, V) of level l: icosphere level l + 1 (sphere) or the torus grid 10*2^(l-1) x 4*2^(l-1)."""
    if W["mesh"] == "torus":
        return 120 * 4 ** (l - 1), 40 * 4 ** (l - 1)
    return 120 * 4**l, 40 * 4**l + 2


def _ct_blocks(L0, L):
    """The blocks the combination technique solves (l1 >= l2 on Lambda_+ and Lambda_-)."""
    plus = [(a, L + L0 - a) for a in range(L0, L + 1) if L0 <= L + L0 - a <= L]
    minus = [(a, L + L0 - 1 - a) for a in range(L0, L + 1) if L0 <= L + L0 - 1 - a <= L]
    return [b for b in plus + minus if b[0] >= b[1]]


def oracle_step(W, L):
    """One complete FOSB step of the FP64 CPU oracle, as it stands, on levels L0..L of the
    workload: per level the steps of oracle.nominal_level (assembly, plane-wave RHS, LAPACK
    solve, far-field matrix, SD right-hand side), each timed, then the CT far-field
    covariance over L0..L (oracle.ct_farfield_covariance).  Returns (F_mean, cov, times)."""
    import oracle as O
    import fosb_synth as S

    O.build()
    xh = _dirs(W)
    meshes = (S.torus_hierarchy(list(range(W["L0"], L + 1))) if W["mesh"] == "torus"
              else [S.icosphere(l + 1) for l in range(W["L0"], L + 1)])
    times = {"levels": {}, "ct": 0.0}
    t_all = time.perf_counter()
    lev = {}
    for l, sm in zip(range(W["L0"], L + 1), meshes):
        m = O.from_synth(sm)
        tl = {}
        t = time.perf_counter()
        Z = O.assemble_z(m, W["k"])
        tl["asm"] = time.perf_counter() - t
        t = time.perf_counter()
        b = O.rhs_planewave(m, W["k"], W["d"], W["p"])[:, 0]
        u = O.solve(Z, b)
        tl["solve"] = time.perf_counter() - t
        t = time.perf_counter()
        A = O.farfield_matrix(m, W["k"], xh)
        B = O.sd_rhs(m, W["k"], u)
        tl["maps"] = time.perf_counter() - t
        lev[l] = O.Level(m, Z, u, A, B)
        times["levels"][l] = tl
    t = time.perf_counter()
    cov = O.ct_farfield_covariance(lev, W["L0"], L, W["kernel"], W["sigma"], W["ell"])
    times["ct"] = time.perf_counter() - t
    times["total"] = time.perf_counter() - t_all
    return lev[L].A @ lev[L].u, cov, times


def _lu_flops(n):
    return (8.0 / 3.0) * float(n) ** 3


def lapack_rate(n, seed=0):
    """Flop rate of the oracle's dense solve (numpy.linalg.solve: LAPACK LU and one right-
    hand side) on a seeded random complex n x n system, counted as 8/3 n^3."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    b = rng.standard_normal(n) + 0j
    t = time.perf_counter()
    np.linalg.solve(A, b)
    return _lu_flops(n) / (time.perf_counter() - t)


def _ct_flops(W, L):
    """Flops of the oracle's CT covariance over L0..L: per block the two LAPACK solves
    (a factorisation of each Z and the triangular solves), C = B1 K B2^H with dense B, and
    the far-field product A1 Sigma A2^H."""
    nd3 = 3 * W["n_dir"]
    f = 0.0
    for l1, l2 in _ct_blocks(W["L0"], L):
        (n1, v1), (n2, v2) = _sizes(W, l1), _sizes(W, l2)
        f += _lu_flops(n1) + _lu_flops(n2) + 8.0 * (n1 * n1 * n2 + n2 * n2 * n1)
        f += 8.0 * (n1 * v1 * v2 + n1 * v2 * n2) + 8.0 * (nd3 * n1 * n2 + nd3 * nd3 * n2)
    return f


def oracle_model(W, times, L, rate):
    """Predicted oracle time of the step over L0..L from a measured step over L0..L-1:
    the measured levels as measured; level L's assembly scaled by N^2 (point pairs) and its
    far-field and SD maps by N from level L-1; level L's LAPACK solve and the whole CT
    covariance over L0..L by their flop counts at `rate` (a LAPACK solve measured at half
    of level L's N)."""
    lv = times["levels"]
    total = sum(sum(t.values()) for t in lv.values())
    r = _sizes(W, L)[0] / _sizes(W, L - 1)[0]
    total += lv[L - 1]["asm"] * r * r + lv[L - 1]["maps"] * r + _lu_flops(_sizes(W, L)[0]) / rate
    return total + _ct_flops(W, L) / rate


def cpu_baseline(W, with_outputs=False):
    """The FP64 CPU oracle, as it stands, on the machine's host cores: a complete oracle step
    one level below the workload's finest (every level's assembly, solve and maps and the
    full CT covariance, measured end to end), extended to the workload by oracle_model
    with a LAPACK rate measured at half the finest N.  The model's error is measured one
    level down: the step two levels below, with a LAPACK rate at half of the next N,
    predicts the measured step."""
    cores = len(os.sched_getaffinity(0))
    L = W["L"]
    _, _, t_cal = oracle_step(W, L - 2)
    F, cov, t_meas = oracle_step(W, L - 1)
    r_cal = lapack_rate(_sizes(W, L - 1)[0] // 2)
    rate = lapack_rate(_sizes(W, L)[0] // 2)
    pred_meas = oracle_model(W, t_cal, L - 1, r_cal)
    value = oracle_model(W, t_meas, L, rate)
    n_f = _sizes(W, L - 1)[0]
    res = {"value": round(value, 2), "unit": "s per FOSB step", "cores": cores, "kind": "oracle",
           "sample": f"complete oracle step over levels {W['L0']}..{L - 1} (N <= {n_f}) measured end to end in "
                     f"{t_meas['total']:.1f} s; modelled: level {L} (assembly x N^2, maps x N) and the LAPACK "
                     f"solves of level {L} and of the CT covariance (flop count at {rate / 1e9:.1f} GFLOP/s, "
                     f"a LAPACK solve measured at N = {_sizes(W, L)[0] // 2})",
           "measured_step": {"levels": [W["L0"], L - 1], "s": round(t_meas["total"], 2),
                             "ct_covariance_s": round(t_meas["ct"], 2),
                             "assembly_finest_s": round(t_meas["levels"][L - 1]["asm"], 2),
                             "assembly_entries_per_s": round(n_f * n_f / t_meas["levels"][L - 1]["asm"], 1)},
           "model_error": {"predicted_s": round(pred_meas, 2), "measured_s": round(t_meas["total"], 2),
                           "rel": round(pred_meas / t_meas["total"] - 1.0, 3),
                           "note": f"the model on the step over {W['L0']}..{L - 2} with a LAPACK rate at "
                                   f"N = {_sizes(W, L - 1)[0] // 2}, against the measured step"}}
    return (res, F, cov) if with_outputs else res


def run_reference(args):
    """The reference arm: no upstream implementation exists (the paper's Bempp scripts are
    not provided), so it is the FP64 CPU oracle.  Each timed step measures the complete
    oracle step one level below the workload's finest and extends it to the workload with
    oracle_model (the LAPACK rate at half the finest N is measured once, before the steps);
    warm-up steps run the step two levels below."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    W = WORKLOADS[args.workload]
    L = W["L"]
    t_all = time.perf_counter()
    for _ in range(args.warmup):
        _, _, cal = oracle_step(W, L - 2)
    rate = lapack_rate(_sizes(W, L)[0] // 2)
    vals, meas = [], []
    for _ in range(args.steps):
        _, _, t = oracle_step(W, L - 1)
        vals.append(oracle_model(W, t, L, rate))
        meas.append(t["total"])
    v = round(statistics.median(vals), 2)
    pred = oracle_model(W, cal, L - 1, lapack_rate(_sizes(W, L - 1)[0] // 2))
    wall = time.perf_counter() - t_all
    cb = {"value": v, "unit": "s per FOSB step", "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
          "sample": f"each step: the complete oracle step over levels {W['L0']}..{L - 1} measured end to end "
                    f"(median {statistics.median(meas):.1f} s), extended to level {L} by the model at "
                    f"{rate / 1e9:.1f} GFLOP/s (LAPACK solve measured at N = {_sizes(W, L)[0] // 2})",
          "model_error": {"predicted_s": round(pred, 2), "measured_s": round(statistics.median(meas), 2),
                          "rel": round(pred / statistics.median(meas) - 1.0, 3)}}
    line = {"metric": METRIC, "value": v, "unit": "s per FOSB step", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(v * 1e3, 1), "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "levels": W["levels"], "k": W["k"], "n_dir": W["n_dir"],
                       "ct": [W["L0"], W["L"]], "parallelism": "host cores"},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "s per FOSB step", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "measured_wall_s": round(wall, 1)}
    print(json.dumps(line), flush=True)


def run_reference_batched(args):
    """Reference arm of the batched workload: the FP64 CPU oracle (cpu_baseline_batched) per
    step; rank 0 only."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    W = WORKLOADS[args.workload]
    for _ in range(args.warmup):
        cpu_baseline_batched(W)
    vals = []
    for _ in range(args.steps):
        r = cpu_baseline_batched(W)
        vals.append(r["value"])
    v = round(statistics.median(vals), 2)
    r["value"] = v
    print(json.dumps({"metric": METRIC, "value": v, "unit": "s per batch step", "n_gpus": ws, "steps": args.steps,
                      "warmup": args.warmup, "ms_per_step": round(v * 1e3, 1), "higher_is_better": False,
                      "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                      "impl": "reference", "config": {"workload": args.workload, "parallelism": "host cores"},
                      "cpu_baseline": r,
                      "e2e": {"value": v, "unit": "s per batch step", "h2d_bytes_per_step": 0,
                              "d2h_bytes_per_step": 0}}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fosb", choices=["fosb", "reference"])
    ap.add_argument("--workload", default="sphere-ka4-ct-L4", choices=sorted(WORKLOADS))
    ap.add_argument("--arith", default="ff", choices=["fp64", "ff"],
                    help="regular-pair assembly arithmetic: float-float on the FP32 pipe (default) or FP64")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison step")
    ap.add_argument("--workers", type=int, default=4, help="host worker threads of the batched solve")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)  # at least three untimed warm-up steps
    kind = WORKLOADS[args.workload].get("kind")
    if args.impl == "reference":
        if kind in ("mc", "lowrank", "pmchwt", "dect"):
            print(json.dumps({"impl": "reference", "unavailable": "the reference arm times the default workload; "
                              "this workload reports its oracle baseline in its own line"}))
        else:
            run_reference_batched(args) if kind == "batched" else run_reference(args)
    elif kind == "batched":
        run_batched(args)
    elif kind == "mc":
        run_mc(args)
    elif kind == "lowrank":
        run_lowrank(args)
    elif kind == "pmchwt":
        run_pmchwt(args)
    elif kind == "dect":
        run_dect(args)
    else:
        run_fosb(args)


if __name__ == "__main__":
    main()
