"""Benchmark: linked rays/s of the ToF forward + adjoint step on the breast
workload (1024^2 grid at 0.2 mm, 512-element ring at 95 mm, 261,632 pairs,
RK4 step 0.02 mm, linking tolerance 1e-4 mm), FP32-compensated (headline)
next to the plain FP64 GPU form, with the roofline of the dominant kernels
against rates measured on the same GPU at start-up, and the FP64 CPU oracle
timed on the host (same algorithm, 1 thread and all cores) as a baseline.

One step = rt_link from a cold start (a fan of 768 rays per transducer
predicts every pair's first angle and bracket; travel time fused) +
rt_tof_adjoint of the L2 misfit 0.5*||T - T_meas||^2, on inputs already
resident in HBM. L2 is flushed (256 MB write) between timed steps. The line
also carries the batched workload (32 uneven instances, one persistent launch
replayed from a CUDA graph, FP32-compensated and FP64) and the ray-Born step
(fan maps + Born apply + adjoint on the tensor cores) as sub-objects.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) the one breast problem is split over the ranks by
emitter (longest chords first on every rank); each rank links and
back-projects its pairs and one NCCL all-reduce of the grid gradient, timed
inside the step, completes it (strong scaling); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "linked rays/s (ToF fwd+adjoint, 512-ring, 1024² grid) FP32 vs FP64 GPU; % roofline"
UNIT = "linked rays/s"
# FLOPs of one RK4 step of the method as written, FMA = 2, div/sqrt = 1: per
# stage sample the bilinear weights (6), the interpolation of c, dc/dx, dc/dy
# (21) and the ray right-hand side (10), i.e. 37 x 4 = 148; the stage state
# updates 24; the final RK4 combination 28; renormalisation 6; the trapezoid
# slowness sample and sum 9; the ring test 4.
FLOP_PER_STEP = 219
# The naive march gathers the 2 x 2 stencil of (c, dc/dx, dc/dy, s) as four
# float4 per sample, four samples per RK4 step: the L2-gather roofline's bytes.
GATHER_BYTES_PER_STEP = 256
# Cold-start fan of the breast workload: 1.5 rays per transducer of the 512-ring.
# A denser fan costs more fan rays (one balanced launch) but leaves fewer
# linking traces, and the multi-trace pairs are what drags out the persistent
# link kernel's drain: over four phantom seeds, link times averaged 108 ms at
# 256 rays, 97 ms at 384, 99 at 512, 98 at 640, 94 at 768 and 102 at 1024.
BREAST_FAN = 768
# The fan only predicts first angles and brackets, so it is traced at h/2 (5x
# the march step): on a 32,704-pair oracle sample it links the same rays
# (travel times within 2.9e-10) with 1.1462 traces per pair against 1.1444.
FAN_DS = 0.1
# RK4 step with the bicubic sampler: per stage the bicubic value and both
# derivatives by Horner (63) and the right-hand side (10), x 4 = 292; stage
# updates 24; combination 28; renormalisation 6; slowness bicubic and Kahan
# sum 33; ring test 4.
FLOP_PER_BSPLINE_STEP = 387
# TF32 tensor rate relative to BF16 (nominal dense: 1.1 / 2.25 PFLOP/s), applied
# to the measured BF16 rate.
TF32_PER_BF16 = 1.1 / 2.25


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-legs", action="store_true", help="skip the batch and ray-Born sub-objects")
    ap.add_argument("--traffic-json", default=os.path.join(ROOT, "profiles", "link_traffic.json"))
    ap.add_argument("--profile", type=int, default=0, metavar="N_EMIT",
                    help="case for ncu captures: twice rt_link + rt_tof_adjoint (fp32c) over the pairs of "
                         "the first N_EMIT emitters of the workload, then exit; with --workload batch, twice "
                         "rt_batch_run over its first N_EMIT instances; with --workload born, the maps of the "
                         "first N_EMIT transducers, then the Born apply and adjoint")
    ap.add_argument("--precision", default="fp32c", choices=["fp32c", "fp64"],
                    help="precision of the --profile case")
    ap.add_argument("--workload", default="breast", choices=["breast", "batch", "born", "small", "fisheye"],
                    help="breast: the headline single problem; batch: 32 uneven instances in one persistent "
                         "launch replayed from a CUDA graph; born: ray-Born maps + apply + adjoint "
                         "(1024^2, 512-ring, 8 frequencies); small: 128^2 / 64-ring; fisheye: the Maxwell "
                         "fish-eye lens 512^2 / 256-ring")
    return ap.parse_args()


def measured_peaks() -> dict:
    """FP32/FP64 FMA rates and L2 gather/read bandwidth of this GPU, measured
    now by the library's microbenchmarks (paper_2511_18511_gb300.peaks), and
    the measured HBM and BF16 rates (MEASURED_PEAKS.json) when present."""
    from paper_2511_18511_gb300 import peaks
    p = peaks.measure()
    try:
        drv = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        p["hbm_gbs"] = float(drv["hbm_gbs"])
        p["bf16_tflops"] = float(drv["bf16_tflops"])
        p["bf16_tflops_sustained"] = float(drv.get("bf16_tflops_sustained", drv["bf16_tflops"]))
    except (OSError, KeyError, ValueError):
        p["bf16_tflops"] = p["bf16_tflops_sustained"] = 1900.0   # the recipe's fallback
        p["hbm_gbs"] = 6800.0
        p["fallback"] = "MEASURED_PEAKS.json absent: HBM and BF16 are the recipe's fallback figures"
    p["tf32_tflops"] = p["bf16_tflops"] * TF32_PER_BF16   # burst: the contractions run 24-48 ms each
    return p


def batch_leg(args, peaks, steps: int = 3, warmup: int = 3, fp64_every: int = 4) -> dict:
    """32 seeded Gaussian-inclusion instances (grids 256^2..1024^2, rings
    64..512): link + adjoint of every pair in one persistent launch, captured
    in a CUDA graph and replayed; kernel variant chosen by the autotuner. The
    plain FP64 form runs on every fp64_every-th instance next to the
    FP32-compensated form on the same instances (the FP64 form is ~25x slower)."""
    import torch
    import paper_2511_18511_gb300 as rt
    from paper_2511_18511_gb300 import autotune
    from paper_2511_18511_gb300 import phantoms as P
    ws = P.cfg_batch()
    ds = ws[0].ds
    insts = [rt.BatchInstance.create(rt.Problem.create(w.grid, w.c, w.tx, w.ring_radius)) for w in ws]
    # "measured" times: the same media 0.5 % faster (set-up, not timed)
    for b in insts:
        c0 = b.prob.c.clone()
        b.prob.c.mul_(1.005)
        rt.rt_batch_run([b], ds)
        b.prob.c.copy_(c0)
        b.tof_ref = b.tof.clone()
        b.g_c = torch.empty_like(b.prob.c)
    total = sum(b.prob.n_pairs for b in insts)
    fan_ds = 0.5 * ws[0].grid.h           # every instance has h = 0.2 mm: the fan traced at 0.1 mm
    best, times = autotune.tune_batch(insts, ds, reps=1, fan_ds=fan_ds)
    kw = dict(block_threads=best[0], step_unroll=best[1], blocks_per_sm=best[2], fan_ds=fan_ds)
    rt.rt_batch_run(insts, ds, **kw)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            rt.rt_batch_run(insts, ds, reset_angles=False, stream=s, **kw)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def reset(group):
        for b in group:
            b.theta.fill_(float("nan"))

    ev = []
    with torch.cuda.stream(s):        # replay, resets and events all on stream s
        for _ in range(warmup):
            reset(insts)
            graph.replay()
        torch.cuda.synchronize()
        for _ in range(steps):
            reset(insts)
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            graph.replay()
            b.record(s)
            ev.append((a, b))
        torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    ok, counts = rt.rt_status_counts()
    achieved = counts[7] * FLOP_PER_STEP / (ms / 1e3) / 1e12

    # FP64 against FP32-compensated on the same sub-batch (plain calls, no graph)
    sub = insts[::fp64_every]
    n_sub = sum(b.prob.n_pairs for b in sub)

    def timed_sub(precision, blk):
        rt.rt_batch_run(sub, ds, precision=precision, **blk)       # sizes the workspace, warms up
        torch.cuda.synchronize()
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        rt.rt_batch_run(sub, ds, precision=precision, **blk)
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    ms_sub32 = timed_sub("fp32c", kw)
    ms_sub64 = timed_sub("fp64", dict(block_threads=128, step_unroll=16, blocks_per_sm=1, fan_ds=fan_ds))
    fp32 = peaks["fp32_tflops"]
    return {"metric": "linked rays/s (batched link+adjoint, 32 uneven instances, one persistent launch, CUDA graph)",
            "value": total / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": steps, "warmup": warmup,
            "config": {"workload": "batch32_uneven", "instances": len(insts), "pairs": total, "ds_mm": ds,
                       "grids": sorted({int(b.prob.grid.nx) for b in insts}),
                       "rings": sorted({b.prob.n_tx for b in insts}), "fan_rays": rt.DEFAULT_FAN, "fan_ds_mm": fan_ds,
                       "autotuned": {"rays_per_block": best[0], "step_unroll": best[1], "blocks_per_sm": best[2]},
                       "autotune_ms": {",".join(map(str, k)): round(v, 2) for k, v in times.items()},
                       "l2": "flushed between timed replays (256 MB write)"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32, "unit": "TFLOP/s",
                         "frac": achieved / fp32,
                         "traffic": (_traffic(os.path.join(ROOT, "profiles", "batch_traffic.json"), BATCH_HASH_FILES)
                                     if tuple(best) == BATCH_PROFILE_VARIANT else None),
                         "kernel": "graph replay (pack + fan + k_batch + finish)", "flop_per_rk4_step": FLOP_PER_STEP,
                         "rk4_steps_per_launch": counts[7], "peak_basis": "measured FP32 FMA rate (rt_peak_fma)"},
            "link": {"all_linked": ok, "status_counts": counts[:7]},
            "fp32c_vs_fp64": {"instances": len(sub), "pairs": n_sub,
                              "fp32c": {"value": n_sub / (ms_sub32 / 1e3), "ms": ms_sub32},
                              "fp64": {"value": n_sub / (ms_sub64 / 1e3), "ms": ms_sub64},
                              "speedup_fp32c_over_fp64": ms_sub64 / ms_sub32},
            "gpu_launches_per_step": 3 * len(insts) + 2}


def run_batch(args):
    """The batched workload as its own JSON line (--workload batch)."""
    import torch
    torch.cuda.set_device(0)
    peaks = measured_peaks()
    clocks = Clocks(0)
    clocks.start()
    leg = batch_leg(args, peaks, steps=args.steps, warmup=args.warmup)
    clk = clocks.stop()
    line = {k: leg[k] for k in ("metric", "value", "unit", "ms_per_step", "config", "roofline", "link",
                                "fp32c_vs_fp64")}
    line.update({"n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
                 "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                 "gpu_launches": args.steps * leg["gpu_launches_per_step"], "clocks": clk, "peaks": peaks})
    print(json.dumps(line), flush=True)


# FLOPs of one RK4 step of the fan-map kernel, as the kernel is written (FMA =
# 2, rcp/sqrt = 1): four samples of the six marched fields in coefficient form
# (144); stage positions 12; ray and paraxial right-hand sides (92); stage
# updates of (d, Q, P) 24; final combination of Q, P and the direction 22;
# compensated position increments and two-sum updates 30; direction
# renormalisation with its double-float split 35; slowness sample and Kahan
# time 12; the 3 x 3 foot test and the candidates that pass (about 0.3 per
# step) 32.
FLOP_PER_BORN_STEP = 403


def _born_cpu_baseline(w, n_fans: int, n_pairs: int, n_nodes: int):
    """The FP64 oracle on bounded samples of the ray-Born step, each part
    extrapolated linearly to the full step: n_fans fans (maps), n_pairs
    emitter-receiver pairs x all frequencies (apply), n_nodes nodes
    (adjoint)."""
    import oracle
    from paper_2511_18511_gb300 import phantoms as P
    oracle.build()
    cores = oracle.num_threads()
    sel = np.linspace(0, w.n_tx - 1, n_fans).astype(int)
    t0 = time.perf_counter()
    T, A = oracle.fan_maps(w.grid, w.c, w.tx[sel], w.ring_radius, w.ds, w.fan_rays)
    t_maps = (time.perf_counter() - t0) * w.n_tx / n_fans
    pairs = np.array([(a, b) for a in range(n_fans) for b in range(n_fans) if a != b][:n_pairs], np.int32)
    t0 = time.perf_counter()
    oracle.born_apply(w.grid, w.ring_radius, T, A, w.f_mhz, w.dc, pairs=pairs)
    t_apply = (time.perf_counter() - t0) * (w.n_tx * (w.n_tx - 1)) / len(pairs)
    # adjoint cost per node is that of all n_tx^2 pairs; time it on a sub-grid
    # of n_nodes nodes around the centre with the full ring of maps replaced by
    # the sampled fans repeated (cost depends on n_tx only)
    gs = P.Grid(int(np.sqrt(n_nodes)), int(np.sqrt(n_nodes)), w.grid.h)
    rng = P.SplitMix64(7)
    j0, i0 = (w.grid.ny - gs.ny) // 2, (w.grid.nx - gs.nx) // 2
    Ts = np.tile(T[:1, j0:j0 + gs.ny, i0:i0 + gs.nx], (w.n_tx, 1, 1))
    As = np.tile(A[:1, j0:j0 + gs.ny, i0:i0 + gs.nx], (w.n_tx, 1, 1))
    n = len(w.f_mhz) * w.n_tx * w.n_tx
    d = (rng.normal(n) + 1j * rng.normal(n)).reshape(len(w.f_mhz), w.n_tx, w.n_tx)
    t0 = time.perf_counter()
    oracle.born_adjoint(gs, 1e9, Ts, As, w.f_mhz, d)
    n_in = int(np.sum(np.hypot(*w.grid.node_xy()) < w.ring_radius))
    t_adj = (time.perf_counter() - t0) * n_in / (gs.nx * gs.ny)
    total = t_maps + t_apply + t_adj
    data = len(w.f_mhz) * w.n_tx * (w.n_tx - 1)
    return {"value": data / total, "unit": "Born data/s", "cores": cores, "kind": "oracle",
            "sample": f"{n_fans} fan maps ({w.fan_rays} rays each, two passes), {len(pairs)} pairs x "
                      f"{len(w.f_mhz)} frequencies of the Born map, {gs.nx * gs.ny} nodes of the adjoint; "
                      f"each extrapolated linearly to the full step: maps {t_maps:.0f} s, apply {t_apply:.0f} s, "
                      f"adjoint {t_adj:.0f} s"}


def _born_tc_flop(n_tx: int, n_in: int, n_freq: int) -> "tuple[float, float]":
    """(algorithmic FLOPs, executed TF32 tensor FLOPs) of one Born apply or
    adjoint: the complex contraction 8 n_tx^2 n_in per frequency; the kernels
    contract only the e-block <= r-block part of 128 x 128 blocks (d is
    symmetric), each real product as 3 TF32 products."""
    nb = (n_tx + 127) // 128
    alg = n_freq * 8.0 * n_tx * n_tx * n_in
    executed = n_freq * (nb * (nb + 1) / 2) * 128 * 256 * (2 * 16 * ((n_in + 15) // 16)) * 3 * 2.0
    return alg, executed


def born_leg(args, peaks, steps: int = 2, warmup: int = 1, variants: bool = False, cpu: bool = False) -> dict:
    """Ray-Born step on the breast model medium: first-arrival maps of all 512
    transducers (rtborn_maps), the Born data of a seeded perturbation at 8
    frequencies (rtborn_apply) and the adjoint of those data (rtborn_adjoint),
    the contractions on the tensor cores (TF32 split)."""
    import torch
    import paper_2511_18511_gb300 as rt
    from paper_2511_18511_gb300 import phantoms as P
    dev = torch.device("cuda", torch.cuda.current_device())
    w = P.cfg_born()
    prob = rt.Problem.create(w.grid, w.c, w.tx, w.ring_radius, device=dev)
    dc = torch.as_tensor(w.dc, dtype=torch.float32, device=dev)
    s = torch.cuda.current_stream(dev)
    nf = len(w.f_mhz)
    maps = rt.rtborn_maps(prob, w.ds, w.fan_rays)
    d = rt.rtborn_apply(maps, w.f_mhz, dc)
    g = rt.rtborn_adjoint(maps, w.f_mhz, d)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(gemm, ev=None):
        if ev:
            ev[0].record(s)
        rt.rtborn_maps(prob, w.ds, w.fan_rays, out=maps)
        if ev:
            ev[1].record(s)
        rt.rtborn_apply(maps, w.f_mhz, dc, gemm=gemm, out=d)
        if ev:
            ev[2].record(s)
        rt.rtborn_adjoint(maps, w.f_mhz, d, gemm=gemm, out=g)
        if ev:
            ev[3].record(s)

    def timed(gemm, n, nwarm):
        for _ in range(nwarm):
            step(gemm)
        torch.cuda.synchronize()
        evs = []
        for _ in range(n):
            flush.zero_()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            step(gemm, ev)
            evs.append(ev)
        torch.cuda.synchronize()
        return np.array([[e[k].elapsed_time(e[k + 1]) for k in range(3)] for e in evs]).mean(0)

    part = timed("tf32x3", steps, warmup)
    _, counts = rt.rt_status_counts()
    steps_per_call = counts[7]
    ms = float(part.sum())
    data = nf * w.n_tx * (w.n_tx - 1)
    n_in = int(np.sum(np.hypot(*w.grid.node_xy()) < w.ring_radius))
    alg, executed = _born_tc_flop(w.n_tx, n_in, nf)
    tf32 = peaks["tf32_tflops"]
    fp32 = peaks["fp32_tflops"]
    maps_tflops = steps_per_call * FLOP_PER_BORN_STEP / (part[0] / 1e3) / 1e12

    def tc_roof(kernel, ms_):
        ach = executed / (ms_ / 1e3) / 1e12
        return {"bound": "tensor", "achieved": ach, "peak": tf32, "unit": "TFLOP/s", "frac": ach / tf32,
                "traffic": None, "kernel": kernel, "algorithmic_tflops": alg / (ms_ / 1e3) / 1e12,
                "executed_flop": executed, "algorithmic_flop": alg,
                "peak_basis": "measured BF16 burst (MEASURED_PEAKS.json) x nominal TF32/BF16 1.1/2.25"}

    leg = {"metric": "ray-Born data/s (fan maps + Born apply + adjoint, 8 frequencies, 512-ring, 1024^2 grid)",
           "value": data / (ms / 1e3), "unit": "Born data/s", "ms_per_step": ms, "steps": steps, "warmup": warmup,
           "config": {"workload": w.name, "grid": f"{w.grid.nx}x{w.grid.ny}", "h_mm": w.grid.h, "ring": w.n_tx,
                      "ring_radius_mm": w.ring_radius, "fan_rays": w.fan_rays, "ds_mm": w.ds,
                      "f_mhz": [float(f) for f in w.f_mhz], "inside_nodes": n_in, "gemm": "tf32x3",
                      "step": "rtborn_maps + rtborn_apply + rtborn_adjoint",
                      "l2": "flushed between timed steps (256 MB write); maps 4.3 GB"},
           "parts_ms": {"maps": float(part[0]), "apply": float(part[1]), "adjoint": float(part[2])},
           "roofline": {"bound": "alu", "achieved": maps_tflops, "peak": fp32, "unit": "TFLOP/s",
                        "frac": maps_tflops / fp32,
                        "traffic": _traffic(os.path.join(ROOT, "profiles", "born_traffic.json"), BORN_HASH_FILES),
                        "kernel": "rtborn_maps call: k_born_fan + pack + unpack",
                        "flop_per_rk4_step": FLOP_PER_BORN_STEP, "rk4_steps_per_launch": steps_per_call,
                        "peak_basis": "measured FP32 FMA rate (rt_peak_fma)"},
           "roofline_apply": tc_roof("k_born_apply_tc (+ finish)", part[1]),
           "roofline_adjoint": tc_roof("k_born_dprep + k_born_adjoint_tc (+ finish)", part[2]),
           "maps": {"rays": w.n_tx * w.fan_rays, "rk4_steps": steps_per_call,
                    "rays_per_s": w.n_tx * w.fan_rays / (part[0] / 1e3)},
           # maps: pack, fan, unpack; apply: apply_tc, finish; adjoint: dprep, adjoint_tc, finish
           "gpu_launches_per_step": 3 + 2 + 3}
    if variants:
        part32 = timed("fp32", 1, 1)
        leg["parts_ms_fp32_simt"] = {"maps": float(part32[0]), "apply": float(part32[1]),
                                     "adjoint": float(part32[2])}
        alpha0 = torch.as_tensor(P.absorption_map(w.c), device=dev)
        for name, kw in (("absorption", dict(alpha0=alpha0, y=1.3)), ("bspline", dict(interpolator="bspline"))):
            m = rt.rtborn_maps(prob, w.ds, w.fan_rays, **kw)
            dd = rt.rtborn_apply(m, w.f_mhz, dc)
            gg = rt.rtborn_adjoint(m, w.f_mhz, dd)
            torch.cuda.synchronize()
            parts = []
            for _ in range(2):
                flush.zero_()
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
                ev[0].record(s)
                rt.rtborn_maps(prob, w.ds, w.fan_rays, out=m, **kw)
                ev[1].record(s)
                rt.rtborn_apply(m, w.f_mhz, dc, out=dd)
                ev[2].record(s)
                rt.rtborn_adjoint(m, w.f_mhz, dd, out=gg)
                ev[3].record(s)
                torch.cuda.synchronize()
                parts.append([ev[k].elapsed_time(ev[k + 1]) for k in range(3)])
            del m, dd, gg
            p_ = np.array(parts).mean(0)
            leg[name] = {"value": data / (p_.sum() / 1e3), "unit": "Born data/s", "ms_per_step": float(p_.sum()),
                         "parts_ms": {"maps": float(p_[0]), "apply": float(p_[1]), "adjoint": float(p_[2])}}
        leg["absorption"]["model"] = "alpha0 = 2e-8 (1 + 20 |c/1500 - 1|) Np (rad/s)^-y m^-1, y = 1.3"
        leg["bspline"]["sampler"] = "interpolating cubic B-spline (c, gradient, Hessian, s)"
    if cpu:
        leg["cpu_baseline"] = _born_cpu_baseline(w, n_fans=16, n_pairs=64, n_nodes=1024)
    return leg


def run_born(args):
    """The ray-Born step as its own JSON line (--workload born), with the
    end-to-end leg through host buffers."""
    import torch
    import paper_2511_18511_gb300 as rt
    from paper_2511_18511_gb300 import phantoms as P
    torch.cuda.set_device(0)
    peaks = measured_peaks()
    clocks = Clocks(0)
    clocks.start()
    leg = born_leg(args, peaks, steps=args.steps, warmup=args.warmup, variants=True,
                   cpu=not args.no_cpu_baseline)
    clk = clocks.stop()
    # e2e: host c and dc in, host data and gradient out
    w = P.cfg_born()
    prob = rt.Problem.create(w.grid, w.c, w.tx, w.ring_radius)
    c_host = torch.as_tensor(w.c).pin_memory()
    dc_host = torch.as_tensor(w.dc, dtype=torch.float32).pin_memory()
    dc = torch.empty_like(dc_host, device="cuda")
    c_dev = torch.empty_like(prob.c)
    maps = rt.rtborn_maps(prob, w.ds, w.fan_rays)
    d = rt.rtborn_apply(maps, w.f_mhz, dc.copy_(dc_host))
    g = rt.rtborn_adjoint(maps, w.f_mhz, d)
    d_host = torch.empty(d.shape, dtype=torch.complex64).pin_memory()
    g_host = torch.empty(g.shape, dtype=torch.float32).pin_memory()

    def e2e_step():
        c_dev.copy_(c_host, non_blocking=True)
        dc.copy_(dc_host, non_blocking=True)
        rt.rtborn_maps(prob, w.ds, w.fan_rays, c=c_dev, out=maps)
        rt.rtborn_apply(maps, w.f_mhz, dc, out=d)
        rt.rtborn_adjoint(maps, w.f_mhz, d, out=g)
        d_host.copy_(d, non_blocking=True)
        g_host.copy_(g, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    n_e2e = 2
    for _ in range(n_e2e):
        e2e_step()
        torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / n_e2e
    data = len(w.f_mhz) * w.n_tx * (w.n_tx - 1)
    line = dict(leg)
    cpu = line.pop("cpu_baseline", None)
    line.update({"n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
                 "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                 "e2e": {"value": data / e2e_s, "unit": "Born data/s",
                         "h2d_bytes_per_step": c_host.numel() * 8 + dc_host.numel() * 4,
                         "d2h_bytes_per_step": d_host.numel() * 8 + g_host.numel() * 4},
                 "gpu_launches": args.steps * leg["gpu_launches_per_step"], "clocks": clk, "peaks": peaks})
    if cpu:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)


def run_profile_case(args):
    """One rt_link on a subset of pairs of the full-size workload (ncu captures);
    with --workload born, rtborn_maps on the first N_EMIT transducers, then the
    Born apply and adjoint (tensor-core path) of those maps at two frequencies."""
    import torch
    if args.workload == "batch":
        import paper_2511_18511_gb300 as rt
        from paper_2511_18511_gb300 import phantoms as P
        ws = P.cfg_batch()[:args.profile]
        insts = [rt.BatchInstance.create(rt.Problem.create(w.grid, w.c, w.tx, w.ring_radius)) for w in ws]
        for b in insts:                  # "measured" times: the same media 0.5 % faster, as the batch leg
            c0 = b.prob.c.clone()
            b.prob.c.mul_(1.005)
            rt.rt_batch_run([b], ws[0].ds)
            b.prob.c.copy_(c0)
            b.tof_ref = b.tof.clone()
            b.g_c = torch.empty_like(b.prob.c)
        kw = dict(zip(("block_threads", "step_unroll", "blocks_per_sm"), BATCH_PROFILE_VARIANT))
        for _ in range(2):
            rt.rt_batch_run(insts, ws[0].ds, fan_ds=0.5 * ws[0].grid.h, **kw)
        torch.cuda.synchronize()
        ok, counts = rt.rt_status_counts()
        print(json.dumps({"profile_case": "batch32_uneven", "instances": len(insts),
                          "pairs": sum(b.prob.n_pairs for b in insts), "variant": list(BATCH_PROFILE_VARIANT),
                          "all_linked": ok, "rk4_steps": counts[7]}))
        return
    if args.workload == "born":
        import paper_2511_18511_gb300 as rt
        from paper_2511_18511_gb300 import phantoms as P
        w = P.cfg_born()
        n = args.profile
        prob = rt.Problem.create(w.grid, w.c, w.tx[:n], w.ring_radius)
        maps = None
        for _ in range(2):
            maps = rt.rtborn_maps(prob, w.ds, w.fan_rays, out=maps)
        torch.cuda.synchronize()
        _, counts = rt.rt_status_counts()
        dc = torch.as_tensor(w.dc, dtype=torch.float32, device="cuda")
        f = list(w.f_mhz[:2])
        d = rt.rtborn_apply(maps, f, dc)
        g = rt.rtborn_adjoint(maps, f, d)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": w.name, "transducers": n, "fan_rays": w.fan_rays,
                          "rk4_steps": counts[7], "born_frequencies": f,
                          "finite": bool(torch.isfinite(d).all()) and bool(torch.isfinite(g).all())}))
        return
    import paper_2511_18511_gb300 as rt
    from paper_2511_18511_gb300 import phantoms as P
    w = workload(0)
    pairs = P.all_pairs(w.n_tx)
    pairs = pairs[pairs[:, 0] < args.profile]
    # all emitters: the implicit all-pairs list, served in the bench's queue order
    prob = rt.Problem.create(w.grid, w.c, w.tx, w.ring_radius, pairs=None if args.profile >= w.n_tx else pairs)
    rows = rt.Rows.create(prob) if args.precision == "fp32c" else None
    for _ in range(2):
        if rows is not None:       # the bench's step: recorded rows
            r = rt.rt_link_rows(prob, w.ds, rows, tol=w.tol, fan_rays=BREAST_FAN, fan_ds=FAN_DS)
            rt.rt_tof_adjoint_rows(prob, rows, r["theta"], r["tof"], w.ds, tof_ref=r["tof"] * 0.999)
        else:
            r = rt.rt_link(prob, w.ds, tol=w.tol, precision=args.precision, fan_rays=BREAST_FAN, fan_ds=FAN_DS)
            rt.rt_tof_adjoint(prob, r["theta"], r["tof"], w.ds, tof_ref=r["tof"] * 0.999, precision=args.precision)
    torch.cuda.synchronize()
    ok, counts = rt.rt_status_counts()
    print(json.dumps({"profile_case": w.name, "pairs": int(len(pairs)), "precision": args.precision,
                      "all_linked": ok, "rk4_steps": counts[7],
                      "mean_traces": float(r["iters"].float().mean().item())}))


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(rank: int):
    from paper_2511_18511_gb300 import phantoms as P
    return P.cfg_breast(seed=3 + rank)


class Clocks:
    """nvidia-smi sampling (every 200 ms) during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except (ValueError, IndexError):
                continue
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(w, n_emit: int = 16, nthreads: int = 0, steps: int = 1) -> dict:
    """The FP64 oracle, as it stands, on a bounded sample of the workload with
    the same algorithm as the GPU step (cold start from a fan of BREAST_FAN
    rays per emitter, then link + misfit adjoint): n_emit emitters spread over
    the ring, each with all its receivers; nthreads 0 = every host core. The
    measured times T_meas come from c_true before timing."""
    import oracle
    from paper_2511_18511_gb300 import phantoms as P
    oracle.build()
    pairs = P.all_pairs(w.n_tx)
    emit = np.arange(0, w.n_tx, max(1, w.n_tx // n_emit))[:n_emit]
    sub = pairs[np.isin(pairs[:, 0], emit)]
    ref = oracle.link(w.grid, w.c_true, w.tx, w.ring_radius, w.ds, tol=w.tol, pairs=sub, fan_rays=BREAST_FAN,
                      fan_ds=FAN_DS, nthreads=nthreads)
    t_meas = ref["tof"]
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        r = oracle.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, tol=w.tol, pairs=sub, fan_rays=BREAST_FAN,
                        fan_ds=FAN_DS, nthreads=nthreads)
        oracle.adjoint(w.grid, w.c, w.tx, w.ring_radius, w.ds, r["theta"], r["tof"] - t_meas, pairs=sub,
                       nthreads=nthreads)
        times.append(time.perf_counter() - t0)
    dt = float(np.median(times))
    cores = oracle.num_threads() if nthreads == 0 else nthreads
    return {"value": len(sub) / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{len(sub)} pairs ({len(emit)} emitters x {w.n_tx - 1} receivers) of the "
                      f"{w.name} workload, cold start from a {BREAST_FAN}-ray fan at {FAN_DS} mm, link + adjoint, "
                      f"{dt:.2f} s per pass on {cores} thread(s)",
            "mean_traces_per_pair": float(np.mean(r["iters"]))}


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores, each step a
    bounded sample (16 emitters x 511 receivers) of the breast workload with
    the GPU step's algorithm. Under torchrun only rank 0 runs it."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w = workload(0)
    vals = []
    for _ in range(args.warmup):
        cpu_baseline(w, n_emit=16)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(w, n_emit=16))
    total = time.perf_counter() - t0
    v = float(np.mean([x["value"] for x in vals]))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / max(args.steps, 1),
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w.name, "grid": f"{w.grid.nx}x{w.grid.ny}", "ring": w.n_tx,
                                            "start": f"cold: fan of {BREAST_FAN} rays per transducer at {FAN_DS} mm",
                                            "pairs_per_step": "16 emitters x 511 receivers (bounded sample)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": vals[0]["cores"], "kind": "oracle",
                             "sample": vals[0]["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_tof_config(args):
    """The ToF step (cold fan start) on one of the smaller configurations as its
    own line: the 128^2 / 64-ring Gaussian-inclusion medium (4,032 pairs;
    FP32-compensated step rt_link_rows + rt_tof_adjoint_rows, as on the
    headline workload) or the fish-eye lens on 512^2 with a 256-ring (65,280
    pairs; rt_link + rt_tof_adjoint: every emitter's rays meet near its
    conjugate point, where the FP64 atomics of either adjoint pile onto a few
    cells (16 ms both ways), so the recording link's extra cost, 84.4 against
    79.6 ms, is not paid back); the FP64 step is rt_link + rt_tof_adjoint; the
    oracle on all host cores and on one thread (bounded samples of the same
    step)."""
    import torch
    import oracle
    import paper_2511_18511_gb300 as rt
    from paper_2511_18511_gb300 import phantoms as P
    torch.cuda.set_device(0)
    peaks = measured_peaks()
    w = P.cfg_small() if args.workload == "small" else P.cfg_fisheye()
    fan, fan_ds = 256, 0.5 * w.grid.h
    prob = rt.Problem.create(w.grid, w.c, w.tx, w.ring_radius)
    t_meas = rt.rt_link(prob, w.ds, tol=w.tol, precision="fp64", c=prob.c * 1.002, fan_rays=fan)["tof"].clone()
    s = torch.cuda.current_stream()
    rows = rt.Rows.create(prob)

    use_rows = args.workload == "small"

    def one(prec, out, g, mid=None):
        if prec == "fp32c" and use_rows:
            r = rt.rt_link_rows(prob, w.ds, rows, tol=w.tol, fan_rays=fan, fan_ds=fan_ds, out=out)
            if mid is not None:
                mid.record(s)
            g = rt.rt_tof_adjoint_rows(prob, rows, r["theta"], r["tof"], w.ds, tof_ref=t_meas, out=g)
        else:
            r = rt.rt_link(prob, w.ds, tol=w.tol, precision=prec, fan_rays=fan, fan_ds=fan_ds, out=out)
            if mid is not None:
                mid.record(s)
            g = rt.rt_tof_adjoint(prob, r["theta"], r["tof"], w.ds, tof_ref=t_meas, precision=prec, out=g)
        return r, g

    def timed(prec, steps, warmup):
        out, g = None, None
        for _ in range(warmup):
            out, g = one(prec, out, g)
        torch.cuda.synchronize()
        ts = []
        for _ in range(steps):
            a, m, b = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            a.record(s)
            one(prec, out, g, m)
            b.record(s)
            ts.append((a, m, b))
        torch.cuda.synchronize()
        ok, counts = rt.rt_status_counts()
        split = (float(np.mean([a.elapsed_time(m) for a, m, _ in ts])), float(np.mean([m.elapsed_time(b) for _, m, b in ts])))
        return float(np.mean([a.elapsed_time(b) for a, _, b in ts])), ok, counts, out, split

    clocks = Clocks(0)
    clocks.start()
    ms, ok, counts, out, split = timed("fp32c", args.steps, args.warmup)
    clk = clocks.stop()
    ms64, ok64, _, _, _ = timed("fp64", 1, 1)
    n = prob.n_pairs
    # the oracle on the same step: a bounded sample of emitters (all cores, then one thread)
    oracle.build()
    pairs = P.all_pairs(w.n_tx)

    def cpu(n_emit, nthreads):
        emit = np.arange(0, w.n_tx, max(1, w.n_tx // n_emit))[:n_emit]
        sub = pairs[np.isin(pairs[:, 0], emit)]
        tm = t_meas.cpu().numpy()[np.isin(pairs[:, 0], emit)]
        t0 = time.perf_counter()
        r = oracle.link(w.grid, w.c, w.tx, w.ring_radius, w.ds, tol=w.tol, pairs=sub, fan_rays=fan, fan_ds=fan_ds,
                        nthreads=nthreads)
        oracle.adjoint(w.grid, w.c, w.tx, w.ring_radius, w.ds, r["theta"], r["tof"] - tm, pairs=sub,
                       nthreads=nthreads)
        dt = time.perf_counter() - t0
        cores = oracle.num_threads() if nthreads == 0 else nthreads
        return {"value": len(sub) / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                "sample": f"{len(sub)} pairs ({len(emit)} emitters x {w.n_tx - 1} receivers), cold fan start, "
                          f"link + adjoint, {dt:.2f} s on {cores} thread(s)"}

    n_all = 16 if w.n_tx >= 64 else w.n_tx
    cb = cpu(n_all, 0)
    cb["one_thread"] = cpu(2, 1)
    line = {"metric": f"linked rays/s (ToF fwd+adjoint, {w.name})", "value": n / (ms / 1e3), "unit": UNIT,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "grid": f"{w.grid.nx}x{w.grid.ny}", "h_mm": w.grid.h, "ring": w.n_tx,
                       "ring_radius_mm": w.ring_radius, "pairs": n, "ds_mm": w.ds, "tol_mm": w.tol,
                       "start": f"cold: fan of {fan} rays per transducer at {fan_ds} mm",
                       "step": ("rt_link_rows + rt_tof_adjoint_rows" if use_rows else "rt_link + rt_tof_adjoint")
                               + " (L2 misfit against times in c x 1.002)"},
            "link": {"all_linked": ok, "status_counts": counts[:7],
                     "mean_traces_per_pair": float(out["iters"].float().mean().item()),
                     "link_ms": split[0], "adjoint_ms": split[1]},
            "fp64_gpu": {"value": n / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64, "all_linked": ok64,
                         "speedup_fp32c_over_fp64": ms64 / ms},
            "gpu_launches": (10 if use_rows else 9) * args.steps, "clocks": clk, "peaks": peaks, "cpu_baseline": cb}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile:
        return run_profile_case(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "born":
        return run_born(args)
    if args.workload in ("small", "fisheye"):
        return run_tof_config(args)
    import torch
    import paper_2511_18511_gb300 as rt
    from paper_2511_18511_gb300 import shard

    rank, world, local = dist_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    peaks = measured_peaks()

    w = workload(0)            # one problem; with N > 1 every rank takes its emitter block
    ctx = rt.Context(local)
    ctx.reserve(w.grid.nx * w.grid.ny)
    sharded = None
    if world > 1:
        sharded = shard.ShardedToF(rank, world, w.n_tx, link=None, adjoint=None)
    prob = rt.Problem.create(w.grid, w.c, w.tx, w.ring_radius, device=dev,
                             pairs=None if sharded is None else sharded.pairs)
    c_true = torch.as_tensor(w.c_true, device=dev)
    stream = torch.cuda.current_stream(dev)
    n = prob.n_pairs
    n_all = w.n_tx * (w.n_tx - 1)

    # "measured" travel times from the true medium (outside any timed region)
    meas = rt.rt_link(prob, w.ds, tol=w.tol, precision="fp64", c=c_true, ctx=ctx)
    t_meas = meas["tof"].clone()
    rows = rt.Rows.create(prob)       # recorded rows of the step's linked rays
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def buffers():
        return dict(theta=torch.empty(n, dtype=torch.float64, device=dev),
                    tof=torch.empty(n, dtype=torch.float64, device=dev),
                    hit=torch.empty((n, 2), dtype=torch.float64, device=dev),
                    status=torch.empty(n, dtype=torch.int32, device=dev),
                    iters=torch.empty(n, dtype=torch.int32, device=dev))

    def step(prec, out, g, ev=None, c=None, tm=None, **kw):
        """Link (cold) + adjoint of the misfit, an event between them: in the
        FP32-compensated bilinear form rt_link_rows + rt_tof_adjoint_rows (the
        link records its rays' rows, the adjoint reads them), otherwise rt_link
        + rt_tof_adjoint; with N > 1 the ShardedToF step: this rank's pairs,
        then one all-reduce of g."""
        tm = t_meas if tm is None else tm
        use_rows = prec == "fp32c" and not kw

        def link(_pairs, cc):
            if use_rows:
                r = rt.rt_link_rows(prob, w.ds, rows, tol=w.tol, c=cc, ctx=ctx, out=out, fan_rays=BREAST_FAN,
                                    fan_ds=FAN_DS)
            else:
                r = rt.rt_link(prob, w.ds, tol=w.tol, precision=prec, c=cc, ctx=ctx, out=out, fan_rays=BREAST_FAN,
                               fan_ds=FAN_DS, **kw)
            if ev:
                ev[1].record(stream)
            return r["theta"], r["tof"]

        def adjoint(_pairs, cc, theta, tof, tof_meas):
            if use_rows:
                return rt.rt_tof_adjoint_rows(prob, rows, theta, tof, w.ds, tof_ref=tof_meas, c=cc, ctx=ctx, out=g)
            return rt.rt_tof_adjoint(prob, theta, tof, w.ds, tof_ref=tof_meas, precision=prec, c=cc, ctx=ctx,
                                     out=g, **kw)

        if ev:
            ev[0].record(stream)
        if sharded is None:
            theta, tof = link(None, c)
            adjoint(None, c, theta, tof, tm)
        else:
            sharded.link, sharded.adjoint = link, adjoint
            sharded.step(c, tm)
        if ev:
            ev[2].record(stream)

    def timed(prec, steps, warmup, clocks=None, **kw):
        out, g = buffers(), torch.empty_like(prob.c)
        for _ in range(warmup):
            step(prec, out, g, **kw)
        torch.cuda.synchronize()
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
        for k in range(steps):
            flush.zero_()
            step(prec, out, g, ev[k], **kw)
        torch.cuda.synchronize()
        clk = clocks.stop() if clocks else None
        if dist is not None:
            dist.barrier()
        step_ms = [a.elapsed_time(c) for a, b, c in ev]
        link_ms = [a.elapsed_time(b) for a, b, c in ev]
        ok, counts = rt.rt_status_counts(ctx)
        return dict(step_ms=step_ms, link_ms=link_ms, counts=counts, ok=ok, clocks=clk,
                    iters=out["iters"].float().mean().item(), g=g, out=out)

    clocks = Clocks(local)
    res = timed("fp32c", args.steps, args.warmup, clocks)
    total_ms = float(np.sum(res["step_ms"]))
    if dist is not None:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = n_all / (ms_per_step / 1e3)
    fp32 = peaks["fp32_tflops"]
    link_ms = float(np.mean(res["link_ms"]))
    adjoint_ms = float(np.mean(res["step_ms"])) - link_ms
    steps_per_launch = res["counts"][7]
    achieved = steps_per_launch * FLOP_PER_STEP / (link_ms / 1e3) / 1e12
    traffic = _traffic(args.traffic_json, ("rt_trace.cuh", "rt_link.cuh", "rt_bspline.cuh", "rt_ray.cu"))

    # e2e through the public API with host buffers (pinned), copies timed
    c_host = torch.as_tensor(w.c).pin_memory()
    tm_host = t_meas.cpu().pin_memory()
    T_host = torch.empty(n, dtype=torch.float64).pin_memory()
    g_host = torch.empty_like(c_host).pin_memory()
    c_dev = torch.empty_like(prob.c)
    tm_dev = torch.empty_like(t_meas)
    out_e, g_e = buffers(), torch.empty_like(prob.c)
    e2e_steps = max(2, min(args.steps, 3))

    def e2e_step():
        c_dev.copy_(c_host, non_blocking=True)
        tm_dev.copy_(tm_host, non_blocking=True)
        step("fp32c", out_e, g_e, c=c_dev, tm=tm_dev)
        T_host.copy_(out_e["tof"], non_blocking=True)
        g_host.copy_(g_e, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
        torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    if dist is not None:
        t = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    h2d = world * (c_host.numel() * 8 + tm_host.numel() * 8)
    d2h = world * (T_host.numel() * 8 + g_host.numel() * 8)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        # one fixed problem whatever the number of ranks (each takes its emitter block)
        "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "grid": f"{w.grid.nx}x{w.grid.ny}", "h_mm": w.grid.h, "ring": w.n_tx,
                   "ring_radius_mm": w.ring_radius, "pairs": n_all, "ds_mm": w.ds, "tol_mm": w.tol,
                   "start": f"cold: fan of {BREAST_FAN} rays per transducer traced at {FAN_DS} mm",
                   "fan_rays": BREAST_FAN, "fan_ds_mm": FAN_DS,
                   "step": "rt_link_rows + rt_tof_adjoint_rows (L2 misfit; the link records its rays' rows "
                           "of the system matrix, the adjoint reads them)" + (
                       "; pairs split over ranks by emitter block (longest chords first), NCCL all-reduce of "
                       "the gradient inside the step" if world > 1 else ""),
                   "precision": "fp32c (FP32 march, compensated direction/sums, FP64 linking)",
                   "l2": "flushed between timed steps (256 MB write)"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32, "unit": "TFLOP/s",
                     "frac": achieved / fp32, "traffic": traffic,
                     "kernel": "rt_link_rows call: k_fan<float> + k_link<float, recording> (+ field pack)",
                     "flop_per_rk4_step": FLOP_PER_STEP, "rk4_steps_per_launch": steps_per_launch,
                     "peak_basis": "FP32 FMA rate measured at start-up on this GPU (rt_peak_fma)"},
        "link": {"mean_traces_per_pair": res["iters"], "all_linked": res["ok"],
                 "status_counts": res["counts"][:7], "link_ms": link_ms, "adjoint_ms": adjoint_ms},
        "e2e": {"value": n_all / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        # per step: rt_link_rows = k_pack, k_tx_phi, k_fan_mark, k_fan, k_link;
        # rt_tof_adjoint_rows = k_pack, k_tx_phi, k_adjoint_rows, k_adjoint_unrecorded, k_adjoint_finish
        "gpu_launches": 10 * args.steps,
        "clocks": res["clocks"],
        "peaks": peaks,
    }
    if world > 1:
        line["library_launches"] = {"nccl_all_reduce": args.steps}
        line["pairs_per_rank"] = n
    if world == 1:
        line.update(single_gpu_legs(args, peaks, rt, torch, prob, w, ctx, timed, res, link_ms, adjoint_ms,
                                    ms_per_step, steps_per_launch, dev, stream, flush, t_meas, buffers, rows))
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, n_emit=16)
        line["cpu_baseline"]["one_thread"] = cpu_baseline(w, n_emit=2, nthreads=1)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def single_gpu_legs(args, peaks, rt, torch, prob, w, ctx, timed, res, link_ms, adjoint_ms, ms_per_step,
                    steps_per_launch, dev, stream, flush, t_meas, buffers, rows) -> dict:
    """Sub-objects of the 1-GPU line: the adjoint kernel's roofline, the
    L2-gather comparison, the plain FP64 form, the warm start, the cubic
    B-spline sampler, the batched workload and the ray-Born step."""
    fp32 = peaks["fp32_tflops"]
    n = prob.n_pairs
    legs = {}
    # the plain FP64 GPU form on the same workload (fewer steps: it is slow on GB300)
    r64 = timed("fp64", max(1, args.fp64_steps), 1)
    ms64 = float(np.mean(r64["step_ms"]))
    legs["fp64_gpu"] = {"value": n / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64,
                        "speedup_fp32c_over_fp64": ms64 / ms_per_step}

    # warm start: the same step relinked from the previous step's angles (the
    # paper's later linearisations, Sec. 3.4.1); one trace per pair, so its
    # RK4 count is also the adjoint's retrace count
    theta_prev = res["out"]["theta"].clone()
    out_w, g_w = buffers(), torch.empty_like(prob.c)
    warm_ms, warm_link = [], []
    for k in range(max(2, min(args.steps, 3)) + 1):
        flush.zero_()
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record(stream)
        r = rt.rt_link(prob, w.ds, tol=w.tol, precision="fp32c", theta0=theta_prev, ctx=ctx, out=out_w)
        b.record(stream)
        rt.rt_tof_adjoint(prob, r["theta"], r["tof"], w.ds, tof_ref=t_meas, precision="fp32c", ctx=ctx, out=g_w)
        c.record(stream)
        torch.cuda.synchronize()
        if k:
            warm_ms.append(a.elapsed_time(c))
            warm_link.append(a.elapsed_time(b))
    _, wcounts = rt.rt_status_counts(ctx)
    retrace_steps = wcounts[7]
    warm = float(np.mean(warm_ms))
    legs["warm_start"] = {"value": n / (warm / 1e3), "unit": UNIT, "ms_per_step": warm,
                          "link_ms": float(np.mean(warm_link)),
                          "mean_traces_per_pair": float(out_w["iters"].float().mean().item()),
                          "start": "the previous step's linked angles"}
    # the adjoint from recorded rows reads every pair's runs (20 B each) and
    # adds four FP64 atomics per run into the L2-resident gradient
    runs = int(rows.len.clamp(min=0).sum().item())
    adj_bytes = runs * 20 + n * (4 + 8 + 8)
    adj_gbs = adj_bytes / (adjoint_ms / 1e3) / 1e9
    hbm = peaks["hbm_gbs"]
    legs["roofline_adjoint"] = {
        "bound": "hbm", "achieved": adj_gbs, "peak": hbm, "unit": "GB/s", "frac": adj_gbs / hbm,
        "traffic": _traffic(os.path.join(ROOT, "profiles", "adjoint_traffic.json"), ("rt_ray.cu", "rt_link.cuh")),
        "kernel": "rt_tof_adjoint_rows call: k_adjoint_rows (+ pack, finish)",
        "bytes_per_launch": adj_bytes, "runs": runs, "runs_per_s": runs / (adjoint_ms / 1e3),
        "note": "algorithmic bytes = the recorded runs (20 B each) + 20 B per pair; the gradient stays in L2 and "
                "takes FP64 atomics, up to four per run (a lane first sums the nodes that consecutive cells of "
                "its ray share)",
        "peak_basis": "measured HBM copy rate (MEASURED_PEAKS.json)"}
    # the link without recording (rt_link), for the cost of the recording
    out_p = buffers()
    tl = []
    for k in range(3):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        rt.rt_link(prob, w.ds, tol=w.tol, precision="fp32c", ctx=ctx, out=out_p, fan_rays=BREAST_FAN, fan_ds=FAN_DS)
        b.record(stream)
        torch.cuda.synchronize()
        if k:
            tl.append(a.elapsed_time(b))
    legs["link_without_rows_ms"] = float(np.mean(tl))
    # the same adjoint by retracing every ray (rt_tof_adjoint), for comparison
    g_r = torch.empty_like(prob.c)
    ta = []
    for k in range(3):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        rt.rt_tof_adjoint(prob, res["out"]["theta"], res["out"]["tof"], w.ds, tof_ref=t_meas, precision="fp32c",
                          ctx=ctx, out=g_r)
        b.record(stream)
        torch.cuda.synchronize()
        if k:
            ta.append(a.elapsed_time(b))
    retrace_ms = float(np.mean(ta))
    adj_ach = retrace_steps * FLOP_PER_STEP / (retrace_ms / 1e3) / 1e12
    legs["adjoint_by_retrace"] = {
        "ms": retrace_ms, "achieved_tflops": adj_ach, "frac_of_fp32": adj_ach / fp32,
        "rk4_steps_per_launch": retrace_steps, "kernel": "rt_tof_adjoint: k_adjoint<float> retraces every ray",
        "max_rel_diff_of_gradient": float(((g_r - res["g"]).abs().max() / g_r.abs().max()).item())}
    gath = steps_per_launch * GATHER_BYTES_PER_STEP / (link_ms / 1e3) / 1e9
    legs["l2_gather"] = {
        "bytes_per_rk4_step": GATHER_BYTES_PER_STEP, "achieved_gbs": gath, "peak_gbs": peaks["l2_gather_gbs"],
        "frac": gath / peaks["l2_gather_gbs"],
        "note": "the rt_link call's RK4 steps x the 256 B a per-sample 2x2 float4 gather would read, over the "
                "measured random-float4 L2 gather rate; above 1 because the kernel caches each cell's "
                "coefficients in registers and reloads them about once per eight steps"}

    # the same step with the interpolating cubic B-spline sampler (Sec. 3.3.1's
    # second scheme), FP32-compensated, cold start
    rb = timed("fp32c", max(2, min(args.steps, 3)), 1, interpolator="bspline")
    bs_ms, bs_link = float(np.mean(rb["step_ms"])), float(np.mean(rb["link_ms"]))
    bs_ach = rb["counts"][7] * FLOP_PER_BSPLINE_STEP / (bs_link / 1e3) / 1e12
    legs["bspline"] = {"value": n / (bs_ms / 1e3), "unit": UNIT, "ms_per_step": bs_ms, "link_ms": bs_link,
                       "adjoint_ms": bs_ms - bs_link, "all_linked": rb["ok"], "mean_traces_per_pair": rb["iters"],
                       "rk4_steps_per_launch": rb["counts"][7], "flop_per_rk4_step": FLOP_PER_BSPLINE_STEP,
                       "achieved_tflops": bs_ach, "frac": bs_ach / fp32,
                       "sampler": "interpolating cubic B-spline (bicubic per cell, analytic gradient)"}
    if not args.no_legs:
        legs["batch"] = batch_leg(args, peaks)
        legs["born"] = born_leg(args, peaks)
    return legs


def _kernel_hash(files=("rt_trace.cuh", "rt_link.cuh", "rt_bspline.cuh", "rt_ray.cu")) -> str:
    import hashlib
    h = hashlib.sha1()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_2511_18511_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:12]


BORN_HASH_FILES = ("rt_trace.cuh", "rt_bspline.cuh", "rt_born.cu")
BATCH_HASH_FILES = ("rt_trace.cuh", "rt_link.cuh", "rt_batch.cu")
# the k_batch variant (rays per block, RK4 steps per queue check, blocks per SM)
# of the committed batch captures; the batch leg reports their traffic only when
# the autotuner picked this variant
BATCH_PROFILE_VARIANT = (128, 16, 5)


def _traffic(path: str, files) -> "int | None":
    """DRAM bytes per launch from a committed ncu summary, or None when the
    kernel sources changed since it was captured."""
    try:
        tj = json.load(open(path))
        return tj.get("bytes_per_launch") if tj.get("kernel_source_hash") == _kernel_hash(files) else None
    except Exception:
        return None


if __name__ == "__main__":
    main()
