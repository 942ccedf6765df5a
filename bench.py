#!/usr/bin/env python
"""Benchmark of the disconnected-loop hot path on GB300.

One step is one pass of the whole path over one synthetic gauge configuration
of the paper's lattice shape (16^3 x 32; Sec. 2): complex Z2 noise with
spin x colour x even-odd dilution and time dilution by translation (64 noise
vectors x 24 = 1536 right-hand sides per rank), the batched mixed-precision
even-odd BiCGStab with FP64 defect correction to a true residual of 1e-10,
and the loop contraction Tr[Gamma M^{-1}(x,x)] on each source timeslice for a
local and a Gaussian-smeared sink (alpha = 4, 50 iterations).

Printed (rank 0, one JSON line): solves/s of that step (right-hand sides
solved to 1e-10 and contracted, summed over ranks), the end-to-end figure
through host buffers (gauge field uploaded from the host and loops read back
every step), the Wilson-hop roofline from CUDA events around every hop launch
of the timed region, the plain single-right-hand-side FP64 solve rate for
comparison, clocks, and the FP64 CPU oracle timed on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "dslash HBM GB/s (% of peak); solves/s and loops/s at res 1e-10 vs plain FP64"
WORKLOAD = dict(name="stochastic_loops_16x16x16x32", dims=(16, 16, 16, 32), kappa=0.140, eps=0.45, seed=1,
                n_noise=64, dilution="spin*colour*evenodd*time", t0="n mod T", tol=1e-10,
                smear_alpha=4.0, smear_iter=50)
# The paper's kappa = 0.157 on links rough enough to keep M subcritical (eps 0.60, plaquette ~0.37)
WORKLOAD_K157 = dict(WORKLOAD, name="stochastic_loops_16x16x16x32_k157", kappa=0.157, eps=0.60)
CHUNK_NOISE = 4  # noise vectors per solve call (96 right-hand sides)
# the Wilson-hop kernel kinds of the autotuner (dl_tune_hop)
HOP_KIND_NAMES = {0: "hop_kernel_cap (direct)", 1: "hop_kernel_pf (cp.async prefetch)",
                  2: "hop_kernel_tma (block-staged)", 3: "hop_kernel (blocked order)",
                  4: "hop_kernel_ws (warp-staged)", 5: "hop_kernel_mma (tensor cores)",
                  6: "hop_kernel_x2 (packed FP32)", 7: "hop_kernel_pair (paired layout)",
                  8: "hop_kernel_pair_cap (paired layout)", 9: "hop_kernel_ws_pair (paired, warp-staged)",
                  10: "hop_kernel_cap (direct, wider register cap)", 11: "hop_kernel_ws (warp-staged, two stages)"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["f32", "bf16"], default="f32")
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--hop-shape", default=None, metavar="R:BLOCK:KIND,R:BLOCK:KIND,R:BLOCK:KIND",
                    help="launch shapes of the plain, the <rhat, v>-fused and the five-reduction fused Wilson "
                         "hops for the benchmark line (default: the autotuner's choice); lets a profiler run "
                         "use the kernels the timed run chose, which the line records")
    ap.add_argument("--kappa-literal", action="store_true",
                    help="the benchmark workload at kappa 0.157 on eps 0.60 links instead of kappa 0.140 on eps 0.45")
    ap.add_argument("--workload", default="stochastic",
                    choices=["stochastic", "exact_4x4x4x4", "single_rhs_16x16x16x32", "tsm_8x8x8x16",
                             "autograd", "correlators_16x16x16x32", "dilution_8x8x8x16",
                             "batch_scan_16x16x16x32", "tsm_16x16x16x32", "mixed_16x16x16x32",
                             "clover_16x16x16x32"],
                    help="stochastic: the benchmark line (default); the others measure the remaining "
                         "configurations and print one JSON line each")
    ap.add_argument("--smear-profile", metavar="N", type=int, default=None,
                    help="time the Gaussian smearing (alpha 4, 50 iterations) of N spin x colour x even-odd "
                         "diluted fields on one timeslice of 16^3x32 alone and exit")
    ap.add_argument("--solve-profile", metavar="N", type=int, default=None,
                    help="time two FP32-inner solves of N time-diluted noise sources on 16^3x32 (batch N) and "
                         "report the defect-correction hop timing of the second, then exit")
    ap.add_argument("--hop-profile", metavar="PREC:N[:KIND[:R:BLOCK]]", default=None,
                    help="time the Wilson hop alone on the 16^3x32 workload (f32|bf16|f64, batch N, kernel kind "
                         "0 direct / 1 prefetch / 2 staged, right-hand sides per thread, block size; default "
                         "autotuned) and exit.  With all five fields the hop launches are, in order: 24 of the "
                         "forced tuning run (two sweeps), 22 timing the choice, 8 plain (3 warm-up), 8 XPAY + "
                         "<rhat, v> (3 warm-up), 8 XPAY + five reductions (3 warm-up)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        p = json.load(open(path))
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# The ncu summary of the FP32 hops at the bench width, and the source files each
# kernel kind it covers is built from: its figures count only while those are unchanged.
# Its per-launch DRAM lines are keyed by kind and hop: plain, r0dot, bicg.
TRAFFIC_PROFILE = os.path.join("profiles", "hop_f32_fused_n32_16x16x16x32.md")
TRAFFIC_SOURCES = {0: ["hop.cuh"], 4: ["hop.cuh", "hop_tma.cuh", "hop_ws.cuh"], 10: ["hop.cuh", "hop_launch.cuh"],
                   11: ["hop.cuh", "hop_tma.cuh", "hop_ws.cuh"]}


def sources_sha(hop_kind: int):
    import hashlib
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES[hop_kind]:
        h.update(open(os.path.join(ROOT, "paper_1012_5168_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def read_traffic(kind: str, hop_kind: int):
    """Per-launch DRAM bytes of the hop kernel kind from the committed ncu summary, if current."""
    path = os.path.join(ROOT, TRAFFIC_PROFILE)
    if hop_kind not in TRAFFIC_SOURCES or not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line and line.startswith("- "):
            k, v = line[2:].split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get(f"kind {hop_kind} sources sha256") != sources_sha(hop_kind):
        return None
    key = f"kind {hop_kind} {kind} dram bytes per launch"
    return float(vals[key]) if key in vals else None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.out = []
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            txt, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            txt, _ = self.proc.communicate()
        rows = [r.split(", ") for r in txt.strip().splitlines() if r.strip()]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, r[4:8]):
                if v.strip() == "Active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# oracle baseline (CPU)
# ---------------------------------------------------------------------------
def oracle_iters_needed() -> int:
    path = os.path.join(ROOT, "tests", "golden", "oracle_bicgstab_iters_16x16x16x32.txt")
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            return int(line.split()[0])
    raise RuntimeError("no iteration count in " + path)


def oracle_sample(seconds: float = 20.0, min_iters: int = 1):
    """Time the oracle's full-lattice BiCGStab on the workload for about `seconds`,
    and over at least `min_iters` iterations.

    Returns (solves/s, description).  The oracle runs whole BiCGStab
    iterations on one 16^3 x 32 Z2 source; solves/s = 1 / (seconds per iteration
    x iterations the oracle needs for 1e-10 on this workload, from
    tests/golden/oracle_bicgstab_iters_16x16x16x32.txt).
    """
    import numpy as np
    import synthetic
    from oracle import noise, wilson
    w = WORKLOAD
    U = synthetic.gauge_field(w["dims"], w["eps"], w["seed"])
    b = noise.z2_noise(w["dims"], 1, 0)
    n_it = max(1, int(min_iters))
    t_iter = None
    cpu0, wall0 = time.process_time(), time.perf_counter()
    while True:
        t0 = time.perf_counter()
        wilson.bicgstab(lambda v: wilson.apply_m(U, v, w["kappa"], -1.0), b, tol=1e-30, max_iter=n_it,
                        max_restarts=0)
        dt = time.perf_counter() - t0
        # subtract the two extra matvecs of the true-residual checks (before and after)
        t_iter = max(dt, 1e-9) / (n_it + 1.0)
        if dt >= seconds / 4 or n_it >= 64:
            break
        if n_it >= min_iters and dt >= seconds / 8:
            break
        n_it = min(64, max(n_it * 2, int(seconds / max(t_iter, 1e-3))))
    cores = (time.process_time() - cpu0) / max(time.perf_counter() - wall0, 1e-9)
    need = oracle_iters_needed()
    rate = 1.0 / (t_iter * need)
    desc = (f"oracle full-lattice FP64 BiCGStab on one 16^3x32 Z2 source: {n_it} iterations timed "
            f"({t_iter:.2f} s each), scaled by the {need} iterations it needs for 1e-10")
    return rate, desc, round(cores, 1)


# ---------------------------------------------------------------------------
# our path
# ---------------------------------------------------------------------------
def run_step(ctx, dl, seed, noise0, params, store_loops):
    """One configuration's worth of the path: 64 noise vectors x 24 diluted sources."""
    w = WORKLOAD
    T = w["dims"][3]
    dil = dl.DIL_SPIN | dl.DIL_COLOUR | dl.DIL_EVENODD | dl.DIL_TIME
    K = 24
    n_solved = 0
    for c0 in range(0, w["n_noise"], CHUNK_NOISE):
        nn = min(CHUNK_NOISE, w["n_noise"] - c0)
        eta = ctx.make_sources(seed, noise0 + c0, nn, dil, t0=-1, out=store_loops["eta"][: nn * K])
        phi, st = ctx.solve(eta, params, x=store_loops["phi"][: nn * K])
        # each diluted source lives on the timeslice of its noise vector (n mod T)
        t_of = [(noise0 + c0 + j // K) % T for j in range(nn * K)]
        lo = ctx.trace_loops(eta, phi, dl.SINK_LOCAL | dl.SINK_SMEARED, smear=(w["smear_alpha"], w["smear_iter"]),
                             t_of_rhs=t_of, group=K)  # [nn][2 sinks][16][T]: one loop per noise vector
        store_loops["loops"].append(lo)
        n_solved += nn * K
    return n_solved


def hop_profile(spec: str):
    """Time the plain and the fused Wilson hop alone (used for ncu captures)."""
    import torch
    import paper_1012_5168_gb300 as dl
    import synthetic
    parts = spec.split(":")
    prec = {"f64": dl.PREC_F64, "f32": dl.PREC_F32, "bf16": dl.PREC_BF16}[parts[0]]
    n = int(parts[1])
    kind = int(parts[2]) if len(parts) > 2 else -1
    force_r = int(parts[3]) if len(parts) > 3 else 0
    force_b = int(parts[4]) if len(parts) > 4 else 0
    w = WORKLOAD
    ctx = dl.Context(w["dims"], t_bc=-1)
    ctx.load_gauge(synthetic.gauge_field(w["dims"], w["eps"], w["seed"]))
    ctx.set_kappa(w["kappa"])
    shape = ctx.tune_hop(prec, n, force_R=force_r, force_block=force_b, force_pf=kind)
    out = {"precision": parts[0], "n_rhs": n,
           "shapes": {name: dict(zip(("R", "block", "kind"), ctx.hop_shape(prec, n, cls)))
                      for cls, name in enumerate(("plain", "fused", "fused_bicg"))}}
    for fused, name in ((0, "plain"), (1, "fused"), (2, "fused_bicg")):
        ms, by = ctx.bench_hop(prec, n, fused, reps=5)
        out[name] = {"ms": round(ms, 5), "GB/s": round(by / ms / 1e6, 1)}
    torch.cuda.synchronize()
    print(json.dumps(out), flush=True)
    ctx.close()


def smear_profile(n: int):
    """Time the smearing of n fields on timeslice 0 (used for ncu captures); 3 repetitions."""
    import torch
    import paper_1012_5168_gb300 as dl
    ctx, U, w = _ctx(dl, "wilson_16x16x16x32")
    dil = dl.DIL_SPIN | dl.DIL_COLOUR | dl.DIL_EVENODD
    x = ctx.make_sources(seed=1, noise_first=0, n_noise=(n + 23) // 24, dilution=dil)[:n].contiguous()
    reps = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.apply_smear(x, 4.0, 50, t_range=(0, 1))
        torch.cuda.synchronize()
        reps.append((time.perf_counter() - t0) * 1e3)
    # per site and field and iteration: 6 directions x 4 spins x 9 complex multiply-adds (8 flops)
    flops = 2 * (w["dims"][0] * w["dims"][1] * w["dims"][2] // 2) * n * 50 * 6 * 4 * 9 * 8
    print(json.dumps({"fields": n, "ms": [round(r, 3) for r in reps], "ms_per_iteration": round(min(reps) / 50, 4),
                      "fp64_equivalent_tflops": round(flops / (min(reps) / 1e3) / 1e12, 3)}), flush=True)
    ctx.close()


def solve_profile(n: int):
    """Two mixed-precision solves of n time-diluted noise sources on 16^3x32 (batch n, FP32
    inner, tol 1e-10) with the defect-correction hop timing of the second (used for ncu
    captures: each solve launches the float-float hop for b_hat and twice per cycle)."""
    import torch
    import paper_1012_5168_gb300 as dl
    ctx, U, w = _ctx(dl, "wilson_16x16x16x32")
    dil = dl.DIL_SPIN | dl.DIL_COLOUR | dl.DIL_EVENODD | dl.DIL_TIME
    eta = ctx.make_sources(seed=3, noise_first=0, n_noise=(n + 23) // 24, dilution=dil)[:n].contiguous()
    params = dl.Params(tol=1e-10, precision=dl.PREC_F32, batch=n)
    out = {"rhs": n, "ms": []}
    for rep in range(2):
        ctx.set_timing(rep == 1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, st = ctx.solve(eta, params)
        torch.cuda.synchronize()
        out["ms"].append(round((time.perf_counter() - t0) * 1e3, 2))
    tim = ctx.get_timing(reset=True)
    n_oh = tim["hop_launches"][2] + tim["hop_launches"][3]
    out["outer"] = [s["outer"] for s in st][:4]
    out["defect_correction_hops"] = {"launches": int(n_oh), "ms_per_launch":
                                     round((tim["hop_ms"][2] + tim["hop_ms"][3]) / max(n_oh, 1), 4)}
    print(json.dumps(out), flush=True)
    ctx.close()


def _ctx(dl, name):
    import synthetic
    w = synthetic.WORKLOADS[name]
    U = synthetic.gauge_field(w["dims"], w["eps"], w["seed"])
    ctx = dl.Context(w["dims"], t_bc=-1)
    ctx.load_gauge(U)
    ctx.set_kappa(w["kappa"])
    return ctx, U, w


def workload_exact():
    """All 12V point sources on 4^4 (kappa 0.10, eps 0.3, tol 1e-12) vs the dense oracle inverse."""
    import numpy as np
    import torch
    import paper_1012_5168_gb300 as dl
    from oracle import loops
    ctx, U, w = _ctx(dl, "exact_4x4x4x4")
    V = int(np.prod(w["dims"]))
    out = {"workload": "exact_4x4x4x4", "point_sources": 12 * V}
    for name, prec in (("f64", dl.PREC_F64), ("f32", dl.PREC_F32)):
        p = dl.Params(tol=w["tol"], precision=prec, batch=64)
        ctx.exact_loops(0, 64, p)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lo, st = ctx.exact_loops(0, 12 * V, p)
        dt = time.perf_counter() - t0
        out[name] = {"seconds": round(dt, 4), "solves_per_s": round(12 * V / dt, 1), "max_true_residual": st["true_residual"]}
        if name == "f64":
            got = lo[0]
    t0 = time.perf_counter()
    ref = loops.exact_loops_dense(U, w["kappa"], -1.0)
    out["oracle_dense_seconds"] = round(time.perf_counter() - t0, 3)
    floor = 1e-6 * np.linalg.norm(ref[0])
    err = np.linalg.norm(got - ref, axis=-1) / np.maximum(np.linalg.norm(ref, axis=-1), floor)
    out["max_rel_error_per_gamma"] = float(err.max())
    print(json.dumps(out), flush=True)


def _hop_rate(tim, kinds):
    """(GB/s, ms per launch) of the hop launches of the given timing kinds."""
    ms = sum(tim["hop_ms"][k] for k in kinds)
    by = sum(tim["hop_bytes"][k] for k in kinds)
    n = sum(tim["hop_launches"][k] for k in kinds)
    return (by / (ms / 1e3) / 1e9 if ms > 0 else 0.0), (ms / n if n else 0.0)


def workload_single_rhs():
    """One right-hand side at a time on 16^3 x 32 to 1e-10: a point source and 8 Z2 sources (seeds
    1-8), plain FP64 vs FP32- and BF16-inner defect correction, at kappa 0.140 (eps 0.45) and at
    kappa 0.157 (eps 0.60); iterations, outer cycles and the hop bandwidth per precision."""
    import torch
    import paper_1012_5168_gb300 as dl
    peak, _ = read_peaks()
    out = {"workload": "single_rhs_16x16x16x32", "tol": 1e-10, "hbm_peak_gbs": peak, "lattices": {}}
    for name in ("wilson_16x16x16x32", "wilson_16x16x16x32_k157"):
        ctx, U, w = _ctx(dl, name)
        srcs = [ctx.make_point_sources(0, 1)] + [ctx.make_sources(s, 0, 1, 0) for s in range(1, 9)]
        res = {"kappa": w["kappa"], "eps": w["eps"]}
        for pname, prec in (("f64", dl.PREC_F64), ("f32", dl.PREC_F32), ("bf16", dl.PREC_BF16)):
            p = dl.Params(tol=w["tol"], precision=prec, batch=1)
            ctx.solve(srcs[1], p)  # tune and warm up
            ctx.set_timing(True)
            ctx.get_timing(reset=True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = [ctx.solve(b, p)[1][0] for b in srcs]
            torch.cuda.synchronize()
            dt = (time.perf_counter() - t0) / len(srcs)
            tim = ctx.get_timing(reset=True)
            ctx.set_timing(False)
            gbs, ms = _hop_rate(tim, (2, 3) if prec == dl.PREC_F64 else (0, 1))
            res[pname] = {"ms_per_solve": round(dt * 1e3, 2), "solves_per_s": round(1 / dt, 2),
                          "iters": [s["iters"] for s in st], "outer": [s["outer"] for s in st],
                          "max_true_residual": max(s["true_residual"] for s in st),
                          "inner_hop_gbs": round(gbs, 1), "inner_hop_frac_of_peak": round(gbs / peak, 3),
                          "inner_hop_ms": round(ms, 4)}
        out["lattices"][name] = res
        ctx.close()
    print(json.dumps(out), flush=True)


def workload_batch_scan():
    """Stochastic-loop solves on 16^3 x 32 (4 noise vectors x 24 diluted sources = 96 right-hand sides,
    FP32 inner to 1e-10) at batch widths N = 16, 32, 64, with and without CUDA graphs; solves/s and
    the bandwidth of the inner hops at each N."""
    import torch
    import paper_1012_5168_gb300 as dl
    peak, _ = read_peaks()
    ctx, U, w = _ctx(dl, "wilson_16x16x16x32")
    dil = dl.DIL_SPIN | dl.DIL_COLOUR | dl.DIL_EVENODD | dl.DIL_TIME
    eta = ctx.make_sources(seed=3, noise_first=0, n_noise=4, dilution=dil, t0=-1)
    out = {"workload": "batch_scan_16x16x16x32", "rhs": int(eta.shape[0]), "hbm_peak_gbs": peak, "runs": []}
    for N in (16, 32, 64):
        shape = ctx.tune_hop(dl.PREC_F32, N)  # (R, block, kernel kind, ms of one plain + one fused hop)
        for graph in (1, 0):
            p = dl.Params(tol=w["tol"], precision=dl.PREC_F32, batch=N, use_graph=graph)
            ctx.solve(eta[:N], p)  # capture graphs
            ctx.set_timing(True)
            ctx.get_timing(reset=True)
            torch.cuda.synchronize()
            clocks = ClockSampler(torch.cuda.current_device())
            t0 = time.perf_counter()
            _, st = ctx.solve(eta, p)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            clk = clocks.stop()
            tim = ctx.get_timing(reset=True)
            ctx.set_timing(False)
            plain, ms_p = _hop_rate(tim, (0,))
            fused, ms_f = _hop_rate(tim, (1,))
            out["runs"].append({"batch": N, "graph": bool(graph), "solves_per_s": round(eta.shape[0] / dt, 1),
                                "mean_iters": round(sum(s["iters"] for s in st) / len(st), 1),
                                "plain_hop_gbs": round(plain, 1), "fused_hop_gbs": round(fused, 1),
                                "fused_hop_frac_of_peak": round(fused / peak, 3),
                                "kernel_launches": tim["kernel_launches"], "clocks": clk,
                                "hop_shape": {"R": shape[0], "block": shape[1], "kind": shape[2],
                                              "tuned_ms": round(shape[3], 4)}})
    print(json.dumps(out), flush=True)


def workload_tsm():
    """TSM on 8^3 x 16 (500 LP + 50 HP noise vectors, HP: FP32-inner to 1e-10) vs the exact loops
    from all 12V point sources; spin x colour dilution, time dilution t0 = n mod T.  Two
    low-precision maps: single-precision CG on the normal equations to 1e-6 (Sec. 2's choice)
    and 30 fixed BF16 BiCGStab iterations."""
    import numpy as np
    import torch
    import paper_1012_5168_gb300 as dl
    ctx, U, w = _ctx(dl, "tsm_8x8x8x16")
    V = int(np.prod(w["dims"]))
    T = w["dims"][3]
    t0 = time.perf_counter()
    exact, st = ctx.exact_loops(0, 12 * V, dl.Params(tol=1e-10, precision=dl.PREC_F32, batch=64))
    t_exact = time.perf_counter() - t0
    exact = exact[0]  # [16][T]
    dil = dl.DIL_SPIN | dl.DIL_COLOUR | dl.DIL_TIME
    hp = dl.Params(tol=1e-10, precision=dl.PREC_F32, batch=64)
    names = dl.GAMMA_NAMES
    out = {"workload": "tsm_8x8x8x16", "exact_point_solves": 12 * V, "exact_seconds": round(t_exact, 2),
           "exact_max_true_residual": st["true_residual"], "n_lp": 500, "n_hp": 50,
           "dilution": "spin*colour*time", "lp_maps": {}}
    lps = {"f32_cgnr_tol1e-6": dl.Params(tol=1e-6, delta=1e-6, precision=dl.PREC_F32, batch=64,
                                         method=dl.METHOD_CGNR),
           "bf16_bicgstab_30_iterations": dl.Params(precision=dl.PREC_BF16, fixed_iters=30, batch=64)}
    cover = np.array([[(i % T) == t for t in range(T)] for i in range(500)])
    for label, lp in lps.items():
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mean, var, pn = ctx.tsm_estimate(1, 500, 50, dil, -1, lp, hp, dl.SINK_LOCAL, per_noise=True)
        torch.cuda.synchronize()
        t_tsm = time.perf_counter() - t0
        mean, var = mean[0], var[0]
        sig = np.sqrt(np.maximum(var.real + var.imag, 1e-300))
        z = np.abs(mean - exact) / sig  # per Gamma and timeslice
        lp_only = pn[:500, 0]
        lp_mean = (lp_only * cover[:, None, :]).sum(0) / cover.sum(0)
        out["lp_maps"][label] = {
            "tsm_seconds": round(t_tsm, 2), "z_median": float(np.median(z)), "z_max": float(z.max()),
            "per_gamma": {names[g]: {"exact_sum_t": [float(exact[g].sum().real), float(exact[g].sum().imag)],
                                     "tsm_sum_t": [float(mean[g].sum().real), float(mean[g].sum().imag)],
                                     "stderr_per_t": float(np.median(sig[g])),
                                     "lp_bias_per_t": float(np.median(np.abs(lp_mean[g] - exact[g])))}
                          for g in range(16)}}
    print(json.dumps(out), flush=True)


def workload_mixed():
    """Batches whose right-hand sides stop at different iterations, on 16^3 x 32 (kappa 0.157, eps 0.60:
    the kappa-literal variant), FP32 inner to 1e-10, width 32: (a) 16 point sources and 16 complex Z2
    sources; (b) a ragged last batch of 17 Z2 sources, whose 15 padding columns never take part.  The
    direct Wilson-hop kernels skip the loads and stores of right-hand sides that have stopped;
    DLOOPS_HOP_SKIP=0 keeps them streaming.  Reported: iterations and the solve time both ways (each
    the best of three, after a warm-up solve)."""
    import numpy as np
    import torch
    import paper_1012_5168_gb300 as dl
    import synthetic
    w = synthetic.WORKLOADS["wilson_16x16x16x32_k157"]
    U = synthetic.gauge_field(w["dims"], w["eps"], w["seed"])
    out = {"workload": "mixed_16x16x16x32", "kappa": w["kappa"], "eps": w["eps"], "batch": 32, "cases": {}}
    for case in ("point_and_z2", "ragged_17_of_32"):
        runs = {}
        for skip in ("1", "0"):
            os.environ["DLOOPS_HOP_SKIP"] = skip
            ctx = dl.Context(w["dims"], t_bc=-1)
            ctx.load_gauge(U)
            ctx.set_kappa(w["kappa"])
            V = int(np.prod(w["dims"]))
            if case == "point_and_z2":
                b = torch.cat([ctx.make_point_sources(12 * (V // 3), 16),
                               ctx.make_sources(seed=5, noise_first=0, n_noise=16, dilution=0)]).contiguous()
            else:  # a last batch of 17 sources: 15 padding columns of the width-32 layout never run
                b = ctx.make_sources(seed=5, noise_first=0, n_noise=17, dilution=0)
            p = dl.Params(tol=1e-10, precision=dl.PREC_F32, batch=32)
            ctx.solve(b, p)
            times = []
            for _ in range(3):
                torch.cuda.synchronize()
                clocks = ClockSampler(torch.cuda.current_device())
                t0 = time.perf_counter()
                _, st = ctx.solve(b, p)
                torch.cuda.synchronize()
                times.append((time.perf_counter() - t0, clocks.stop()))
            best = min(times, key=lambda x: x[0])
            runs["skip" if skip == "1" else "no_skip"] = {
                "seconds": round(best[0], 4), "clocks": best[1], "iters": [s["iters"] for s in st],
                "outer": sorted(set(s["outer"] for s in st)),
                "max_true_residual": max(s["true_residual"] for s in st)}
            ctx.close()
        os.environ.pop("DLOOPS_HOP_SKIP", None)
        runs["speedup"] = round(runs["no_skip"]["seconds"] / runs["skip"]["seconds"], 3)
        out["cases"][case] = runs
    print(json.dumps(out), flush=True)


def workload_clover():
    """The clover-improved operator M = A - kappa D against the Wilson matrix on the benchmark lattice
    (16^3 x 32, eps 0.45 links), kappa 0.13, c_sw 1.0: 32 time-diluted complex Z2 sources, FP32 inner
    solve with FP64 defect correction to 1e-10, width 32.  Each operator: a warm-up solve, then the best
    of three timed solves, the iterations, and the inner hops' CUDA-event timing (the clover hops also
    stream A^-1 of every output site: 576 B in FP32)."""
    import torch
    import paper_1012_5168_gb300 as dl
    import synthetic
    w = synthetic.WORKLOADS["wilson_16x16x16x32"]
    U = synthetic.gauge_field(w["dims"], w["eps"], w["seed"])
    peak, src = read_peaks()
    kappa, csw = 0.13, 1.0
    out = {"workload": "clover_16x16x16x32", "kappa": kappa, "c_sw": csw, "eps": w["eps"], "batch": 32,
           "tol": 1e-10, "runs": {}}
    for name, c_sw in (("wilson", 0.0), ("clover", csw)):
        ctx = dl.Context(w["dims"], t_bc=-1)
        ctx.load_gauge(U)
        ctx.set_kappa(kappa)
        ctx.set_clover(c_sw)
        b = ctx.make_sources(seed=9, noise_first=0, n_noise=32, dilution=dl.DIL_TIME, t0=-1)
        p = dl.Params(tol=1e-10, precision=dl.PREC_F32, batch=32)
        ctx.solve(b, p)
        ctx.set_timing(True)
        times = []
        for _ in range(3):
            ctx.get_timing(reset=True)
            torch.cuda.synchronize()
            clocks = ClockSampler(torch.cuda.current_device())
            t0 = time.perf_counter()
            _, st = ctx.solve(b, p)
            torch.cuda.synchronize()
            times.append((time.perf_counter() - t0, clocks.stop(), ctx.get_timing(), st))
        el, clk, tim, st = min(times, key=lambda x: x[0])
        fused_ms = tim["hop_ms"][1] / max(1, tim["hop_launches"][1])
        fused_gbs = tim["hop_bytes"][1] / max(1e-30, tim["hop_ms"][1] * 1e-3) / 1e9
        out["runs"][name] = {
            "seconds": round(el, 4), "solves_per_s": round(len(st) / el, 2), "clocks": clk,
            "iters_max": max(s["iters"] for s in st), "iters_mean": round(sum(s["iters"] for s in st) / len(st), 1),
            "outer": sorted(set(s["outer"] for s in st)), "max_true_residual": max(s["true_residual"] for s in st),
            "status": sorted(set(s["status"] for s in st)),
            "inner_fused_hop": {"ms_per_launch": round(fused_ms, 5), "GB/s": round(fused_gbs, 1),
                                "frac_of_hbm_peak": round(fused_gbs / peak, 4), "peak_source": src + " hbm_gbs"}}
        ctx.close()
    r = out["runs"]
    out["clover_cost_per_iteration"] = round((r["clover"]["seconds"] / r["clover"]["iters_max"]) /
                                             (r["wilson"]["seconds"] / r["wilson"]["iters_max"]), 3)
    print(json.dumps(out), flush=True)


def workload_tsm_paper():
    """The truncated solver method at the paper's sizes (Sec. 2): 5000 low-precision solves
    (single-precision CG on the normal equations, tolerance 1e-6) and 500 high-precision corrections
    (FP32 inner with FP64 defect correction, 1e-10) on 16^3 x 32, complex Z2 noise, time dilution by
    translation (t0 = n mod T; the paper states no dilution for this ensemble).  No exact loops exist
    at this volume (12V = 1.57 million solves), so the report is the estimate per Gamma with its
    error, the share of the variance from the low-precision ensemble and from the correction, and
    the bias the correction removed (<L_HP - L_LP> against its error)."""
    import numpy as np
    import torch
    import paper_1012_5168_gb300 as dl
    ctx, U, w = _ctx(dl, "wilson_16x16x16x32")
    T = w["dims"][3]
    n_lp, n_hp = 5000, 500
    lp = dl.Params(tol=1e-6, delta=1e-6, precision=dl.PREC_F32, batch=32, method=dl.METHOD_CGNR)
    hp = dl.Params(tol=1e-10, precision=dl.PREC_F32, batch=32)
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    t0 = time.perf_counter()
    mean, var, pn = ctx.tsm_estimate(1, n_lp, n_hp, dl.DIL_TIME, -1, lp, hp, dl.SINK_LOCAL, per_noise=True)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    clk = clocks.stop()
    mean, var = mean[0], var[0]
    lp_l, hp_l, lph_l = pn[:n_lp, 0], pn[n_lp:n_lp + n_hp, 0], pn[n_lp + n_hp:, 0]
    cover_lp = np.array([[(i % T) == t for t in range(T)] for i in range(n_lp)])
    cover_hp = np.array([[((n_lp + i) % T) == t for t in range(T)] for i in range(n_hp)])

    def mv(a, cov):
        cnt = cov.sum(0)
        m = (a * cov[:, None, :]).sum(0) / cnt
        d = (a - m[None]) * cov[:, None, :]
        return m, (np.abs(d) ** 2).sum(0) / (cnt - 1) / cnt

    m_lp, v_lp = mv(lp_l, cover_lp)
    m_d, v_d = mv(hp_l - lph_l, cover_hp)
    names = dl.GAMMA_NAMES
    out = {"workload": "tsm_16x16x16x32", "n_lp": n_lp, "n_hp": n_hp, "dilution": "time",
           "lp": "FP32 CGNR to 1e-6", "hp": "FP32 inner + FP64 defect correction to 1e-10",
           "seconds": round(el, 2), "solves": n_lp + 2 * n_hp,
           "solves_per_s": round((n_lp + 2 * n_hp) / el, 1), "clocks": clk, "per_gamma": {}}
    for g in range(16):
        err = float(np.sqrt((var[g].real + var[g].imag).mean()))
        out["per_gamma"][names[g]] = {
            "estimate_sum_t": [float(mean[g].sum().real), float(mean[g].sum().imag)],
            "error_per_t": err,
            "lp_variance_share": float((v_lp[g].real + v_lp[g].imag).sum() / max((var[g].real + var[g].imag).sum(), 1e-300)),
            "correction_per_t": float(np.abs(m_d[g]).mean()),
            "correction_error_per_t": float(np.sqrt(v_d[g].mean()))}
    print(json.dumps(out), flush=True)


def workload_correlators():
    """Sec. 3 two-point functions on 16^3 x 32 (kappa 0.140): the connected pion from one point source
    (12 solves) and the disconnected function of 16 spin x colour x even-odd diluted noise vectors
    (384 solves, all timeslices) at the 7 momenta 0, +-e_x, +-e_y, +-e_z; ratio D/C_pi (Eq. 4)."""
    import numpy as np
    import torch
    import paper_1012_5168_gb300 as dl
    ctx, U, w = _ctx(dl, "wilson_16x16x16x32")
    T = w["dims"][3]
    moms = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
    p = dl.Params(tol=w["tol"], precision=dl.PREC_F32, batch=32)
    out = {"workload": "correlators_16x16x16x32", "momenta": moms}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    prop, st = ctx.solve(ctx.make_point_sources(0, 12), p)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    C = ctx.meson_correlators(prop, (0, 0, 0, 0), moms)
    t2 = time.perf_counter()
    n_noise = 16
    dil = dl.DIL_SPIN | dl.DIL_COLOUR | dl.DIL_EVENODD
    eta = ctx.make_sources(seed=7, noise_first=0, n_noise=n_noise, dilution=dil)
    K = eta.shape[0] // n_noise
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    phi, _ = ctx.solve(eta, p)
    torch.cuda.synchronize()
    t4 = time.perf_counter()
    L = ctx.trace_loops_mom(eta, phi, moms, dl.SINK_LOCAL, group=K)[:, 0]  # [n_noise][Q][16][T]
    t5 = time.perf_counter()
    D = ctx.disconnected(L, moms)
    t6 = time.perf_counter()
    pion, dg5 = C[0, 5, 5], D[0, 5, 5]
    out.update({
        "point_solves_s": round(t1 - t0, 3), "meson_contraction_s": round(t2 - t1, 4),
        "noise_solves": int(eta.shape[0]), "noise_solve_s": round(t4 - t3, 3),
        "momentum_loops_s": round(t5 - t4, 4), "disconnected_s": round(t6 - t5, 4),
        "pion_t0_4": [float(v) for v in pion.real[:5]],
        "pion_p1_t0_4": [float(v) for v in C[1, 5, 5].real[:5]],
        "D_g5g5_t0_4": [float(v) for v in dg5.real[:5]],
        "ratio_D_over_Cpi_t0_4": [float(v) for v in (dg5.real / pion.real)[:5]],
    })
    print(json.dumps(out), flush=True)


def workload_dilution():
    """Stochastic error per inversion for each dilution scheme (the study of Sec. 3, Figs. 3-4, without
    the gauge-noise line, which needs an ensemble).  8^3 x 16 (kappa 0.140, eps 0.45), time dilution by
    translation in every scheme, exact loops from all 12V point sources as the reference.  The library
    (dl_dilution_error) solves each noise vector's K diluted sources, forms its loop estimate on the
    source timeslice t0 = n mod T and returns sigma^2, the mean squared deviation of those estimates from
    the exact loops; an estimate that costs N_inv inversions has the error sqrt(sigma^2 K / N_inv).
    Reported per Gamma: sqrt(sigma^2 K), the error per unit inversion, with clocks per scheme."""
    import numpy as np
    import torch
    import paper_1012_5168_gb300 as dl
    ctx, U, w = _ctx(dl, "tsm_8x8x8x16")
    V = int(np.prod(w["dims"]))
    p = dl.Params(tol=1e-10, precision=dl.PREC_F32, batch=64)
    t0 = time.perf_counter()
    exact, _ = ctx.exact_loops(0, 12 * V, p)
    exact = exact[0]  # [16][T]
    S, C, E, Q, TD = dl.DIL_SPIN, dl.DIL_COLOUR, dl.DIL_EVENODD, dl.DIL_CUBIC, dl.DIL_TIME
    schemes = {"time": TD, "spin": S | TD, "colour": C | TD, "evenodd": E | TD, "cubic": Q | TD,
               "spin_colour": S | C | TD, "spin_colour_evenodd": S | C | E | TD, "spin_colour_cubic": S | C | Q | TD}
    names = dl.GAMMA_NAMES
    out = {"workload": "dilution_8x8x8x16", "exact_seconds": round(time.perf_counter() - t0, 2),
           "inversions_per_scheme": 3072, "exact_rms_per_gamma": {names[g]: float(np.sqrt((np.abs(exact[g]) ** 2)
                                                                                      .mean())) for g in range(16)},
           "schemes": {}}
    for label, dil in schemes.items():
        K = dl.n_classes(dil)
        n_noise = max(16, 3072 // K)
        torch.cuda.synchronize()
        clocks = ClockSampler(torch.cuda.current_device())
        t1 = time.perf_counter()
        sigma2 = ctx.dilution_error(11, n_noise, dil, -1, p, exact)
        el = time.perf_counter() - t1
        out["schemes"][label] = {
            "classes": K, "noise_vectors": n_noise, "seconds": round(el, 3), "clocks": clocks.stop(),
            "error_per_unit_inversion": {names[g]: float(np.sqrt(sigma2[g] * K)) for g in range(16)}}
    print(json.dumps(out), flush=True)


def workload_autograd():
    """d/dkappa Tr[g5 M^-1] and grad wrt the Z2 sources through LoopTrace, 32 right-hand sides,
    on 8^3 x 16 and 16^3 x 32; FP64 central finite difference dkappa = 1e-5 as the check."""
    import torch
    import paper_1012_5168_gb300 as dl
    from paper_1012_5168_gb300.autograd import loop_trace
    res = {"workload": "autograd"}
    for name in ("tsm_8x8x8x16", "wilson_16x16x16x32"):
        ctx, U, w = _ctx(dl, name)
        params = dl.Params(tol=1e-12, precision=dl.PREC_F32, batch=32)
        eta = ctx.make_sources(seed=3, noise_first=0, n_noise=32, dilution=0).requires_grad_(True)
        k = torch.tensor(w["kappa"], dtype=torch.float64, requires_grad=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        L = loop_trace(eta, k, ctx, params)
        torch.cuda.synchronize()
        t_fwd = time.perf_counter() - t0
        loss = L[:, 5].real.sum()
        t0 = time.perf_counter()
        loss.backward()
        torch.cuda.synchronize()
        t_bwd = time.perf_counter() - t0
        dk = 1e-5
        with torch.no_grad():
            lp = loop_trace(eta.detach(), torch.tensor(w["kappa"] + dk, dtype=torch.float64), ctx, params)[:, 5].real.sum()
            lm = loop_trace(eta.detach(), torch.tensor(w["kappa"] - dk, dtype=torch.float64), ctx, params)[:, 5].real.sum()
        fd = (lp - lm).item() / (2 * dk)
        # directional derivative along a random source perturbation
        d = torch.randn_like(eta.detach())
        h = 1e-6
        with torch.no_grad():
            fp = loop_trace(eta.detach() + h * d, k.detach(), ctx, params)[:, 5].real.sum()
            fm = loop_trace(eta.detach() - h * d, k.detach(), ctx, params)[:, 5].real.sum()
        fd_eta = (fp - fm).item() / (2 * h)
        an_eta = torch.sum((eta.grad.conj() * d).real).item()  # PyTorch: grad = 2 df/dconj(eta)
        res[name] = {"rhs": 32, "dloss_dkappa": k.grad.item(), "central_difference": fd,
                     "rel_diff_kappa": abs(k.grad.item() - fd) / abs(fd),
                     "directional_grad_eta": an_eta, "directional_fd_eta": fd_eta,
                     "rel_diff_eta": abs(an_eta - fd_eta) / abs(fd_eta),
                     "forward_s": round(t_fwd, 3), "backward_s": round(t_bwd, 3),
                     "backward_over_forward": round(t_bwd / t_fwd, 2)}
        ctx.close()
    print(json.dumps(res), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.hop_profile:
        return hop_profile(args.hop_profile)
    if args.smear_profile:
        return smear_profile(args.smear_profile)
    if args.solve_profile:
        return solve_profile(args.solve_profile)
    if args.workload != "stochastic":
        return {"exact_4x4x4x4": workload_exact, "single_rhs_16x16x16x32": workload_single_rhs,
                "tsm_8x8x8x16": workload_tsm, "autograd": workload_autograd,
                "correlators_16x16x16x32": workload_correlators,
                "dilution_8x8x8x16": workload_dilution, "tsm_16x16x16x32": workload_tsm_paper,
                "mixed_16x16x16x32": workload_mixed, "batch_scan_16x16x16x32": workload_batch_scan,
                "clover_16x16x16x32": workload_clover}[args.workload]()
    if args.impl == "reference":
        return reference_arm(args, rank, world)

    import numpy as np
    import torch
    import torch.distributed as tdist

    torch.cuda.set_device(local)
    if world > 1:
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_1012_5168_gb300 as dl
    import synthetic

    w = WORKLOAD_K157 if args.kappa_literal else WORKLOAD
    prec = dl.PREC_F32 if args.precision == "f32" else dl.PREC_BF16
    params = dl.Params(tol=w["tol"], precision=prec, batch=args.batch, use_graph=1)
    U = synthetic.gauge_field(w["dims"], w["eps"], w["seed"])
    ctx = dl.Context(w["dims"], t_bc=-1)
    ctx.load_gauge(U)
    ctx.set_kappa(w["kappa"])
    K = 24
    store = dict(eta=ctx.new_fields(CHUNK_NOISE * K), phi=ctx.new_fields(CHUNK_NOISE * K), loops=[])
    noise0 = rank * w["n_noise"]
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            tdist.barrier()

    def max_over_ranks(x):
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        return float(t.item())

    # ---- the hop's launch shape for this width (the tuner the solver would run), then warm-up
    # (captures the CUDA graphs with their timing events, fills caches)
    if args.hop_shape:
        for cls, spec in enumerate(args.hop_shape.split(",")):
            r_, b_, k_ = (int(v) for v in spec.split(":"))
            ctx.set_hop_shape(prec, args.batch, cls, r_, b_, k_)
    else:
        ctx.tune_hop(prec, args.batch)
    hop_shape = [ctx.hop_shape(prec, args.batch, cls) for cls in (0, 1, 2)]  # (R, block, kind) per class
    ctx.set_timing(True)
    for s in range(args.warmup):
        run_step(ctx, dl, 1000 + s, noise0, params, store)

    # ---- timed: inputs resident in HBM
    ctx.get_timing(reset=True)
    store["loops"] = []
    barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    solved = 0
    for s in range(args.steps):
        solved += run_step(ctx, dl, 1 + s, noise0, params, store)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1))
    tim = ctx.get_timing(reset=True)
    total_solved = solved * world
    value = total_solved / (ms / 1e3)

    # ---- end to end: gauge uploaded from host, loops read back, every step
    U_host = np.ascontiguousarray(U)
    barrier()
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    store["loops"] = []
    f0.record(stream)
    e2e_solved = 0
    for s in range(args.steps):
        ctx.load_gauge(U_host, check_unitarity=False)
        e2e_solved += run_step(ctx, dl, 1 + s, noise0, params, store)
    f1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms_e2e = max_over_ranks(f0.elapsed_time(f1))
    h2d = U_host.nbytes
    d2h = sum(a.nbytes for a in store["loops"]) // max(args.steps, 1) + 24 * (w["n_noise"] * K)

    # ---- plain single-right-hand-side FP64 solve rate (the comparison of the metric)
    eta1 = ctx.make_sources(5, 0, 1, 0)
    ctx.solve(eta1[:1], dl.Params(tol=w["tol"], precision=dl.PREC_F64, batch=1))
    torch.cuda.synchronize()
    n64 = 3
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    eta3 = ctx.make_sources(6, 0, n64, 0)
    ctx.get_timing(reset=True)
    g0.record(stream)
    _, st64 = ctx.solve(eta3, dl.Params(tol=w["tol"], precision=dl.PREC_F64, batch=1))
    g1.record(stream)
    torch.cuda.synchronize()
    fp64_rate = n64 / (g0.elapsed_time(g1) / 1e3)
    # the FP64 hop is bound by FP64 issue: compare its flop rate (1320 per site and RHS)
    # with the FMA rate measured on this GPU
    t64 = ctx.get_timing(reset=True)
    vh = int(np.prod(w["dims"])) // 2
    ms64 = t64["hop_ms"][2] + t64["hop_ms"][3]
    n_hop64 = t64["hop_launches"][2] + t64["hop_launches"][3]
    fma64, _ = dl.bench_fma(dl.PREC_F64)
    fma32, _ = dl.bench_fma(dl.PREC_F32)
    hop64_tflops = 1320.0 * vh * n_hop64 / (ms64 / 1e3) / 1e12 if ms64 > 0 else 0.0

    # ---- roofline of the dominant hop kernel (low precision, events over the timed region)
    peak, peak_src = read_peaks()
    kinds = ["low_plain", "low_fused", "f64_plain", "f64_fused"]
    dom = max(range(4), key=lambda k: tim["hop_ms"][k])
    per_launch_ms = tim["hop_ms"][dom] / max(tim["hop_launches"][dom], 1)
    per_launch_bytes = tim["hop_bytes"][dom] / max(tim["hop_launches"][dom], 1)
    achieved = per_launch_bytes / (per_launch_ms / 1e3) / 1e9
    def traffic_of(name, kind):  # name: plain, r0dot or bicg
        return read_traffic(name, kind) if args.batch == 32 and args.precision == "f32" else None

    def shape_desc(sh):
        return f"{HOP_KIND_NAMES.get(sh[2], sh[2])} ({sh[0]} right-hand side(s) per thread, block {sh[1]})"

    def class_info(k):  # kernel description, kind(s) and ncu traffic of timing class k
        if k == 0:
            return f"plain hop: {shape_desc(hop_shape[0])}", hop_shape[0][2], traffic_of("plain", hop_shape[0][2])
        if k == 1:
            t1, t2 = traffic_of("r0dot", hop_shape[1][2]), traffic_of("bicg", hop_shape[2][2])
            return (f"fused hops: <rhat, v> {shape_desc(hop_shape[1])}; five reductions {shape_desc(hop_shape[2])}",
                    [hop_shape[1][2], hop_shape[2][2]], (t1 + t2) / 2 if t1 and t2 else None)
        return "hop_kernel<double> (FP64)", 0, None

    dkernel, dkind, traffic = class_info(dom)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "kernel": f"{kinds[dom]} ({args.precision} storage, batch {args.batch}): {dkernel}",
                "hop_kind": dkind,
                "peak_source": f"{peak_src} hbm_gbs", "algorithmic_bytes_per_launch": per_launch_bytes,
                "launches": tim["hop_launches"][dom], "ms_per_launch": round(per_launch_ms, 5),
                "hop_share_of_step": round(sum(tim["hop_ms"]) / ms, 3) if ms > 0 else None}
    # the other low-precision hop class of the same steps (plain D_oe p and D_oe s, or the fused ones)
    other = 1 - dom if dom < 2 else None
    if other is not None and tim["hop_launches"][other] > 0:
        o_ms = tim["hop_ms"][other] / tim["hop_launches"][other]
        o_bytes = tim["hop_bytes"][other] / tim["hop_launches"][other]
        okernel, okind, otraffic = class_info(other)
        roofline["other_hop"] = {"class": kinds[other], "kernel": okernel, "hop_kind": okind,
                                 "ms_per_launch": round(o_ms, 5),
                                 "achieved": round(o_bytes / (o_ms / 1e3) / 1e9, 1),
                                 "frac": round(o_bytes / (o_ms / 1e3) / 1e9 / peak, 4),
                                 "algorithmic_bytes_per_launch": o_bytes, "traffic": otraffic}

    # defect-correction hops (b_hat, reconstruction, residual) of the timed steps
    n_oh = tim["hop_launches"][2] + tim["hop_launches"][3]
    outer_hop = {"arith": "fp64" if os.environ.get("DLOOPS_OUTER_DFF", "1").startswith("0") or w["tol"] < 1e-11
                 else "float-float", "launches": int(n_oh),
                 "ms_per_launch": round((tim["hop_ms"][2] + tim["hop_ms"][3]) / n_oh, 4) if n_oh else None,
                 "share_of_step": round((tim["hop_ms"][2] + tim["hop_ms"][3]) / ms, 4) if ms > 0 else None}

    line = {
        "metric": METRIC,
        "value": round(value, 2),
        "unit": "solves/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms / args.steps, 2),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if prec == dl.PREC_F32 else "bf16",
        "data": f"synthetic (seeded SU(3) links U=exp(i*{w['eps']}*H), plaquette "
                f"~{0.57 if w['eps'] == 0.45 else 0.37}; complex Z2 noise)",
        "config": {"workload": w["name"], "lattice": "16x16x16x32", "kappa": w["kappa"], "eps": w["eps"],
                   "noise_vectors_per_gpu": w["n_noise"], "rhs_per_gpu": w["n_noise"] * K,
                   "dilution": w["dilution"], "tol": w["tol"], "solver": "even-odd BiCGStab, "
                   f"{args.precision} inner + defect correction on FP64 fields, batch {args.batch}, CUDA graphs",
                   "sinks": "local + smeared(alpha=4, n=50)", "l2": "inputs larger than L2 (no flush)",
                   "parallelism": f"replicas x{world} (disjoint noise ranges)"},
        "loops_per_s": round(value / K, 3),
        "fp64_plain_single_rhs": {"solves_per_s": round(fp64_rate, 3),
                                  "iters": [s["iters"] for s in st64],
                                  "hop_roofline": {"bound": "alu", "achieved": round(hop64_tflops, 4),
                                                   "peak": round(fma64, 4), "unit": "TFLOP/s",
                                                   "frac": round(hop64_tflops / fma64, 4) if fma64 else None,
                                                   "peak_source": "measured FP64 FMA chains (dl_bench_fma)"}},
        "fma_peak_tflops": {"f64": round(fma64, 3), "f32": round(fma32, 2)},
        "speedup_vs_fp64_plain": round(value / world / fp64_rate, 2),
        "e2e": {"value": round(e2e_solved * world / (ms_e2e / 1e3), 2), "unit": "solves/s",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(tim["kernel_launches"]),
        "roofline": roofline,
        "defect_correction_hops": outer_hop,
        "clocks": clk,
    }
    # the oracle baseline's stored iteration count belongs to the default workload
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.kappa_literal:
        rate, desc, cores = oracle_sample(20.0)
        line["cpu_baseline"] = {"value": rate, "unit": "solves/s", "cores": cores, "kind": "oracle", "sample": desc}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        tdist.destroy_process_group()


def reference_arm(args, rank, world):
    """The FP64 CPU oracle, as it stands, on the same workload and metric."""
    if rank != 0:
        return
    steps = []
    desc, cores = "", 1
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        # warm-up steps: one iteration; timed steps: at least 5 whole iterations each
        timed = s >= args.warmup
        rate, desc, cores = oracle_sample(8.0, min_iters=5 if timed else 1)
        if timed:
            steps.append((rate, time.perf_counter() - t0))
    value = statistics.median(r for r, _ in steps)
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(1e3 * statistics.mean(t for _, t in steps), 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        "config": {"workload": WORKLOAD["name"], "lattice": "16x16x16x32", "kappa": WORKLOAD["kappa"],
                   "eps": WORKLOAD["eps"], "tol": WORKLOAD["tol"]},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
