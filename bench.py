#!/usr/bin/env python
"""Throughput of the LR-CCSD Jacobian-vector product sigma = A X on GB300.

One step = one complete sigma(X) (singles + doubles, one right-hand side) of the hot path:
the particle-particle ladder with <ab|ef>~ formed on the fly from the T1-dressed Cholesky
vectors, the ring / crossed, hole-hole and three-body terms, and the antisymmetrisers.
Workload: o=32 occupied, v=240 virtual spinors, naux=1200 Cholesky vectors (synthetic,
seeded; T1 = 0, first-order T2), the single-RHS sigma configuration.

Beside the headline (TF32 on the tensor cores) the line carries: sigma-vectors/s in every
precision mode, the batched sigma (9 RHS), the HBM-bound kernels against the copy bandwidth,
time-to-alpha (FP64 against mixed precision at o=10 v=40; mixed precision by both response
routes at o=32 v=240), the 21-RHS batch at o=40 v=320 and the o=56 v=480 workload with their
device memory, and the CPU oracle timed on the host cores.

  python bench.py [--gpus N --steps K --warmup W --prec tf32|3xtf32|bf16x3|fp32|fp64]
  python bench.py --impl reference     (the CPU oracle on a bounded sample)

Prints one JSON line (rank 0).  N > 1 (torchrun): independent replicas, one per GPU
(right-hand sides are independent problems), no data-path collective; timing is the max
over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "sigma-vectors/s and time-to-alpha(omega) vs FP64 GPU path at |dalpha|<1e-4 a.u."
WORKLOAD = "C2"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cclr", choices=["cclr", "reference"])
    ap.add_argument("--prec", default=os.environ.get("CCLR_BENCH_PREC", "tf32"))
    ap.add_argument("--config", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-ladder-chunks", type=int, default=2)
    ap.add_argument("--no-alpha", action="store_true")
    ap.add_argument("--alpha-config", default="C1")
    ap.add_argument("--alpha-scale", type=float, default=0.2)
    ap.add_argument("--batch-rhs", type=int, default=9)
    ap.add_argument("--no-alpha-large", action="store_true")
    ap.add_argument("--no-ablation", action="store_true")
    ap.add_argument("--no-precisions", action="store_true")
    ap.add_argument("--no-hbm", action="store_true")
    ap.add_argument("--no-c3", action="store_true")
    ap.add_argument("--no-c5", action="store_true")
    ap.add_argument("--no-ccsd", action="store_true")
    ap.add_argument("--ccsd-config", default="C2")
    ap.add_argument("--ccsd-prec", default="3xtf32")
    ap.add_argument("--ccsd-scale", type=float, default=0.01)
    ap.add_argument("--ccsd-fp64-check", action="store_true")
    ap.add_argument("--solve-large", default="",
                    help="only run a large mixed-precision solve and print its JSON: "
                         "'C3' (3 components x {0, +-0.02, +-0.0428, +-0.0656} = 21 systems in one block) "
                         "or 'C5' (zz at omega = 0 by both routes, alpha tolerance, 180 GB budget)")
    ap.add_argument("--solve-scale", type=float, default=0.0)
    ap.add_argument("--alpha-large-config", default="C2")
    ap.add_argument("--alpha-large-scale", type=float, default=0.05)
    return ap.parse_args()


def algorithmic(o, v, naux):
    """cMAC counts per sigma (one RHS) with packed pair indices (i<j, a<b, e<f)."""
    Po, Pv = o * (o - 1) // 2, v * (v - 1) // 2
    form = naux * Pv * v * v          # <ab|ef>~ for a<b, all (e, f)
    contr = Po * Pv * Pv              # sum_{e<f} <ab||ef>~ X_ij^ef
    ring = o ** 3 * v ** 3
    hh = 3 * Po * Po * Pv
    ovn = o * o * v * v * naux
    return {"ladder_cmac": form + contr, "form_cmac": form, "ring_cmac": ring,
            "total_cmac": form + contr + ring + hh + ovn, "n_unique": o * v + Po * Pv}


# DRAM bytes (read + write) per executed FLOP of the formation GEMM: one ncu capture of one
# formation launch of the workload (M = 28800 rows (b,f), N = 7680 complex columns (a,e),
# K = 1200: 1.793388 GB read + 1.740861 GB written for 8 M N K = 2.1234e12 FLOP).  With K =
# naux fixed, both the output writes and the per-band operand reads scale with M N, so the
# ratio carries over to every group of the same workload.
FORMATION_BYTES_PER_FLOP = (1.793388e9 + 1.740861e9) / (8 * 28800 * 7680 * 1200)


def formation_flops_executed(v, naux, ga):
    """Real FLOP the formation GEMMs execute per sigma with group size ga (rows (b,f) with
    b >= a0 for each group of ga a values)."""
    tot = 0
    for a0 in range(0, v - 1, ga):
        a1 = min(v, a0 + ga)
        tot += 8 * (v - a0) * v * (a1 - a0) * v * naux
    return tot


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def ladder_peak(prec):
    """Peak (TFLOP/s) of the unit the ladder runs on, and how it was obtained."""
    d, how = peaks()
    if prec in ("tf32", "3xtf32"):
        # tf32 dense is half the bf16 dense rate (1.1 vs 2.25 PFLOP/s nominal)
        return "tensor", d["bf16_tflops"] * (1.1 / 2.25), f"{how} bf16 x nominal tf32/bf16 ratio"
    if prec == "bf16x3":
        return "tensor", d["bf16_tflops"], f"{how} bf16"
    if prec == "fp32":
        # 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz
        return "alu", 152 * 128 * 2 * 2.07e9 / 1e12, "derived: SM count x FP32 lanes x max clock"
    # FP64: nominal per-GPU rate (no measured figure on this machine)
    return "alu", 1.25, "nominal FP64 rate"


def reduce_max(x: float) -> float:
    """Max over ranks (identity without a process group); NCCL needs a device tensor."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world: int, units_per_rank: int, ms_max: float) -> float:
    """Whole-job units/s for independent replicas: all ranks' units over the slowest rank's time."""
    return world * units_per_rank / (ms_max / 1e3)


class Clocks:
    """Sample SM clocks and throttle reasons with nvidia-smi while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        import statistics
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def host_cpu():
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for l in out.splitlines():
            if l.startswith("Model name"):
                model = l.split(":", 1)[1].strip()
    except Exception:
        pass
    return {"nproc": os.cpu_count(), "model": model}


class OracleTiming:
    """The oracle as it stands (oracle.sampled's whole-vector sigma: every term but the ladder
    vectorised, the ladder's <ab|ef>~ formed chunk by chunk of 8 a values from L~_vv), timed on
    the host cores.  T-dependent intermediates (first-order T2, dressed blocks, Wovvo, Wovoo) are
    set-up and excluded, as the library's init is; the X-dependent work is timed."""

    CHUNK = 8

    def __init__(self, cfg, seed):
        import torch
        from oracle import ccsd, sampled
        from oracle.integrals import as_t
        from paper_2604_12914_gb300.inputs import make_config
        s = make_config(cfg, seed=seed)
        self.cfg, self.o, self.v, self.naux = cfg, s.o, s.v, s.naux
        t0 = time.perf_counter()
        eps, L = as_t(s.eps), as_t(s.L)
        t2 = ccsd.first_order_t2_from_L(eps, L, s.o)
        self.E = sampled.EntrySigma(eps, L, torch.zeros(s.o, s.v, dtype=torch.complex128), t2)
        self.E.Wovvo_full()
        self.E.Wovoo_full()
        self.setup = time.perf_counter() - t0
        self.threads = torch.get_num_threads()
        self.nchunks = (s.v + self.CHUNK - 1) // self.CHUNK
        self.seed = seed
        self.t_rest = None
        self.k = 0

    def rest(self):
        """X-dependent work of one sigma except the ladder (seconds)."""
        from oracle.integrals import as_t
        from paper_2604_12914_gb300.inputs import random_amplitudes
        x1, x2 = map(as_t, random_amplitudes(self.o, self.v, seed=self.seed + 1000))
        t0 = time.perf_counter()
        self.E.set_x(x1, x2)
        _, self.s2 = self.E.sigma_rest()
        self.t_rest = time.perf_counter() - t0
        return self.t_rest

    def chunk(self):
        """One ladder chunk (the next of evenly spread a0 values), seconds."""
        a0 = ((self.k * 7) % self.nchunks) * self.CHUNK
        self.k += 1
        t0 = time.perf_counter()
        self.E.ladder_chunk(a0, min(self.v, a0 + self.CHUNK), self.s2)
        return time.perf_counter() - t0

    def sigma_time(self, chunk_times):
        return self.t_rest + self.nchunks * sum(chunk_times) / len(chunk_times)

    def describe(self, nchunks_timed):
        return (f"one sigma at {self.cfg} o={self.o} v={self.v} naux={self.naux}: oracle.sampled's X-dependent "
                f"work (set_x + sigma_rest, {self.t_rest:.1f} s, timed whole) plus {nchunks_timed} of the "
                f"{self.nchunks} ladder chunks of {self.CHUNK} a values (timed, scaled to all chunks); T-dependent "
                f"set-up ({self.setup:.1f} s) excluded")


def cpu_small(cfg="C1"):
    """The oracle's whole sigma at a small workload, all threads and one thread."""
    import torch
    from oracle import ccsd, sampled
    from oracle.integrals import as_t
    from paper_2604_12914_gb300.inputs import make_config, random_amplitudes
    s = make_config(cfg, seed=1)
    eps, L = as_t(s.eps), as_t(s.L)
    E = sampled.EntrySigma(eps, L, torch.zeros(s.o, s.v, dtype=torch.complex128),
                           ccsd.first_order_t2_from_L(eps, L, s.o))
    E.Wovvo_full()
    E.Wovoo_full()
    x1, x2 = map(as_t, random_amplitudes(s.o, s.v, seed=5))
    out = {"workload": f"{cfg} o={s.o} v={s.v} naux={s.naux}, whole sigma (oracle.sampled.sigma_blocked)"}
    nt = torch.get_num_threads()
    for label, threads in (("all_threads", nt), ("one_thread", 1)):
        torch.set_num_threads(threads)
        E.set_x(x1, x2)
        E.sigma_blocked()
        t0 = time.perf_counter()
        E.set_x(x1, x2)
        E.sigma_blocked()
        el = time.perf_counter() - t0
        out[label] = {"threads": threads, "seconds": el, "sigma_vectors_per_s": 1.0 / el}
    torch.set_num_threads(nt)
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2604_12914_gb300.inputs import CONFIGS
    c = CONFIGS[args.config]
    T = OracleTiming(args.config, 2)
    T.rest()
    times = []
    for k in range(args.warmup + args.steps):
        t = T.chunk()
        if k >= args.warmup:
            times.append(t)
    v = 1.0 / T.sigma_time(times)
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "sigma-vectors/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 / v, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "c128", "data": "synthetic (seeded; T1=0, first-order T2)",
           "config": {"workload": f"{args.config} o={c['o']} v={c['v']} naux={c['naux']} single-RHS sigma"},
           "cpu_baseline": {"value": v, "unit": "sigma-vectors/s", "cores": T.threads, "kind": "oracle",
                            "host": host_cpu(),
                            "sample": T.describe(args.steps) + "; each timed step is one ladder chunk"},
           "e2e": {"value": v, "unit": "sigma-vectors/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "gpu_launches": 0}
    print(json.dumps(out), flush=True)


def time_to_alpha(cfg, scale, prec_mixed, comps=(0, 1, 2), omegas=(0.0, 0.0428), tol=1e-6):
    """Wall time of cc_lr_solve (Lambda + X(+-w) solves + alpha), FP64 path vs mixed path,
    on the same synthetic system and to the same relative residual tol; returns both times
    and max |delta alpha| (a.u.)."""
    import numpy as np
    import torch
    from paper_2604_12914_gb300 import binding
    from paper_2604_12914_gb300.inputs import make_config
    s = make_config(cfg, scale=scale)
    out = {"workload": f"{cfg} o={s.o} v={s.v} naux={s.naux}, Cholesky vectors scaled by {scale}",
           "components": list(comps), "omegas": list(omegas), "tol": tol}
    res = {}
    for tag, prec in (("fp64", "fp64"), ("mixed", prec_mixed)):
        stream = torch.cuda.Stream()
        ctx = binding.Context(s.o, s.v, s.naux, s.eps, s.L, s.mu, prec=prec, stream=stream.cuda_stream)
        ctx.cc_lr_set_graphs(True)              # both arms replay repeated products from CUDA graphs
        if tag == "mixed":
            ctx.cc_lr_set_refinement("3xtf32")  # accurate products on the tensor cores too
        t0 = time.perf_counter()
        al, st = ctx.cc_lr_solve(list(omegas), comps, tol=tol, allow_noconv=True)
        el = time.perf_counter() - t0
        graphs = ctx.cc_lr_graph_stats()
        ctx.close()
        res[tag] = al
        out[tag] = {"seconds": el,
                    "precision_mode": prec if tag == "fp64" else f"{prec} corrections, 3xtf32 refinement",
                    "graph_captures_launches": list(graphs), "iterations": st["iterations"],
                    "sigma_calls": st["sigma_calls"], "fp64_refinements": st["refinements"],
                    "converged": st["converged"], "max_rel_residual": st["max_rel_residual"]}
    out["max_abs_delta_alpha_au"] = float(np.abs(res["fp64"] - res["mixed"]).max())
    out["alpha_zz_fp64"] = [float(res["fp64"][w, -1, -1].real) for w in range(len(omegas))]
    out["speedup_mixed_vs_fp64"] = out["fp64"]["seconds"] / out["mixed"]["seconds"]
    return out


def time_to_alpha_large(cfg, scale, comps=(2,), omegas=(0.0,), tol=1e-6):
    """Wall time of cc_lr_solve on the large workload with tensor-core arithmetic throughout
    the solve (TF32 corrections, 3xTF32 refinement residuals and F X stencils; FP64 vectors,
    Krylov subspace and alpha contractions), then alpha again by the left-hand route
    (cc_lr_solve_left): the two routes agree to the solves' accuracy, so |alpha_left -
    alpha_right| is an a-posteriori estimate of the error.  (One FP64 sigma at this size takes
    tens of seconds on this GPU; the FP64 path's solve is not run here.)"""
    import numpy as np
    from paper_2604_12914_gb300 import binding
    from paper_2604_12914_gb300.inputs import make_config
    s = make_config(cfg, scale=scale)
    t0 = time.perf_counter()
    ctx = binding.Context(s.o, s.v, s.naux, s.eps, s.L, s.mu, prec="tf32")
    ctx.cc_lr_set_refinement("3xtf32")
    t_init = time.perf_counter() - t0
    t0 = time.perf_counter()
    al, st = ctx.cc_lr_solve(list(omegas), comps, tol=tol, allow_noconv=True)
    el = time.perf_counter() - t0
    t0 = time.perf_counter()
    alL, stL = ctx.cc_lr_solve_left(list(omegas), comps, tol=tol, allow_noconv=True)
    elL = time.perf_counter() - t0
    mem = ctx.cc_lr_memory()
    ctx.close()
    return {"workload": f"{cfg} o={s.o} v={s.v} naux={s.naux}, Cholesky vectors scaled by {scale}",
            "components": list(comps), "omegas": list(omegas), "tol": tol,
            "precision_mode": "tf32 corrections, 3xtf32 refinement, fp64 vectors",
            "seconds": el, "init_seconds": t_init, "iterations": st["iterations"],
            "sigma_calls": st["sigma_calls"], "refinements": st["refinements"],
            "converged": st["converged"], "max_rel_residual": st["max_rel_residual"],
            "seconds_solve_lambda_alpha": [st["time_solve_ms"] / 1e3, st["time_lambda_ms"] / 1e3,
                                           st["time_alpha_ms"] / 1e3],
            "alpha": [[float(al[w, a, a].real) for a in range(len(comps))] for w in range(len(omegas))],
            "left_route": {"seconds": elL, "converged": stL["converged"],
                           "alpha": [[float(alL[w, a, a].real) for a in range(len(comps))] for w in range(len(omegas))],
                           "max_abs_left_minus_right_au": float(np.abs(alL - al).max())},
            "device_memory_peak_gb": mem[1] / 1e9}


def packed_batch(cfg, nrhs, precs, reps=2, budget=0):
    """sigma-vectors/s of an nrhs batch in the packed unique-amplitude layout at workload cfg
    (the FP64 state is released), with the context's device memory; budget > 0 runs the context
    under that HBM budget (every allocation charged and checked)."""
    import torch
    from paper_2604_12914_gb300 import binding
    from paper_2604_12914_gb300.inputs import make_config
    s = make_config(cfg)
    t0 = time.perf_counter()
    stream = torch.cuda.current_stream()
    ctx = binding.Context(s.o, s.v, s.naux, s.eps, s.L, s.mu, prec=precs[0], stream=stream.cuda_stream,
                          hbm_budget=int(budget))
    ctx.cc_lr_set_refinement("3xtf32")          # no FP64 product: its set is released
    out = {"workload": f"{cfg} o={s.o} v={s.v} naux={s.naux}, {nrhs} RHS per call in the packed layout "
                       "(split into as few batched products as the device memory allows: products_per_batch)",
           "init_seconds": time.perf_counter() - t0, "nrhs": nrhs, "budget_gb": budget / 1e9 if budget else None}
    del s
    g = torch.Generator(device="cuda")
    g.manual_seed(11)
    x = torch.randn(nrhs, ctx.n_packed(), dtype=torch.complex128, device="cuda", generator=g)
    y = torch.empty_like(x)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for p in precs:
        ctx.cc_lr_set_precision(p)
        ctx.sigma_packed(x, y, nrhs=nrhs)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            ctx.sigma_packed(x, y, nrhs=nrhs)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        tm = ctx.cc_lr_last_timings()
        out[p] = {"ms_per_batch": ms, "sigma_vectors_per_s": nrhs / (ms / 1e3),
                  "products_per_batch": int(tm[4]), "last_product_ladder_ms": float(tm[0]),
                  "last_product_formation_ms": float(tm[3]), "ladder_group_size": ctx.cc_lr_ladder_tuning(p)[0]}
    used, peak, _ = ctx.cc_lr_memory()
    out["device_memory_gb"] = {"held": used / 1e9, "peak": peak / 1e9,
                               "caller_vectors": 2 * x.numel() * 16 / 1e9}
    ctx.close()
    return out


def solve_large(cfg, scale):
    """A mixed-precision solve at a large workload (TF32 corrections, 3xTF32 refinement, FP64
    vectors) with its wall time, iterations and device memory: at o=40 v=320 the 21 systems of 3
    components x {0, +-0.02, +-0.0428, +-0.0656} in one block (every iteration applies the operator
    to all unconverged systems in batched products); at o=56 v=480 the zz component at omega = 0 to
    an absolute alpha tolerance of 1e-4 a.u. (left- and right-route alphas), under a 180 GB budget."""
    import numpy as np
    from paper_2604_12914_gb300 import binding
    from paper_2604_12914_gb300.inputs import make_config
    c5 = cfg == "C5"
    scale = scale or (0.035 if c5 else 0.045)
    s = make_config(cfg, scale=scale)
    budget = int(180e9) if c5 else 0
    t0 = time.perf_counter()
    ctx = binding.Context(s.o, s.v, s.naux, s.eps, s.L, s.mu, prec="tf32", hbm_budget=budget)
    out = {"workload": f"{cfg} o={s.o} v={s.v} naux={s.naux}, Cholesky vectors scaled by {scale}",
           "init_seconds": time.perf_counter() - t0, "budget_gb": budget / 1e9 if budget else None}
    del s
    ctx.cc_lr_set_refinement("3xtf32")
    t0 = time.perf_counter()
    if c5:
        ctx.cc_lr_set_solver("gmres", 20, 200)
        al, est, st = ctx.cc_lr_solve_alpha_tol([0.0], (2,), tol_alpha=1e-4, allow_noconv=True)
        out.update({"what": "alpha_zz(0) to |alpha_left - alpha_right| < 1e-4 a.u.",
                    "alpha_zz": [float(al[0, 0, 0].real), float(al[0, 0, 0].imag)], "estimate_au": est})
    else:
        ctx.cc_lr_set_solver("block", 20, 300)
        omegas = [0.0, 0.02, 0.0428, 0.0656]
        al, st = ctx.cc_lr_solve(omegas, (0, 1, 2), tol=1e-5, allow_noconv=True)
        out.update({"what": "3 components x 7 shifts = 21 systems in one block, relative residual 1e-5",
                    "alpha_diag": [[float(al[w, a, a].real) for a in range(3)] for w in range(len(omegas))],
                    "max_abs_imag_diag": float(np.abs(np.imag(np.diagonal(al, axis1=1, axis2=2))).max())})
    out["seconds"] = time.perf_counter() - t0
    out["stats"] = st
    used, peak, _ = ctx.cc_lr_memory()
    out["device_memory_gb"] = {"held": used / 1e9, "peak": peak / 1e9}
    ctx.close()
    return out


def ground_state(cfg, scale, prec, tol, fp64_check=False):
    """Ground-state CCSD on the device: Omega(T) = 0 from the first-order guess by quasi-Newton
    steps with DIIS, each residual from two intermediate builds and two sigma products (exact
    two-point Gauss-Legendre rule); wall time, residuals formed, energy, and (fp64_check) the FP64
    residual norm of the final amplitudes, an independent check that the mixed-precision solve met
    its tolerance (at o=32 v=240 that one FP64 residual takes over a minute on this GPU's FP64
    rate).  The Cholesky scale keeps the synthetic system weakly correlated enough for the
    first-order start: |Omega(T1st)| is about 500 at o=32 v=240 with s = 0.05."""
    import numpy as np
    from paper_2604_12914_gb300 import binding
    from paper_2604_12914_gb300.inputs import make_config
    s = make_config(cfg, scale=scale)
    t0 = time.perf_counter()
    ctx = binding.Context(s.o, s.v, s.naux, s.eps, s.L, s.mu, prec=prec)
    out = {"workload": f"{cfg} o={s.o} v={s.v} naux={s.naux}, Cholesky vectors scaled by {scale}",
           "init_seconds": time.perf_counter() - t0, "residual_products": prec, "tol": tol}
    t0 = time.perf_counter()
    e, rn, its = ctx.cc_lr_ccsd(tol=tol, max_iterations=80, allow_noconv=True)
    el = time.perf_counter() - t0
    out.update({"seconds": el, "residuals": its, "seconds_per_residual": el / max(its, 1),
                "residual_norm": rn, "converged": rn < tol, "energy": [e.real, e.imag]})
    # then the ground-state Lambda at the converged T (lambda A = -dE/dT): TF32 corrections with
    # 3xTF32 refinement residuals, relative residual 1e-6
    ctx.cc_lr_set_precision("tf32")
    ctx.cc_lr_set_refinement("3xtf32")
    t0 = time.perf_counter()
    try:
        ctx.cc_lr_lambda(tol=1e-6)
        out["lambda_seconds"] = time.perf_counter() - t0
        out["lambda_precision_mode"] = "tf32 corrections, 3xtf32 refinement, relative residual 1e-6"
    except binding.CclrError as err:
        out["lambda_error"] = str(err)
    if fp64_check:
        t1, t2 = ctx.cc_lr_get_t()
        t0 = time.perf_counter()
        r1, r2, e64 = ctx.cc_lr_ccsd_residual(t1, t2, prec="fp64")
        out["fp64_residual_seconds"] = time.perf_counter() - t0
        iu = np.triu_indices(s.o, 1)
        ju = np.triu_indices(s.v, 1)
        out["fp64_residual_norm"] = float(np.sqrt(np.sum(np.abs(r1) ** 2) +
                                                  np.sum(np.abs(r2[iu][:, ju[0], ju[1]]) ** 2)))
    used, peak, _ = ctx.cc_lr_memory()
    out["device_memory_peak_gb"] = peak / 1e9
    ctx.close()
    return out


def cublas_tf32_tflops():
    """cuBLAS TF32 GEMM 8192^3 (torch.matmul on FP32 with TF32 allowed), best of 5, CUDA events."""
    import torch
    n = 8192
    a = torch.randn(n, n, device="cuda")
    b = torch.randn(n, n, device="cuda")
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    best = 1e30
    for _ in range(6):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    torch.backends.cuda.matmul.allow_tf32 = prev
    del a, b
    torch.cuda.empty_cache()
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


def run_cclr(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cpu = None
    cpu_c1 = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # before any GPU call: the oracle on the host cores
        T = OracleTiming(args.config, 2)
        T.rest()
        ch = [T.chunk() for _ in range(max(1, args.cpu_ladder_chunks))]
        cpu = {"value": 1.0 / T.sigma_time(ch), "unit": "sigma-vectors/s", "cores": T.threads, "kind": "oracle",
               "host": host_cpu(), "sample": T.describe(len(ch)),
               "seconds_per_sigma": T.sigma_time(ch), "seconds_rest": T.t_rest, "seconds_per_ladder_chunk": ch}
        del T
        cpu_c1 = cpu_small("C1")

    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2604_12914_gb300 import binding
    from paper_2604_12914_gb300.inputs import make_config, random_amplitudes

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    s = make_config(args.config, seed=2)
    o, v, naux = s.o, s.v, s.naux
    stream = torch.cuda.current_stream()
    ctx = binding.Context(o, v, naux, s.eps, s.L, s.mu, prec=args.prec, stream=stream.cuda_stream)
    x1h, x2h = random_amplitudes(o, v, seed=3 + rank)
    x1 = torch.from_numpy(x1h).cuda()
    x2 = torch.from_numpy(x2h).cuda()
    s1 = torch.empty_like(x1)
    s2 = torch.empty_like(x2)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        ctx.sigma_into(x1, x2, s1, s2)
    barrier()
    n0 = binding.cc_lr_launch_count()
    lad, form = [], []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as ck:
        torch.cuda.profiler.start()       # profiler range = the timed region (ncu --profile-from-start off)
        e0.record(stream)
        for _ in range(args.steps):
            ctx.sigma_into(x1, x2, s1, s2)
            tm = ctx.cc_lr_last_timings()
            lad.append(float(tm[0]))
            form.append(float(tm[3]))
        e1.record(stream)
        barrier()
        torch.cuda.profiler.stop()
    ms = e0.elapsed_time(e1)
    launches = binding.cc_lr_launch_count() - n0
    ms_max = reduce_max(ms)
    value = replica_throughput(world, args.steps, ms_max)
    clk = ck.summary()

    # end to end through the public API with host buffers (pinned)
    x1p = torch.from_numpy(x1h).pin_memory()
    x2p = torch.from_numpy(x2h).pin_memory()
    s1p = torch.empty_like(x1p).pin_memory()
    s2p = torch.empty_like(x2p).pin_memory()
    for _ in range(max(1, args.warmup // 2)):
        ctx.sigma_into(x1p, x2p, s1p, s2p)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        ctx.sigma_into(x1p, x2p, s1p, s2p)
    e1.record(stream)
    barrier()
    e2e = replica_throughput(world, args.steps, reduce_max(e0.elapsed_time(e1)))
    bytes_io = (x1p.numel() + x2p.numel()) * 16
    del x1p, x2p, s1p, s2p

    # batched: several right-hand sides share each formed <ab||ef>~ block
    batched = None
    if args.batch_rhs > 1:
        nb = args.batch_rhs
        xb1h, xb2h = random_amplitudes(o, v, seed=50 + rank, nvec=nb)
        xb1 = torch.from_numpy(xb1h).cuda()
        xb2 = torch.from_numpy(xb2h).cuda()
        del xb2h
        sb1 = torch.empty_like(xb1)
        sb2 = torch.empty_like(xb2)
        ctx.sigma_into(xb1, xb2, sb1, sb2, nrhs=nb)
        barrier()
        e0.record(stream)
        reps = max(1, args.steps // 3)
        lad_b = []
        for _ in range(reps):
            ctx.sigma_into(xb1, xb2, sb1, sb2, nrhs=nb)
            lad_b.append(float(ctx.cc_lr_last_timings()[0]))
        e1.record(stream)
        barrier()
        msb = reduce_max(e0.elapsed_time(e1)) / reps
        batched = {"nrhs": nb, "sigma_vectors_per_s": replica_throughput(world, nb, msb), "ms_per_batch": msb,
                   "ladder_ms_per_batch": sum(lad_b) / len(lad_b)}
        del xb1, xb2, sb1, sb2

    ablation = None
    if args.prec in ("tf32", "3xtf32") and not args.no_ablation:
        # ablation: the packed <ab||ef>~ kept in HBM after the first product (no re-formation)
        ctx.cc_lr_set_ladder_storage(True)
        for _ in range(2):
            ctx.sigma_into(x1, x2, s1, s2)
        barrier()
        lad_s = []
        e0.record(stream)
        for _ in range(args.steps):
            ctx.sigma_into(x1, x2, s1, s2)
            lad_s.append(float(ctx.cc_lr_last_timings()[0]))
        e1.record(stream)
        barrier()
        ms_s = reduce_max(e0.elapsed_time(e1)) / args.steps
        Pv = v * (v - 1) // 2
        ablation = {"what": "stored packed <ab||ef>~ (P_v x P_v kept in HBM; deviates from on-the-fly formation)",
                    "sigma_vectors_per_s": replica_throughput(world, args.steps, ms_s * args.steps),
                    "ms_per_step": ms_s, "ladder_ms": sum(lad_s) / len(lad_s),
                    "stored_gb": Pv * Pv * 8 * (3 if args.prec == "3xtf32" else 1) / 1e9}
        ctx.cc_lr_set_ladder_storage(False)

    alg = algorithmic(o, v, naux)
    lad_ms = sum(lad) / len(lad)
    form_ms = sum(form) / len(form)
    tga = ctx.cc_lr_ladder_tuning(args.prec)[0] if args.prec in ("tf32", "3xtf32", "bf16x3") else None

    # every precision mode on the same workload and context
    precisions = None
    if not args.no_precisions:
        precisions = {}
        for p in ("3xtf32", "bf16x3", "fp32", "fp64"):
            if p == args.prec:
                continue
            ctx.cc_lr_set_precision(p)
            ctx.sigma_into(x1, x2, s1, s2)
            barrier()
            k = 1 if p == "fp64" else 3
            lp = []
            e0.record(stream)
            for _ in range(k):
                ctx.sigma_into(x1, x2, s1, s2)
                lp.append(float(ctx.cc_lr_last_timings()[0]))
            e1.record(stream)
            barrier()
            msp = e0.elapsed_time(e1) / k
            bnd, pk, how = ladder_peak(p)
            precisions[p] = {"sigma_vectors_per_s": 1e3 / msp, "ms_per_sigma": msp, "ladder_ms": sum(lp) / len(lp),
                             "whole_sigma_rate_tflops": alg["total_cmac"] * 8 / (msp * 1e-3) / 1e12,
                             "unit_peak_tflops": pk, "unit": bnd, "peak_source": how, "steps": k}
        ctx.cc_lr_set_precision(args.prec)
    ctx.close()
    del x1, x2, s1, s2

    bound, peak, how = ladder_peak(args.prec)
    lad_achieved = alg["ladder_cmac"] * 8 / (lad_ms * 1e-3) / 1e12
    # the dominant kernel: the tensor-core GEMMs that form <ab|ef>~ (CUDA events around each)
    traffic = None
    if form_ms > 0:
        kernel = "tc_gemm_kernel: pp-ladder formation <ab|ef>~ = sum_P L~_ae L~_bf (all groups of one sigma)"
        achieved = alg["form_cmac"] * 8 / (form_ms * 1e-3) / 1e12
        if args.prec == "tf32" and tga:
            traffic = FORMATION_BYTES_PER_FLOP * formation_flops_executed(v, naux, tga)
    else:
        kernel = "pp-ladder (formation + contraction)"
        achieved = lad_achieved
    ms_step = ms_max / args.steps

    hbm = None
    if rank == 0 and not args.no_hbm:
        d, howp = peaks()
        hbm = {"peak_gbs": d["hbm_gbs"], "peak_source": f"{howp} copy bandwidth", "kernels": {}}
        # the complex128 vector kernels also do FP64 arithmetic, which this GPU runs at a nominal
        # 1.25 TFLOP/s: their FP64 flops per entry of a solver vector (o v + P_o P_v entries)
        nt = o * v + (o * (o - 1) // 2) * (v * (v - 1) // 2)
        fp64_flops = {"vec_precond": 10.0 * nt, "vec_dot": 8.0 * nt, "vec_axpy": 4.0 * nt}
        for k, (msk, byt) in binding.cc_lr_bench_hbm(o, v, reps=5).items():
            gbs = byt / (msk * 1e-3) / 1e9
            hbm["kernels"][k] = {"ms": msk, "algorithmic_gb": byt / 1e9, "achieved_gbs": gbs,
                                 "frac": gbs / d["hbm_gbs"]}
            if k in fp64_flops:
                tf = fp64_flops[k] / (msk * 1e-3) / 1e12
                hbm["kernels"][k].update({"fp64_tflops": tf, "fp64_frac_of_nominal_1.25": tf / 1.25})
    tf32_cublas = cublas_tf32_tflops() if rank == 0 else None

    def extra(fn, *a, **k):
        # a secondary measurement that fails is reported in the line instead of losing the line
        try:
            return fn(*a, **k)
        except Exception as e:  # noqa: BLE001
            return {"error": f"{type(e).__name__}: {e}"}

    tta = None
    tta_large = None
    if rank == 0 and not args.no_alpha:
        tta = extra(time_to_alpha, args.alpha_config, args.alpha_scale,
                    "tf32" if args.prec in ("tf32", "fp64") else args.prec)
        if not args.no_alpha_large:
            tta_large = extra(time_to_alpha_large, args.alpha_large_config, args.alpha_large_scale)
    c3 = c5 = None
    if rank == 0 and not args.no_c3:
        c3 = extra(packed_batch, "C3", 21, ["tf32", "3xtf32"])
    if rank == 0 and not args.no_c5:
        c5 = extra(packed_batch, "C5", 1, ["tf32", "bf16x3"], budget=180e9)
    gs = None
    if rank == 0 and not args.no_ccsd:
        gs = extra(ground_state, args.ccsd_config, args.ccsd_scale, args.ccsd_prec, 1e-5, args.ccsd_fp64_check)
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "sigma-vectors/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"tf32": "c64-tf32", "3xtf32": "c64-3xtf32", "bf16x3": "c64-bf16x3", "fp32": "c64",
                      "fp64": "c128"}[args.prec],
            "data": "synthetic (seeded; T1=0, first-order T2, random X)",
            "config": {"workload": f"{args.config} o={o} v={v} naux={naux} single-RHS sigma",
                       "precision_mode": args.prec, "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (X2 c128 %.2f GB, L~vv %.2f GB)" % (o * o * v * v * 16 / 1e9, naux * v * v * 16 / 1e9)},
            "roofline": {"kernel": kernel, "bound": bound,
                         "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "peak_source": how, "traffic": traffic,
                         "traffic_source": "ncu dram bytes per FLOP of one formation launch, scaled to the "
                                           "FLOP of one sigma's formation launches" if traffic else None,
                         "kernel_ms": form_ms if form_ms > 0 else lad_ms,
                         "ladder_ms": lad_ms, "ladder_share": lad_ms / ms_step,
                         "ladder_achieved": lad_achieved, "ladder_frac": lad_achieved / peak,
                         "whole_sigma_achieved": alg["total_cmac"] * 8 / (ms_step * 1e-3) / 1e12,
                         "whole_sigma_frac": alg["total_cmac"] * 8 / (ms_step * 1e-3) / 1e12 / peak,
                         "tf32_cublas_measured_tflops": tf32_cublas,
                         "frac_of_cublas_tf32": achieved / tf32_cublas if tf32_cublas else None},
            "clocks": clk,
            "e2e": {"value": e2e, "unit": "sigma-vectors/s", "h2d_bytes_per_step": bytes_io,
                    "d2h_bytes_per_step": bytes_io},
            "gpu_launches": int(launches),
        }
        if precisions is not None:
            out["precisions"] = precisions
        if hbm is not None:
            out["hbm_kernels"] = hbm
        if tta is not None:
            out["time_to_alpha"] = tta
        if tta_large is not None:
            out["time_to_alpha_large"] = tta_large
        if batched is not None:
            out["batched"] = batched
        if ablation is not None:
            out["ablation_stored_ladder"] = ablation
        if c3 is not None:
            out["c3_batched"] = c3
        if c5 is not None:
            out["c5"] = c5
        if gs is not None:
            out["ground_state_ccsd"] = gs
        if cpu is not None:
            out["cpu_baseline"] = cpu
            out["cpu_c1_whole_sigma"] = cpu_c1
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    a = parse()
    if a.solve_large:
        print(json.dumps({"solve_large": solve_large(a.solve_large, a.solve_scale)}), flush=True)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_cclr(a)
