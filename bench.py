#!/usr/bin/env python
"""Throughput of y = sgn(H_w(mu)) x: mixed-precision batched form vs plain FP64.

Workload (default): 16^3 x 32 lattice (N = 1,572,864), synthetic SU(3)
field U = exp(i eps X) with eps = 0.6 and seed 5, mu = 0.1, m_w = -1.5,
LR deflation of m = 100 critical eigenvectors (set-up timed separately),
Krylov dimension k = 250, 16 complex Gaussian right-hand sides of unit norm.
One step = one ovs_sign_apply of the 16 right-hand sides in the mixed form
(complex64 links, matvec and Krylov basis; FP64 Gram-Schmidt accumulation,
Hessenberg matrix, deflation coefficients and Newton sign). The same
application in plain FP64 with one right-hand side is timed beside it and
the mixed result of that right-hand side is checked against it (relative
2-norm <= 1e-6).

Prints one JSON line (rank 0). ``--impl reference`` times the CPU oracle on
a bounded sample of the same workload instead.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "sgn(H_w(μ))x applications/s at 1e-6 rel err, mixed+batched vs plain FP64"
UNIT = "applications/s"
DEFAULT = dict(dims=(16, 16, 16, 32), eps=0.6, seed=5, mu=0.1, m_w=-1.5, m=100, k=250, nrhs=16, src_seed=2,
               eig_tol=1e-6, setup_budget_s=150.0)
CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def parse_args():
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--dims", type=int, nargs=4, default=None)
    p.add_argument("--m", type=int, default=None)
    p.add_argument("--k", type=int, default=None)
    p.add_argument("--nrhs", type=int, default=None)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-long-ref", action="store_true", help="skip the FP64 k=790 reference of right-hand side 0")
    p.add_argument("--stencil-shape", type=int, nargs=3, default=None, metavar=("RT", "SITES", "RB"),
                   help="pin the stencil launch shape of the mixed form instead of autotuning it")
    p.add_argument("--workload", choices=["single", "batched", "overlap-solve"], default="single",
                   help="batched: the multi-instance recipe (32 instances of 4^4/6^4/8^4, m = 20 each, "
                        "per-vector convergence stop) in one ovs_sign_apply_batched call; its own JSON line")
    p.add_argument("--instances", type=int, default=32)
    p.add_argument("--batched-tol", type=float, default=1e-8, help="per-vector stop of the batched workload")
    p.add_argument("--batched-cap", type=int, default=600, help="Krylov cap of the batched workload")
    p.add_argument("--batched-every", type=int, default=10, help="check interval of the batched workload")
    p.add_argument("--batched-prec", choices=["mixed", "f64"], default="mixed")
    p.add_argument("--batched-every-check", action="store_true",
                   help="batched workload: check every interval instead of the skip-ahead schedule")
    p.add_argument("--full-application", action="store_true",
                   help="with --impl reference: time one complete oracle application instead of samples")
    p.add_argument("--no-variants", action="store_true",
                   help="skip the harmonic / D_ov / Schur sub-measurements of the default line")
    p.add_argument("--no-batched", action="store_true",
                   help="skip the batched multi-instance sub-measurement of the default line")
    return p.parse_args()


def workload(args):
    w = dict(DEFAULT)
    if args.dims:
        w["dims"] = tuple(args.dims)
    for key in ("m", "k", "nrhs"):
        if getattr(args, key) is not None:
            w[key] = getattr(args, key)
    w["V"] = w["dims"][0] * w["dims"][1] * w["dims"][2] * w["dims"][3]
    w["N"] = 12 * w["V"]
    d = w["dims"]
    w["name"] = (f"{d[0]}^3x{d[3]}" if d[0] == d[1] == d[2] else "x".join(map(str, d))) + \
        f" LR-deflated sgn(H_w(mu))x, m={w['m']}, k={w['k']}, {w['nrhs']} RHS, mixed+batched"
    return w


def config_of(w, world):
    return {
        "workload": w["name"],
        "lattice": list(w["dims"]), "N": w["N"], "gauge": f"U=exp(i eps X), eps={w['eps']}, seed={w['seed']}",
        "mu": w["mu"], "m_w": w["m_w"], "m_deflated": w["m"], "k": w["k"], "nrhs_per_gpu": w["nrhs"],
        "global_batch": w["nrhs"] * world,
        "precision": "complex64 links/matvec/Krylov basis; FP64 Gram-Schmidt accumulation, Hessenberg, "
                     "deflation coefficients, Newton sign",
        "l2": "inputs larger than L2: the Krylov basis streamed every step is "
              f"{w['nrhs'] * (w['k'] + 1) * w['N'] * 8 / 1e9:.1f} GB per GPU",
        "parallelism": f"replicas x{world} (independent right-hand-side batches)",
    }


# --------------------------------------------------------------- distributed
def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def dist_init(world, local, backend):
    import torch
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        if backend == "nccl":
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group("gloo")


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def job_value(nrhs_per_rank, steps, world, ms_max):
    """Whole-job applications/s: the right-hand sides all ranks processed in
    the timed steps over the slowest rank's time."""
    return nrhs_per_rank * steps * world / (ms_max / 1e3)


def max_over_ranks(value, world, device):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# -------------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={CLOCK_QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        power = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(power) if power else None}


# ------------------------------------------------------------- CPU baseline
class CpuSample:
    """The oracle on a bounded sample of one application, and its scaling.

    Sample: one right-hand side of the full lattice; the oracle's LR
    deflation with m random (biorthonormalised) vectors and its CGS2
    Arnoldi run for k_sample steps. The wall time of each Arnoldi step j
    (matvec plus the Gram-Schmidt passes over the j previous vectors, read
    off the times of successive matvec calls) is fitted as a + c j and summed
    to k steps; the projection before the first step is timed as it is; the
    Newton sign is timed on a k x k matrix; the recombination y = V_k c
    (one pass over V_k) is counted as a quarter of the Gram-Schmidt time of
    step k. The operator is built once (not timed).
    """

    def __init__(self, w, k_sample=16):
        import numpy as np

        import synth
        from oracle import lattice

        self.w, self.ks = w, k_sample
        links = synth.gauge_links(w["dims"], w["seed"], w["eps"])
        self.h = lattice.hw_operator(links, w["dims"], w["mu"], w["m_w"])
        n, m = w["N"], w["m"]
        rng = np.random.default_rng(1234)
        self.r = (rng.standard_normal((n, m)) + 1j * rng.standard_normal((n, m))) / np.sqrt(n) if m else None
        self.l = (rng.standard_normal((n, m)) + 1j * rng.standard_normal((n, m))) / np.sqrt(n) if m else None
        self.lam = rng.standard_normal(m) + 0.5j * rng.standard_normal(m) if m else None
        self.t_newton = None

    def newton_time(self):
        """Roberts' iteration on a k x k matrix with eigenvalues off the
        imaginary axis (the cost depends on k and the iteration count only)."""
        import numpy as np

        from oracle import newton
        if self.t_newton is None:
            k = self.w["k"]
            rng = np.random.default_rng(7)
            d = rng.uniform(0.05, 2.0, k) * rng.choice([-1.0, 1.0], k)
            a = np.triu(0.05 * (rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k))), -1)
            a[np.diag_indices(k)] = d
            t0 = time.perf_counter()
            newton.roberts_sign(a)
            self.t_newton = time.perf_counter() - t0
        return self.t_newton

    def run(self, seed_offset=0):
        """One sample. Returns (modelled seconds per application, measured
        seconds of the sample, description)."""
        import numpy as np

        import synth
        from oracle import deflation

        w, h, k, m = self.w, self.h, self.w["k"], self.w["m"]
        ks = max(3, min(self.ks, k))  # sampled steps: at most the workload's k, 3 for the fit
        x = synth.gaussian_vectors(w["N"], 1, w["src_seed"] + seed_offset)[0]
        stamps = []

        def mv(v):
            stamps.append(time.perf_counter())
            return h @ v

        t_start = time.perf_counter()
        deflation.lr_sign_apply(mv, x, self.r, self.l, self.lam, ks)
        t_sample = time.perf_counter() - t_start
        t_proj = stamps[0] - t_start
        steps = np.diff(np.asarray(stamps))  # step j (j = 0 .. ks-2) lasted steps[j]
        j = np.arange(len(steps))
        c, a = np.polyfit(j, steps, 1)
        c = max(c, 0.0)
        t_arnoldi = k * a + c * k * (k - 1) / 2
        t_recomb = 0.25 * c * k
        t_app = t_proj + t_arnoldi + self.newton_time() + t_recomb
        desc = (f"1 RHS of the full lattice: LR projection (m={m}) + {ks} of {k} CGS2 Arnoldi steps timed "
                f"({t_sample:.1f} s); the application's time MODELLED from it: step j lasts a + c j "
                f"(a={a:.3f} s, c={c:.2e} s, fitted), summed to k, plus the projection, a k x k Newton sign "
                f"({self.newton_time():.2f} s) and the recombination; numpy/scipy FP64")
        return t_app, t_sample, desc


def cpu_cores():
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(var):
            return int(os.environ[var])
    return os.cpu_count() or 1


# ------------------------------------------------------------------- ours
def run_ours(args, w, world, rank, local):
    import numpy as np
    import torch

    import paper_0704_3486_gb300 as ovs
    import synth

    if not os.path.exists(ovs.LIB_PATH):
        from paper_0704_3486_gb300 import build
        build.build()
    ovs.load()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist_init(world, local, "nccl")
    stream = torch.cuda.current_stream()

    g = ovs.create_gauge(w["dims"], w["seed"], w["eps"], ovs.MIXED)
    ovs.set_mu(g, w["mu"], w["m_w"])
    if args.stencil_shape is not None:
        ovs.set_stencil_shape(g, ovs.MIXED, w["nrhs"], tuple(args.stencil_shape))
    setup = {"m": w["m"], "seconds": 0.0, "status": "none"}
    if w["m"] > 0:
        ovs.set_setup_budget(g, w["setup_budget_s"])
        t0 = time.perf_counter()
        lam, st = ovs.deflate_setup(g, w["m"], w["eig_tol"], allow_unconverged=True)
        torch.cuda.synchronize()
        stats = ovs.deflate_stats(g)
        setup = {"m": w["m"], "seconds": round(time.perf_counter() - t0, 2), "status": ovs.STATUS.get(st, st),
                 "tol": w["eig_tol"], "max_rel_resid": stats["max_resid"], "budget_s": w["setup_budget_s"],
                 "iterations": stats["iterations"], "matvecs": stats["matvecs"],
                 "abs_lambda_range": [float(np.min(np.abs(lam))), float(np.max(np.abs(lam)))],
                 "min_abs_re_lambda": float(np.min(np.abs(lam.real)))}
    x_host = synth.gaussian_vectors(w["N"], w["nrhs"], w["src_seed"] + 1000 * rank)
    x = torch.from_numpy(x_host).to(dev)
    y = torch.empty_like(x)
    k = w["k"]

    for _ in range(args.warmup):
        ovs.sign_apply(g, x, y, k, prec=ovs.MIXED, stream=stream, want_info=False)
    torch.cuda.synchronize()

    def timed_steps(timing):
        """args.steps applications between a barrier and two CUDA events on
        the launching stream; per-launch event tracing on or off."""
        ovs.profile_enable(g, timing=timing)
        barrier(world)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            ovs.sign_apply(g, x, y, k, prec=ovs.MIXED, stream=stream, want_info=False)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        return e0.elapsed_time(e1), ovs.profile_read(g)

    # the timed region: launches counted, no per-launch events
    clocks = ClockSampler(local)
    clocks.start()
    ms_total, prof_count = timed_steps(False)
    clk = clocks.stop()
    status, info = ovs.get_info(g, w["nrhs"])
    ms_max = max_over_ranks(ms_total, world, dev)
    value = job_value(w["nrhs"], args.steps, world, ms_max)
    # the same steps again with every launch bracketed by CUDA events: the
    # per-class device times of the roofline, and the cost of the tracing
    ms_traced, prof = timed_steps(True)
    ovs.profile_enable(g, timing=False)
    traced_value = job_value(w["nrhs"], args.steps, world, max_over_ranks(ms_traced, world, dev))
    y_mixed = y.clone()

    # end to end through the C ABI with pinned host buffers: H2D of x and
    # D2H of y inside the timed region (the library stages host pointers),
    # right after the device-timed steps, with the clocks sampled as there
    e2e = None
    if not args.no_e2e:
        xh = torch.from_numpy(x_host).pin_memory()
        yh = torch.empty_like(xh).pin_memory()
        ovs.sign_apply(g, xh, yh, k, prec=ovs.MIXED, stream=stream, want_info=False)  # untimed
        barrier(world)
        torch.cuda.synchronize()
        clocks_e2e = ClockSampler(local)
        clocks_e2e.start()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ovs.sign_apply(g, xh, yh, k, prec=ovs.MIXED, stream=stream, want_info=False)
        torch.cuda.synchronize()
        t_e2e = max_over_ranks(time.perf_counter() - t0, world, dev)
        clk_e2e = clocks_e2e.stop()
        nbytes = x_host.size * 16
        e2e = {"value": w["nrhs"] * args.steps * world / t_e2e, "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes, "clocks": clk_e2e}

    # plain FP64, one right-hand side per call, same (m, k), for every
    # right-hand side of the batch: its throughput, and the error of each
    # mixed result against it
    y64 = torch.empty_like(x[:1])
    ovs.sign_apply(g, x[:1].contiguous(), y64, k, prec=ovs.F64, stream=stream, want_info=False)
    torch.cuda.synchronize()
    rel_errs, ms64 = [], 0.0
    for r in range(w["nrhs"]):
        xr = x[r:r + 1].contiguous()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        ovs.sign_apply(g, xr, y64, k, prec=ovs.F64, stream=stream, want_info=False)
        f1.record(stream)
        torch.cuda.synchronize()
        ms64 += f0.elapsed_time(f1)
        rel_errs.append(float(torch.linalg.norm(y_mixed[r] - y64[0]) / torch.linalg.norm(y64[0])))
    fp64_value = w["nrhs"] / (ms64 / 1e3)
    rel_err = max(rel_errs)
    # Krylov truncation at k on this basis: the FP64 result at the largest
    # supported Krylov dimension for right-hand side 0 (a longer reference on
    # the same deflation; not an exact sign when the basis is not converged)
    long_ref = None
    if not args.no_long_ref:
        k_long = 790
        ovs.sign_apply(g, x[:1].contiguous(), y64, k_long, prec=ovs.F64, stream=stream, want_info=False)
        y_k64 = torch.empty_like(y64)
        ovs.sign_apply(g, x[:1].contiguous(), y_k64, k, prec=ovs.F64, stream=stream, want_info=False)
        torch.cuda.synchronize()
        nrm = torch.linalg.norm(y64[0])
        long_ref = {"k_long": k_long,
                    "rel_diff_fp64_k_vs_k_long": float(torch.linalg.norm(y_k64[0] - y64[0]) / nrm),
                    "rel_diff_mixed_k_vs_k_long": float(torch.linalg.norm(y_mixed[0] - y64[0]) / nrm)}

    # roofline of the dominant kernel class (device time share in the timed region)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    peak = peaks.get("hbm_gbs")
    peak_src = "measured"
    if peak is None:
        peak, peak_src = 6800.0, "fallback"
    top = max(("dots", "update", "matvec"), key=lambda c: prof[c]["ms"])
    ach = prof[top]["bytes"] / (prof[top]["ms"] / 1e3) / 1e9 if prof[top]["ms"] > 0 else 0.0
    # DRAM traffic per launch: the ncu capture of the current kernel of each
    # class (16^3x32, 2 RHS, J = 30; profiles/) gave traffic / algorithmic
    # bytes; traffic grows in proportion to the vectors read, so a launch of
    # the timed step moves that ratio times its algorithmic bytes.
    traffic_ratio = {"dots": 808.41 / 805.31, "update": 848.11 / 855.64}.get(top)
    per_launch = prof[top]["bytes"] / max(prof[top]["launches"], 1)
    traffic = round(per_launch * traffic_ratio) if traffic_ratio else None
    share = {c: round(prof[c]["ms"] / max(sum(p["ms"] for p in prof.values()), 1e-9), 4) for c in prof}
    roofline = {"bound": "hbm", "kernel": {"dots": "k_gdots2_ws (CGS2 inner products)",
                                            "update": "k_arnoldi_update_ws (CGS2 update)",
                                            "matvec": "k_wilson (H_w stencil)"}[top],
                "achieved": round(ach, 1), "peak": peak, "unit": "GB/s", "frac": round(ach / peak, 4),
                "peak_source": f"{peak_src} hbm_gbs (copy)", "traffic": traffic,
                "measured_in": "a second timed pass of the same steps with per-launch CUDA events",
                "algorithmic_bytes_per_launch": round(per_launch),
                "per_class": {c: {"ms_per_step": round(prof[c]["ms"] / args.steps, 3),
                                  "launches_per_step": prof[c]["launches"] // max(args.steps, 1),
                                  "gbs": round(prof[c]["bytes"] / (prof[c]["ms"] / 1e3) / 1e9, 1)
                                  if prof[c]["ms"] > 0 else None,
                                  "share": share[c]} for c in prof}}
    launches = sum(p["launches"] for p in prof_count.values())

    # the metric holds only at 1e-6: a batch whose mixed result misses the
    # FP64 result at equal (m, k) by more on any right-hand side scores 0
    metric_met = rel_err <= 1e-6
    out = {
        "metric": METRIC, "value": round(value, 4) if metric_met else 0.0, "unit": UNIT, "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config_of(w, world),
        "fp64_single_rhs": {"value": round(fp64_value, 4), "unit": UNIT, "applications_timed": w["nrhs"],
                            "rel_err_mixed_vs_fp64": rel_err,
                            "rel_err_mixed_vs_fp64_per_rhs": [float(f"{e:.3e}") for e in rel_errs],
                            "within_1e-6": rel_err <= 1e-6,
                            "speedup_mixed_batched": round(value / world / fp64_value, 3)},
        "long_reference": long_ref,
        "accuracy": {"metric_met": metric_met,
                     "reading": "1e-6 = relative 2-norm of the mixed result against the FP64 result at equal "
                                "(m, k), every right-hand side of the batch (max in fp64_single_rhs)",
                     "deflation_basis": f"device set-up within its budget: status {setup['status']} "
                                        f"(residuals in deflation_setup)",
                     "krylov_truncation": "long_reference: FP64 at k against FP64 at k_long on the same basis"},
        "tracing": {"value_with_per_launch_events": round(traced_value, 4),
                    "overhead_frac": round(1.0 - traced_value / value, 4)},
        "deflation_setup": setup,
        "apply_info": {"k_used": sorted({i["k_used"] for i in info}),
                       "newton_iters": sorted({i["newton_iters"] for i in info}),
                       "status": ovs.STATUS.get(status, status)},
        "roofline": roofline, "gpu_launches": int(launches), "clocks": clk, "e2e": e2e,
    }
    if not args.no_variants:
        out["variants"] = run_variants(ovs, g, x, y, k, stream, w)
    tuned = ovs.stencil_tuning(g, ovs.MIXED, w["nrhs"])
    if tuned is not None:  # the autotuner's choice for the timed stencil launches
        rt, sites, rb = tuned["shape"]
        out["stencil_shape"] = {"rhs_per_thread": rt, "sites_per_block": sites, "rhs_tiles_per_block": rb,
                                "candidates_ms": {f"{a}x{b}x{c}": round(t, 4) for (a, b, c), t in tuned["ms"].items()}}
    g.destroy()
    return out


def run_variants(ovs, g, x, y, k, stream, w, steps=2):
    """The method's variants on the timed workload's handle and batch (same
    lattice, k, right-hand sides, mixed form): the harmonic variant (Sec. 4),
    D_ov(mu) x (Sec. 2, Eq. Dov) and Schur deflation (Sec. 5.2) built from the
    installed right vectors. Each: applications/s over `steps` CUDA-event
    timed calls after one untimed call, the per-class device times of one
    traced call, and the relative difference of the result from the LR form
    at the same k (harmonic, Schur: a different approximation, not an
    error)."""
    import torch

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        ovs.profile_enable(g, timing=True)
        fn()
        prof = ovs.profile_read(g)
        ovs.profile_enable(g, timing=False)
        per = {c: {"ms": round(v["ms"], 2), "gbs": round(v["bytes"] / (v["ms"] / 1e3) / 1e9, 1) if v["ms"] > 0 else None}
               for c, v in prof.items() if v["launches"]}
        return {"value": round(w["nrhs"] / (ms / 1e3), 4), "unit": "applications/s", "ms_per_call": round(ms, 2),
                "per_class": per}

    def reldiff(a):
        return float(torch.max(torch.linalg.vector_norm(a - y_lr, dim=1) / torch.linalg.vector_norm(y_lr, dim=1)))

    out = {}
    y_lr = torch.empty_like(x)
    ovs.sign_apply(g, x, y_lr, k, prec=ovs.MIXED, stream=stream, want_info=False)
    yv = torch.empty_like(x)
    out["harmonic"] = timed(lambda: ovs.sign_apply(g, x, yv, k, prec=ovs.MIXED, stream=stream, want_info=False,
                                                   harmonic=True))
    out["harmonic"]["max_rel_diff_vs_lr"] = reldiff(yv)
    out["overlap_apply"] = timed(lambda: ovs.overlap_apply(g, x, yv, k, prec=ovs.MIXED, stream=stream,
                                                          want_info=False))
    if w["m"] > 0:
        R, _, _ = ovs.deflate_get(g)
        ovs.deflate_load_schur(g, R)
        del R
        out["schur"] = timed(lambda: ovs.sign_apply(g, x, yv, k, prec=ovs.MIXED, stream=stream, want_info=False))
        out["schur"]["max_rel_diff_vs_lr"] = reldiff(yv)
        out["schur"]["basis"] = "Schur vectors of the LR set-up's right vectors (same m)"
    return out


def run_batched(args, world, rank, local, steps, warmup):
    """The batched multi-instance workload: synth.batched_instances recipe,
    device set-up of 20 deflation vectors per instance (1 s budget each),
    one ovs_sign_apply_batched of all instances with the per-vector stop
    (by default tol 1e-8 within k = 600, checks on multiples of 10 steps on
    the skip-ahead schedule), mixed form. Applications/s counts every
    right-hand side of every instance per call."""
    import numpy as np
    import torch

    import paper_0704_3486_gb300 as ovs
    import synth

    if not os.path.exists(ovs.LIB_PATH):
        from paper_0704_3486_gb300 import build
        build.build()
    ovs.load()
    torch.cuda.set_device(local)
    dist_init(world, local, "nccl")
    k_cap, every, tol, m, budget = args.batched_cap, args.batched_every, args.batched_tol, 20, 1.0
    prec = ovs.F64 if args.batched_prec == "f64" else ovs.MIXED
    skip = not args.batched_every_check
    specs = synth.batched_instances(args.instances)
    gs, xs, ys = [], [], []
    t0 = time.perf_counter()
    for sp in specs:
        g = ovs.create_gauge(sp["dims"], sp["gauge_seed"], sp["eps"], ovs.MIXED)
        ovs.set_mu(g, sp["mu"], -1.5)
        ovs.set_setup_budget(g, budget)
        ovs.deflate_setup(g, m, 1e-8, allow_unconverged=True)
        n = 12 * int(np.prod(sp["dims"]))
        x = torch.from_numpy(synth.gaussian_vectors(n, sp["nrhs"], sp["source_seed"])).cuda()
        gs.append(g)
        xs.append(x)
        ys.append(torch.empty_like(x))
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        ovs.sign_apply_batched(gs, xs, ys, k_cap, prec=prec, check_every=every, tol=tol, want_info=False,
                               skip_ahead=skip)
    torch.cuda.synchronize()
    barrier(world)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        ovs.sign_apply_batched(gs, xs, ys, k_cap, prec=prec, check_every=every, tol=tol, want_info=False,
                               skip_ahead=skip)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms_max = max_over_ranks(e0.elapsed_time(e1), world, torch.device("cuda", local))
    st, info = ovs.sign_apply_batched(gs, xs, ys, k_cap, prec=prec, check_every=every, tol=tol, skip_ahead=skip)
    total = sum(sp["nrhs"] for sp in specs)
    ks = np.array([i["k_used"] for i in info])
    # FP64 single-RHS reference of one right-hand side per lattice size, at
    # the Krylov dimension the mixed form stopped at
    errs, off = {}, 0
    for sp, g, x, y in zip(specs, gs, xs, ys):
        key = "x".join(map(str, sp["dims"]))
        if prec == ovs.MIXED and key not in errs:
            k0 = int(info[off]["k_used"])
            y64 = torch.empty_like(x[:1])
            ovs.sign_apply(g, x[:1].contiguous(), y64, max(k0, 1), prec=ovs.F64)
            errs[key] = float(torch.linalg.vector_norm(y[:1] - y64) / torch.linalg.vector_norm(y64))
        off += sp["nrhs"]
    out = {
        "metric": "batched sgn(H_w(mu))x applications/s, multi-instance recipe, per-vector stop",
        "value": round(job_value(total, steps, world, ms_max), 3), "unit": UNIT, "n_gpus": world,
        "steps": steps, "warmup": warmup, "ms_per_step": round(ms_max / steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == ovs.F64 else "f32", "data": "synthetic",
        "config": {"workload": f"{len(specs)} instances (4^4/6^4/8^4 cycle, mu 0.1/0.2/0.3), "
                               f"{total} RHS, m={m} each, stop at {tol} on multiples of {every} steps "
                               f"({'every interval' if not skip else 'skip-ahead schedule'}), cap k={k_cap}",
                   "checks": "every interval" if not skip else "skip-ahead",
                   "instances": len(specs), "rhs_total": total, "setup_budget_s_each": budget,
                   "setup_seconds_total": round(t_setup, 1), "parallelism": "replicas"},
        "k_used": {"min": int(ks.min()), "median": float(np.median(ks)), "max": int(ks.max()),
                   "converged_fraction": round(float(np.mean([i["status"] == 0 for i in info])), 3)},
        "rel_err_mixed_vs_fp64_at_equal_k": errs,
    }
    for g in gs:
        g.destroy()
    return out


def run_overlap_solve(args, world, rank, local):
    """Nested inversion D_ov(mu) x = b (Sec. 2, Eq. Dov; Secs. 6, 7) on the
    deflated FP64 configuration's lattice: 8^4, eps 0.7, seed 3, mu 0.2,
    m_w -1.5, m = 30 critical vectors from the device set-up (tol 1e-9),
    16 right-hand sides, inner k = 200, outer GMRES(20). Mixed inner form to
    an outer tolerance of 1e-6, FP64 inner form to 1e-10. Reports the solve
    time, the outer iterations (each one D_ov application of all right-hand
    sides) and the true relative residuals."""
    import numpy as np
    import torch

    import paper_0704_3486_gb300 as ovs
    import synth

    if not os.path.exists(ovs.LIB_PATH):
        from paper_0704_3486_gb300 import build
        build.build()
    ovs.load()
    torch.cuda.set_device(local)
    dims, seed, eps, mu, m, k, nrhs, restart = (8, 8, 8, 8), 3, 0.7, 0.2, 30, 200, 16, 20
    g = ovs.create_gauge(dims, seed, eps, ovs.MIXED)
    ovs.set_mu(g, mu, -1.5)
    t0 = time.perf_counter()
    _, st_setup = ovs.deflate_setup(g, m, 1e-9, allow_unconverged=True)
    t_setup = time.perf_counter() - t0
    n = 12 * int(np.prod(dims))
    b = torch.from_numpy(synth.gaussian_vectors(n, nrhs, 17)).cuda()
    x = torch.empty_like(b)
    out = {"metric": "D_ov(mu) x = b solves/s (nested GMRES around the deflated sign)", "unit": "solves/s",
           "n_gpus": world, "data": "synthetic",
           "config": {"workload": f"8^4 eps=0.7 mu=0.2 m={m} (device set-up {ovs.STATUS.get(st_setup)}, "
                                  f"{t_setup:.1f} s), inner k={k}, GMRES({restart}), {nrhs} RHS",
                      "lattice": list(dims), "m_deflated": m, "k": k, "restart": restart, "nrhs": nrhs}}
    for name, prec, tol in (("mixed_inner", ovs.MIXED, 1e-6), ("fp64_inner", ovs.F64, 1e-10)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, info = ovs.overlap_solve(g, b, x, k, restart, tol, max_cycles=50, prec=prec)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out[name] = {"seconds": round(dt, 3), "value": round(nrhs / dt, 4), "status": ovs.STATUS.get(st, st),
                     "outer_iterations": info[0]["iters"], "cycles": info[0]["cycles"],
                     "max_rel_resid": max(i["rel_resid"] for i in info), "tol": tol,
                     "dov_applications_per_s": round(nrhs * (info[0]["iters"] + info[0]["cycles"]) / dt, 2)}
    g.destroy()
    return out


def run_reference_full(w):
    """One complete oracle application (no sampling, no model): one
    right-hand side, LR deflation with m seeded random vectors, CGS2 Arnoldi
    to k, Roberts' iteration on H_k, recombination. Checks the cost model of
    the bounded sample; its time is the measured one."""
    sampler = CpuSample(w)
    import synth
    from oracle import deflation
    x = synth.gaussian_vectors(w["N"], 1, w["src_seed"])[0]
    t0 = time.perf_counter()
    _, info = deflation.lr_sign_apply(lambda v: sampler.h @ v, x, sampler.r, sampler.l, sampler.lam, w["k"])
    t_app = time.perf_counter() - t0
    t_model, _, _ = sampler.run()
    return {"impl": "reference", "kind": "full_application", "config": config_of(w, 1),
            "seconds_per_application": round(t_app, 2), "applications_per_s": 1.0 / t_app,
            "modelled_seconds_per_application": round(t_model, 2), "cores": cpu_cores(),
            "newton_iters": info["newton_iters"]}


def run_reference(args, w, world, rank):
    """CPU oracle on bounded samples; rank 0 only (other ranks exit).

    Each step runs one bounded sample (CpuSample) and takes its measured
    wall time as the step's time; the fraction of an application a sample
    covers comes from the sample's cost model, so value = fraction / step
    time = 1 / (modelled seconds per application)."""
    if rank != 0:
        return None
    sampler = CpuSample(w)
    t_apps, t_steps = [], []
    desc = ""
    for i in range(args.warmup + args.steps):
        t_app, t_sample, desc = sampler.run(seed_offset=i)
        if i >= args.warmup:
            t_apps.append(t_app)
            t_steps.append(t_sample)
    t_app = statistics.median(t_apps)
    t_step = statistics.median(t_steps)
    value = 1.0 / t_app
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config_of(w, 1),
        "applications_per_step": t_step / t_app,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    args = parse_args()
    w = workload(args)
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        out = run_reference_full(w) if args.full_application and rank == 0 else run_reference(args, w, world, rank)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    if args.workload == "overlap-solve":
        out = run_overlap_solve(args, world, rank, local)
        if rank == 0:
            print(json.dumps(out), flush=True)
        return
    if args.workload == "batched":
        out = run_batched(args, world, rank, local, args.steps, args.warmup)
        if rank == 0:
            print(json.dumps(out), flush=True)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    out = run_ours(args, w, world, rank, local)
    if not args.no_batched:
        b = run_batched(args, world, rank, local, steps=1, warmup=1)
        out["batched"] = {key: b[key] for key in ("metric", "value", "unit", "steps", "warmup", "ms_per_step",
                                                  "config", "k_used", "rel_err_mixed_vs_fp64_at_equal_k")}
    if rank == 0:
        if not args.no_cpu_baseline:
            t_app, t_sample, desc = CpuSample(w).run()
            out["cpu_baseline"] = {"value": 1.0 / t_app, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                                   "sample": desc}
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
