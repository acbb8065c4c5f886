"""Benchmark of the GB300 preconditioned iPEPS hot path.

One step is one pass of the whole hot path on one tensor of the workload:
the CTMRG environment run to its fixed point (warm-started from the previous
pass's environment), the energy and its fixed-point gradient, and the
local-metric preconditioner P^-1 g (GMRES(30), delta = |g|^2).  The tensors
visited are the seeded start tensor of the workload plus 1e-3 U[-1, 1]
perturbations, one per pass (the trial points of an optimiser).  The default
workload is the square-lattice Heisenberg model on a 1x1 cell with d=2, D=4,
chi=64, started from the Neel-like D=1 state embedded in D=4 plus noise.
Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--prec fp64_tc|fp64|bf16x3|tf32x3|tf32x3_all] [--workload NAME]
                  [--mode pass|optimize|ctmrg|gemm|ttt]

--impl reference runs the CPU FP64 oracle on the same passes (the oracle is
the only reference this method has: the paper's own code is not available).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PASS_EPS = 1e-3      # perturbation of the tensor between passes
PASS_SEED = 11       # seed of the perturbation sequence
PASS_TOL = 1e-10     # CTMRG tolerance of a pass
PASS_MAXIT = 200     # CTMRG iteration limit of a pass
# DRAM bytes per launch of the dominant kernels from one ncu capture (see
# profiles/); a kernel changed since its capture has no entry.  A profiler
# class spans launches of many shapes, so a single captured launch does not
# give the class's per-launch traffic: those captures are listed as samples
# (one launch, its shape, its DRAM bytes and its own algorithmic bytes).
NCU_TRAFFIC = {}
NCU_SAMPLES = {
    "dgemm": {"launch": "dgemm_kernel 64 x 1024 x 64, split K 4 (profiles/dgemm_heis_d4_chi64_ncu.md)",
              "dram_bytes": 582400, "operand_bytes": 8 * (64 * 64 + 64 * 1024), "us": 25.2},
    "jacobi_pair": {"launch": "jacobi_pair_kernel, N = 1024 cold-start SVD pair step "
                              "(profiles/jacobi_pair_heis_d4_chi64_ncu.md)",
                    "dram_bytes": 9243648, "us": 2482.0},
}


def pass_config(workload):
    """The workload part of the JSON line's config, the same for both arms."""
    from paper_2511_09546_gb300 import inputs

    w = inputs.WORKLOADS[workload]
    desc = (": Heisenberg square lattice 1x1, d=2, D=4, chi=64, Neel-like D=1 seed in D=4 + 1e-2 noise (seed 0)"
            if workload == "heis_d4_chi64" else "")
    return {"workload": workload + desc,
            "pass": f"tensor_k = start + {PASS_EPS:g} U[-1,1] (seed {PASS_SEED}); CTMRG to {PASS_TOL:g} "
                    "warm-started from pass k-1; energy + fixed-point gradient; P^-1 g with delta = |g|^2, GMRES(30)",
            "chi": w["chi"], "D": w["D"]}


def metric_name(workload):
    return (f"hot-path passes/s ({workload}: warm-started CTMRG fixed point + energy + fixed-point "
            "gradient + local-metric GMRES(30) preconditioner per pass)")


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def ctmrg_flops_per_iteration(w):
    """Algorithmic FLOPs of one CTMRG iteration (2 per multiply-add): per
    projector pair four enlarged corners (chi^3 D^2 + chi^3 D^4 + 2 chi^2 D^6 d
    each), the two half-system products and the four-corner product
    (3 (chi D^2)^3) and the absorption (2 chi^3 D^4 + 2 chi^2 D^6 d + 3 chi^3 D^2);
    4 directional moves x Lx Ly projector pairs."""
    chi, D, d = w["chi"], w["D"], w["d"]
    n = chi * D * D
    corner = chi ** 3 * D ** 2 + chi ** 3 * D ** 4 + 2 * chi ** 2 * D ** 6 * d
    absorb = 2 * chi ** 3 * D ** 4 + 2 * chi ** 2 * D ** 6 * d + 3 * chi ** 3 * D ** 2
    return 2.0 * 4 * w["Lx"] * w["Ly"] * (4 * corner + 3 * n ** 3 + absorb)


class Clocks:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index):
        self.proc = None
        # raw samples go to $IPEPS_BENCH_OUT (default: the system temp directory)
        out_dir = os.environ.get("IPEPS_BENCH_OUT", tempfile.gettempdir())
        self.path = os.path.join(out_dir, f"clocks_{os.getpid()}.csv")
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={index}",
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if sm:
            out["sm_mhz"] = statistics.median(sm)
            out["sm_max_mhz"] = max(smax)
        out["reasons"] = sorted(reasons)
        return out


def replica_rate(local_ms, n_units, world):
    """Whole-job rate of `world` independent replicas, each timing n_units units
    in local_ms: (slowest rank's ms, world * n_units / slowest time in s).  The
    max over ranks is an all-reduce on the process group's own device."""
    import torch

    t = torch.tensor([float(local_ms)], dtype=torch.float64)
    if world > 1:
        dev = "cuda" if torch.distributed.get_backend() == "nccl" else "cpu"
        t = t.to(dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        t = t.cpu()
    slowest = float(t[0])
    return slowest, (world * n_units / (slowest / 1000.0) if slowest > 0 else 0.0)


def measured_peaks_live():
    """cuBLAS FP64 and TF32 GEMM rates on this GPU (torch.matmul, best of 3),
    the denominators for kernels whose dtype MEASURED_PEAKS.json does not cover."""
    import torch

    out = {}
    for name, dt, n, tf32 in (("fp64_tflops", torch.float64, 4096, False), ("tf32_tflops", torch.float32, 8192, True)):
        prev = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = tf32
        a = torch.randn((n, n), dtype=dt, device="cuda")
        b = torch.randn((n, n), dtype=dt, device="cuda")
        c = a @ b
        best = float("inf")
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            c = a @ b
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        torch.backends.cuda.matmul.allow_tf32 = prev
        out[name] = 2.0 * n ** 3 / (best * 1e-3) / 1e12
        del a, b, c
    return out


def _ham(ipeps, w):
    return ipeps.ham_heisenberg(True) if w["d"] == 2 else ipeps.ham_kitaev(-1.0)


PRECS = ["fp64", "tf32x3", "tf32x3_all", "fp64_tc", "bf16x3"]


def _prec(ipeps, name):
    return {"fp64": ipeps.FP64, "tf32x3": ipeps.TF32X3, "tf32x3_all": ipeps.TF32X3_ALL, "fp64_tc": ipeps.FP64_TC,
            "bf16x3": ipeps.BF16X3}[name]


def roofline(prof, peaks_live):
    """Roofline of the dominant kernel class (live CUDA events over the timed
    region): achieved = algorithmic work of its launches / their summed time."""
    if not prof:
        return None
    dom = max(prof, key=lambda k: prof[k]["ms"])
    st = prof[dom]
    peaks = _peaks()
    total = sum(v["ms"] for v in prof.values())
    if dom == "tc_gemm":
        roof = {"kernel": dom, "bound": "tensor", "achieved": 3 * st["flops"] / (st["ms"] * 1e-3) / 1e12,
                "peak": peaks_live.get("tf32_tflops"), "unit": "TFLOP/s",
                "peak_source": "measured: cuBLAS TF32 GEMM 8192^3 on this GPU (torch.matmul, best of 3)",
                "note": "achieved = issued TF32 FLOP/s (3 products per term)"}
    elif dom.startswith("oz") and dom.endswith("_gemm"):
        digits = int(dom[2:-5])
        products = digits * (digits + 1) // 2
        roof = {"kernel": dom, "bound": "tensor", "achieved": products * st["flops"] / (st["ms"] * 1e-3) / 1e12,
                "peak": peaks.get("bf16_tflops_sustained", 1705.9), "unit": "TFLOP/s",
                "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (kernel timed inside a long step)",
                "note": f"achieved = issued BF16 FLOP/s ({products} digit products per FP64 term); "
                        f"FP64-equivalent {st['flops'] / (st['ms'] * 1e-3) / 1e12:.2f} TFLOP/s"}
    elif st["flops"] > 0:
        roof = {"kernel": dom, "bound": "alu", "achieved": st["flops"] / (st["ms"] * 1e-3) / 1e12,
                "peak": peaks_live.get("fp64_tflops"), "unit": "TFLOP/s",
                "peak_source": "measured: cuBLAS FP64 GEMM 4096^3 on this GPU (torch.matmul, best of 3)"}
        if dom == "jacobi_pair":
            roof["note"] = ("FP64 pipe bound (ncu sample); achieved counts only the 32 x 32 Gram products of "
                            "each pair step (a lower bound: rotations and the inner eigensolve are excluded)")
    else:
        roof = {"kernel": dom, "bound": "hbm", "achieved": st["bytes"] / (st["ms"] * 1e-3) / 1e9,
                "peak": peaks.get("hbm_gbs", 6784.5), "unit": "GB/s", "peak_source": "MEASURED_PEAKS.json hbm_gbs"}
    roof["frac"] = roof["achieved"] / roof["peak"] if roof["peak"] else None
    tr = NCU_TRAFFIC.get(dom)
    roof["traffic"] = tr["bytes_per_launch"] if tr else None
    if dom in NCU_SAMPLES:
        roof["ncu_sample"] = NCU_SAMPLES[dom]
    roof["algorithmic_bytes_per_launch"] = st["bytes"] / max(1, st["count"])
    roof["share"] = st["ms"] / max(1e-9, total)
    roof["launches"] = st["count"]
    roof["avg_launch_us"] = 1e3 * st["ms"] / max(1, st["count"])
    return roof


def gpu_pass(ipeps, A, env, w, ham, prec, t_ctm=None):
    """One hot-path pass through the C ABI; returns (env, E, g, x, CTMRG iterations)."""
    import torch

    if t_ctm is not None:
        t_ctm[0].record()
    env, it, _ = ipeps.ctmrg(A, w["chi"], tol=PASS_TOL, maxit=PASS_MAXIT, prec=prec, env=env)
    if t_ctm is not None:
        t_ctm[1].record()
    E, g = ipeps.energy_grad(A, env, ham)
    x, _ = ipeps.precondition(A, env, g, -1.0)
    del torch
    return env, E, g, x, it


def run_ours(args, rank, world, local):
    import torch

    import __graft_entry__ as entry

    entry.build()
    from paper_2511_09546_gb300 import inputs, ipeps

    torch.cuda.set_device(local)
    w = inputs.WORKLOADS[args.workload]
    cell0 = w["gen"]()
    ham = _ham(ipeps, w)
    prec = _prec(ipeps, args.prec)
    K, W = args.steps, args.warmup
    cells = inputs.perturbed_cells(cell0, W + K, PASS_EPS, PASS_SEED + rank)
    hostA = [torch.as_tensor(ipeps.cell_tensor(c)) for c in cells]
    devA = [a.cuda() for a in hostA]  # resident in HBM before the timed region
    peaks_live = measured_peaks_live()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2
    stream = torch.cuda.current_stream()
    # cold start (untimed)
    env, _, _ = ipeps.ctmrg(torch.as_tensor(ipeps.cell_tensor(cell0), device="cuda"), w["chi"], tol=PASS_TOL,
                            maxit=PASS_MAXIT, prec=prec)
    for k in range(W):
        env, E, g, x, it = gpu_pass(ipeps, devA[k], env, w, ham, prec)
        print(f"[bench] warm-up pass {k}: ctm {it} E {E:.12f}", file=sys.stderr, flush=True)
    env_after_warmup = env
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = Clocks(local)
    ipeps.profile(True)
    launch0 = ipeps.launch_count()
    lat, ctm_ms, ctm_its, energies = [], [], [], []
    for k in range(W, W + K):
        flush.fill_(float(k))  # L2 flush between passes, outside the timed spans
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        env, E, g, x, it = gpu_pass(ipeps, devA[k], env, w, ham, prec, t_ctm=(c0, c1))
        e1.record(stream)
        torch.cuda.synchronize()
        lat.append(e0.elapsed_time(e1))
        ctm_ms.append(c0.elapsed_time(c1))
        ctm_its.append(it)
        energies.append(E)
        print(f"[bench] pass {k}: ctm {it} E {E:.12f} {lat[-1]:.1f} ms", file=sys.stderr, flush=True)
    torch.cuda.synchronize()
    launches = ipeps.launch_count() - launch0
    prof = ipeps.profile_stats()
    ipeps.profile(False)
    clk = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    total_ms, value = replica_rate(sum(lat), K, world)

    # ---- end to end through the C ABI with host buffers: every pass copies its
    # tensor from pinned host memory and reads back g and P^-1 g and E
    pinned = [a.pin_memory() for a in hostA[W:W + K]]
    g_host = torch.empty_like(pinned[0]).pin_memory()
    x_host = torch.empty_like(pinned[0]).pin_memory()
    env = env_after_warmup
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(K):
        Ad = pinned[k].to("cuda", non_blocking=True)
        env, E, g, x, _ = gpu_pass(ipeps, Ad, env, w, ham, prec)
        g_host.copy_(g, non_blocking=True)
        x_host.copy_(x, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    nbytes = pinned[0].numel() * 8

    ctm_flops = ctmrg_flops_per_iteration(w)
    rec = {
        "metric": metric_name(args.workload),
        "value": value,
        "unit": "passes/s",
        "n_gpus": world,
        "steps": K,
        "warmup": W,
        "ms_per_step": total_ms / K,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {ipeps.FP64: "f64", ipeps.FP64_TC: "f64 from bf16 digits (tensor cores, fp32/int64 accumulate)",
                  ipeps.BF16X3: "bf16x3+f64", ipeps.TF32X3: "tf32x3+f64", ipeps.TF32X3_ALL: "tf32x3"}[prec],
        "data": "synthetic",
        "config": dict(pass_config(args.workload), precision=args.prec,
                       l2="flushed (256 MB write) between timed passes",
                       parallelism="replicas" if world > 1 else "single GPU"),
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
        "ctmrg": {"iterations_per_pass": statistics.mean(ctm_its), "ms_per_pass": statistics.mean(ctm_ms),
                  "algorithmic_tflop_per_iteration": ctm_flops / 1e12,
                  "tflops": ctm_flops * sum(ctm_its) / (sum(ctm_ms) * 1e-3) / 1e12 if sum(ctm_ms) > 0 else None},
        "energy": energies[-1],
        "roofline": roofline(prof, peaks_live),
        "peaks_live": peaks_live,
        "e2e": {"value": K / e2e_s, "unit": "passes/s", "h2d_bytes_per_step": int(nbytes),
                "d2h_bytes_per_step": int(2 * nbytes + 8)},
        "gpu_launches": int(launches),
        "launches_per_step": launches / K,
        "clocks": clk,
        "kernels": {k: {"count": v["count"], "ms": round(v["ms"], 3),
                        "tflops": round(v["flops"] / max(1e-9, v["ms"] * 1e-3) / 1e12, 4)}
                    for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])},
        "hbm_kernels": hbm_kernels(prof, _peaks().get("hbm_gbs", 6784.5)),
    }
    rec["preconditioners_ms"] = precond_timings(ipeps, devA[W + K - 1], env, g)
    return rec


def hbm_kernels(prof, hbm_peak):
    """Achieved GB/s of the data-movement kernel classes (permutations, digit
    packing) over the timed passes, against the measured copy bandwidth."""
    out = {}
    for k, v in prof.items():
        if v["flops"] == 0 and v["bytes"] > 0 and v["ms"] > 0:
            gbs = v["bytes"] / (v["ms"] * 1e-3) / 1e9
            out[k] = {"launches": v["count"], "gb_per_launch": v["bytes"] / max(1, v["count"]) / 1e9,
                      "achieved_gbs": gbs, "frac": gbs / hbm_peak if hbm_peak else None}
    return out


def precond_timings(ipeps, A, env, g, reps=3):
    """Milliseconds per call of the two preconditioners at the last pass's
    tensor (local metric + GMRES(30); mean-field metric), outside the timed
    region; None where a call fails (reported, not fatal)."""
    import torch

    res = {}
    for name, fn in (("local_metric_gmres30", lambda: ipeps.precondition(A, env, g, -1.0)),
                     ("mean_field_bp", lambda: ipeps.precondition_bp(A, g, -1.0))):
        try:
            fn()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                r = fn()
            torch.cuda.synchronize()
            res[name] = 1e3 * (time.perf_counter() - t0) / reps
            if name == "mean_field_bp":
                res["mean_field_bp_sweeps"] = r[1]
        except Exception as exc:  # noqa: BLE001 - reported in the JSON line
            res[name] = None
            res[name + "_error"] = str(exc)[:200]
    return res


# --------------------------------------------------------------- oracle side
def oracle_passes(workload, count, seed_offset=0, sink=None):
    """The oracle on the host cores, the same passes as the GPU arm: cold CTMRG at
    the start tensor (untimed), then per pass a warm-started CTMRG fixed point,
    the energy and fixed-point gradient and P^-1 g (delta = |g|^2, GMRES(30)) of
    every tensor.  Returns the per-pass seconds and the thread count."""
    import torch

    from oracle import ctmrg as OC
    from oracle import gradient as OG
    from oracle import metric as OMt
    from oracle import models as OM
    from paper_2511_09546_gb300 import inputs

    w = inputs.WORKLOADS[workload]
    cell0 = w["gen"]()
    Lx, Ly = w["Lx"], w["Ly"]
    ham = OM.heisenberg(True) if w["d"] == 2 else OM.kitaev_dimer(-1.0)
    env, _, _ = OC.ctmrg(cell0, w["chi"], tol=PASS_TOL, maxit=PASS_MAXIT)
    cells = inputs.perturbed_cells(cell0, count, PASS_EPS, PASS_SEED + seed_offset)
    times = []
    for k, cell in enumerate(cells):
        t0 = time.perf_counter()
        env, _, _ = OC.ctmrg(cell, w["chi"], tol=PASS_TOL, maxit=PASS_MAXIT, env=env)
        E, g, info = OG.energy_and_gradient(cell, ham, w["chi"], tol=PASS_TOL, env=env, return_info=True)
        env = info["env"]
        delta = max(sum(float(np.sum(g[x][y] ** 2)) for x in range(Lx) for y in range(Ly)), 1e-12)
        A = OC.as_torch_cell(cell)
        for x in range(Lx):
            for y in range(Ly):
                M = OMt.local_metric(env, A[x][y], x, y).numpy()
                OMt.precondition(M, g[x][y], delta)
        times.append(time.perf_counter() - t0)
        if sink:
            sink(k, times[-1], E)
    return times, torch.get_num_threads()


def cpu_baseline(workload, passes=1):
    """The oracle's pass rate on a bounded sample: `passes` oracle passes after an
    untimed cold CTMRG (about 10-20 s of CPU work at the D=4, chi=64 workload)."""
    times, cores = oracle_passes(workload, passes)
    v = len(times) / sum(times)
    return {"value": v, "unit": "passes/s", "cores": cores, "kind": "oracle",
            "sample": f"{len(times)} oracle pass(es) of the same workload (first perturbed tensor), "
                      f"{sum(times):.1f} s; cold CTMRG at the start tensor untimed"}


def run_reference(args, rank, world):
    """--impl reference: the oracle (FP64, host cores) on the same passes; W
    untimed passes then K timed, each one whole oracle pass."""
    if rank != 0:
        return
    K, W = args.steps, args.warmup

    def sink(k, t, E):
        print(f"[reference] pass {k}: {t:.2f} s E {E:.12f}", file=sys.stderr, flush=True)

    times, cores = oracle_passes(args.workload, W + K, sink=sink)
    t = sum(times[W:])
    v = K / t
    rec = {"impl": "reference", "metric": metric_name(args.workload), "value": v, "unit": "passes/s",
           "n_gpus": world, "steps": K, "warmup": W, "ms_per_step": 1e3 * t / K, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": dict(pass_config(args.workload), precision="fp64 (oracle)", parallelism="host cores"),
           "cpu_baseline": {"value": v, "unit": "passes/s", "cores": cores, "kind": "oracle",
                            "sample": f"{K} timed oracle passes after {W} untimed ones (whole passes: CTMRG, "
                                      "energy, fixed-point gradient, preconditioner)"},
           "e2e": {"value": v, "unit": "passes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(rec), flush=True)


# --------------------------------------------------------------- other modes
def run_optimize(args):
    """--mode optimize: preconditioned L-BFGS iterations at the workload (W warm-up
    iterations, K timed), each a CTMRG fixed point + energy + gradient +
    preconditioner per line-search evaluation.  Prints one JSON line."""
    import torch

    import __graft_entry__ as entry

    entry.build()
    from paper_2511_09546_gb300 import inputs, ipeps

    w = inputs.WORKLOADS[args.workload]
    A = torch.as_tensor(ipeps.cell_tensor(w["gen"]()), device="cuda")
    prec = _prec(ipeps, args.prec)
    K, W = args.steps, args.warmup
    opts = ipeps.default_opts(chi=w["chi"], maxiter=W + K, precondition=1, ctm_tol=1e-10, ctm_maxit=120,
                              prec=prec, gtol=0.0)
    walls = []

    def cb(rec):
        print(f"[bench] iter {rec['iter']} E={rec['E']:.12f} |g|={rec['gnorm']:.3e} evals={rec['evals']} "
              f"ctm={rec['ctm_iters']} wall={rec['wall_ms']:.0f} ms", file=sys.stderr, flush=True)
        if rec["iter"] > W:
            walls.append(rec["wall_ms"])
        return 0

    torch.cuda.synchronize()
    _, log, status = ipeps.optimize(A, _ham(ipeps, w), opts, callback=cb)
    rec = {"mode": "optimize", "workload": args.workload, "precision": args.prec, "iterations": len(walls),
           "iterations_per_s": 1e3 * len(walls) / sum(walls) if walls else None,
           "latency_ms": {"p50": float(np.percentile(walls, 50)) if walls else None,
                          "p99": float(np.percentile(walls, 99)) if walls else None},
           "energy": log[-1]["E"] if log else None, "status": status}
    print(json.dumps(rec), flush=True)


def run_ctmrg(args):
    """--mode ctmrg: CTMRG throughput.  W warm-up iterations (cold start and chi
    growth), then K timed iterations, each one full CTMRG iteration (4 directional
    moves, Lx*Ly projector pairs each) warm-started from the previous one; prints
    one JSON line with iterations/s, moves/s and TFLOP/s (library profiler)."""
    import torch

    import __graft_entry__ as entry

    entry.build()
    from paper_2511_09546_gb300 import inputs, ipeps

    w = inputs.WORKLOADS[args.workload]
    A = torch.as_tensor(ipeps.cell_tensor(w["gen"]()), device="cuda")
    prec = _prec(ipeps, args.prec)
    free0 = torch.cuda.mem_get_info()[0]
    env = None
    for _ in range(args.warmup):
        env, _, _ = ipeps.ctmrg(A, w["chi"], tol=1e-30, maxit=1, prec=prec, env=env, allow_unconverged=True)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    peaks_live = measured_peaks_live()
    ipeps.profile(True)
    lat = []
    for _ in range(args.steps):
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        env, _, err = ipeps.ctmrg(A, w["chi"], tol=1e-30, maxit=1, prec=prec, env=env, allow_unconverged=True)
        t1.record()
        torch.cuda.synchronize()
        lat.append(t0.elapsed_time(t1))
    st = ipeps.profile_stats()
    ipeps.profile(False)
    tot_ms = sum(lat)
    tf32_peak = peaks_live["tf32_tflops"]
    model = ctmrg_flops_per_iteration(w)
    gm = st.get("tc_gemm", {"ms": 0.0, "flops": 0.0, "count": 0})
    rec = {"mode": "ctmrg", "workload": args.workload, "precision": args.prec, "iterations": len(lat),
           "ms_per_iteration": tot_ms / max(1, len(lat)),
           "ctmrg_iterations_per_s": 1e3 * len(lat) / tot_ms, "moves_per_s": 4e3 * len(lat) / tot_ms,
           "algorithmic_tflop_per_iteration": model / 1e12,
           "algorithmic_tflops": model * len(lat) / (tot_ms * 1e-3) / 1e12,
           "tc_gemm": {"share": gm["ms"] / tot_ms, "launches": gm["count"],
                       "logical_tflops": gm["flops"] / max(1e-9, gm["ms"] * 1e-3) / 1e12,
                       "issued_frac_of_tf32_peak": 3 * gm["flops"] / max(1e-9, gm["ms"] * 1e-3) / 1e12 / tf32_peak},
           "digit_gemm": {k: {"share": st[k]["ms"] / tot_ms, "launches": st[k]["count"],
                              "logical_tflops": st[k]["flops"] / max(1e-9, st[k]["ms"] * 1e-3) / 1e12,
                              "issued_frac_of_bf16_peak": prods * st[k]["flops"] / max(1e-9, st[k]["ms"] * 1e-3)
                              / 1e12 / _peaks().get("bf16_tflops_sustained", 1705.9)}
                          for k, prods in (("oz2_gemm", 3), ("oz8_gemm", 36)) if k in st},
           "peaks_live": peaks_live,
           "last_change": err, "device_bytes_after_warmup": int(free0 - free1),
           "kernels": {k: {"count": v["count"], "ms": round(v["ms"], 2),
                           "tflops": round(v["flops"] / max(1e-9, v["ms"] * 1e-3) / 1e12, 3)}
                       for k, v in sorted(st.items(), key=lambda kv: -kv[1]["ms"])[:10]}}
    print(json.dumps(rec), flush=True)


def run_ttt(args):
    """--mode ttt: time to E - E_ref <= 1e-7 from the workload's seeded start.
    Run 1, the preconditioned path in --prec (default fp64_tc), continues until
    its energy has changed by less than 1e-10 over 10 iterations (or
    --ttt-maxiter); E_ref is its lowest energy (the reading of |dE| of the paper's
    tables: E_k - E_ref with E_ref from a long preconditioned run) and its time
    to tolerance is the wall time of the first iteration within 1e-7 of E_ref.
    Run 2, plain L-BFGS on the FP64 CUDA-core path, stops at E_ref + 1e-7 or
    after --ttt-plain-seconds.  Wall times with the device synchronised."""
    import torch

    import __graft_entry__ as entry

    entry.build()
    from paper_2511_09546_gb300 import inputs, ipeps

    w = inputs.WORKLOADS[args.workload]
    A0 = torch.as_tensor(ipeps.cell_tensor(w["gen"]()), device="cuda")
    ham = _ham(ipeps, w)
    pname = args.prec if args.prec != "fp64" else "fp64_tc"
    out = {"mode": "ttt", "workload": args.workload, "tolerance": 1e-7}
    clocks = Clocks(0)
    # ---- run 1: preconditioned, to stagnation
    opts = ipeps.default_opts(chi=w["chi"], maxiter=args.ttt_maxiter, precondition=1, ctm_tol=1e-10, ctm_maxit=200,
                              prec=_prec(ipeps, pname), gtol=0.0)
    hist = []
    t0 = time.perf_counter()

    def cb1(rec):
        hist.append((time.perf_counter() - t0, rec["E"], rec["evals"]))
        print(f"[ttt] preconditioned_{pname} iter {rec['iter']} E {rec['E']:.13f} |g| {rec['gnorm']:.2e} "
              f"evals {rec['evals']} t {hist[-1][0]:.1f} s", file=sys.stderr, flush=True)
        return 1 if len(hist) > 10 and abs(hist[-11][1] - hist[-1][1]) < 1e-10 else 0

    torch.cuda.synchronize()
    A1, log1, st1 = ipeps.optimize(A0, ham, opts, callback=cb1)
    torch.cuda.synchronize()
    e_ref = min(h[1] for h in hist)
    first = next(h for h in hist if h[1] - e_ref <= 1e-7)
    out["E_ref"] = e_ref
    out["E_ref_source"] = f"lowest energy of run 1 ({len(hist) - 1} preconditioned {pname} iterations, status {st1})"
    out["preconditioned_" + pname] = {"seconds": first[0], "iterations": hist.index(first),
                                      "evaluations": sum(h[2] for h in hist[:hist.index(first) + 1]),
                                      "run_seconds": hist[-1][0], "run_iterations": len(hist) - 1}
    # ---- run 2: plain FP64 (CUDA cores), capped in wall time
    opts = ipeps.default_opts(chi=w["chi"], maxiter=100000, precondition=0, ctm_tol=1e-10, ctm_maxit=200,
                              prec=ipeps.FP64, gtol=0.0, E_target=e_ref + 1e-7)
    hist2 = []
    t0 = time.perf_counter()

    def cb2(rec):
        hist2.append((time.perf_counter() - t0, rec["E"], rec["evals"]))
        print(f"[ttt] plain_fp64 iter {rec['iter']} E {rec['E']:.13f} dE {rec['E'] - e_ref:.2e} evals {rec['evals']} "
              f"t {hist2[-1][0]:.1f} s", file=sys.stderr, flush=True)
        return 1 if hist2[-1][0] > args.ttt_plain_seconds else 0

    torch.cuda.synchronize()
    _, log2, st2 = ipeps.optimize(A0, ham, opts, callback=cb2)
    torch.cuda.synchronize()
    reached = [h for h in hist2 if h[1] - e_ref <= 1e-7]
    out["plain_fp64"] = {"seconds": reached[0][0] if reached else None, "reached": bool(reached),
                         "run_seconds": hist2[-1][0], "run_iterations": len(hist2) - 1,
                         "best_dE": min(h[1] for h in hist2) - e_ref, "status": st2}
    out["speedup_vs_plain_fp64"] = (reached[0][0] / first[0]) if reached else None
    out["speedup_lower_bound"] = None if reached else hist2[-1][0] / first[0]
    out["clocks"] = clocks.stop()
    print(json.dumps(out), flush=True)


def run_serve(args):
    """--mode serve: the serving mix.  Jobs arrive as a seeded Poisson stream
    (mean gap 50 ms): J1-J2 Heisenberg with J2 ~ U[0, 0.6], D ~ U{2 .. --serve-dmax},
    chi = 2 D^2 or 4 D^2, 1x1 (sublattice-rotated) or 2x2 cell, A ~ U[-1, 1];
    each job runs --serve-iters preconditioned L-BFGS iterations in --prec (default
    bf16x3) on the server's slots.  Reports per-iteration p50/p99 latency, job
    throughput and time from submission to completion."""
    import torch

    import __graft_entry__ as entry

    entry.build()
    from paper_2511_09546_gb300 import inputs, ipeps

    rng = np.random.default_rng(0)
    prec = _prec(ipeps, args.prec if args.prec != "fp64_tc" else "bf16x3")
    specs = []
    t = 0.0
    for k in range(args.serve_jobs):
        t += rng.exponential(0.05)
        D = int(rng.integers(2, args.serve_dmax + 1))
        chi = int(D * D * (2 if rng.random() < 0.5 else 4))
        cell = (1, 1) if rng.random() < 0.5 else (2, 2)
        J2 = float(rng.uniform(0.0, 0.6))
        A = ipeps.cell_tensor(inputs.uniform_cell(cell[0], cell[1], 2, D, 1000 + k))
        specs.append((t, D, chi, cell, J2, A))
    srv = ipeps.Server(slots=args.serve_slots)
    clocks = Clocks(0)
    t0 = time.perf_counter()
    ids = []
    for (ta, D, chi, cell, J2, A) in specs:
        while time.perf_counter() - t0 < ta:
            time.sleep(0.001)
        ham = ipeps.ham_j1j2(1.0, J2, rotated=(cell == (1, 1)))
        o = ipeps.default_opts(chi=chi, maxiter=args.serve_iters, precondition=1, ctm_tol=1e-10, ctm_maxit=300,
                               prec=prec)
        ids.append((srv.submit(A, ham, o), ta, D, chi, cell))
    res = []
    for j, ta, D, chi, cell in ids:
        r = srv.wait(j, 7200)
        res.append(dict(r, D=D, chi=chi, cell=f"{cell[0]}x{cell[1]}", total_ms=r["queued_ms"] + r["run_ms"]))
        print(f"[serve] job {j} D={D} chi={chi} cell={cell} {r['state']} it={r['iterations']} E={r['E']:.10f} "
              f"queued {r['queued_ms']:.0f} ms run {r['run_ms']:.0f} ms", file=sys.stderr, flush=True)
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    done = [r for r in res if r["state"] == "done"]
    its = sum(r["iterations"] for r in done)
    rec = {"mode": "serve", "precision": args.prec, "jobs": len(res), "done": len(done), "slots": args.serve_slots,
           "iterations_per_job": args.serve_iters, "wall_s": wall, "jobs_per_s": len(done) / wall,
           "iterations_per_s": its / wall,
           "iter_latency_ms": {"p50": st["iter_ms_p50"], "p99": st["iter_ms_p99"]},
           "job_latency_ms": {"p50": float(np.percentile([r["total_ms"] for r in done], 50)) if done else None,
                              "p99": float(np.percentile([r["total_ms"] for r in done], 99)) if done else None},
           "mix": f"Poisson arrivals (mean gap 50 ms, seed 0), D in 2..{args.serve_dmax}, chi in {{2D^2, 4D^2}}, "
                  "1x1 / 2x2, J2 ~ U[0, 0.6]",
           "clocks": clocks.stop(), "failed": [r for r in res if r["state"] != "done"]}
    print(json.dumps(rec), flush=True)


def run_fdcheck(args):
    """--mode fdcheck: the fixed-point gradient of the workload (default the Kitaev
    1x2, d=4, D=6, chi=72 cell) against central differences of the energy
    (step 1e-6) on 32 entries drawn by seed 1, everything on the GPU in --prec."""
    import torch

    import __graft_entry__ as entry

    entry.build()
    from paper_2511_09546_gb300 import inputs, ipeps

    w = inputs.WORKLOADS[args.workload]
    A = torch.as_tensor(ipeps.cell_tensor(w["gen"]()), device="cuda")
    ham = _ham(ipeps, w)
    prec = _prec(ipeps, args.prec)
    tol = 1e-11
    t0 = time.perf_counter()
    env, it, err = ipeps.ctmrg(A, w["chi"], tol=tol, maxit=1000, prec=prec)
    t_ctm = time.perf_counter() - t0
    t0 = time.perf_counter()
    E, g = ipeps.energy_grad(A, env, ham)
    torch.cuda.synchronize()
    t_grad = time.perf_counter() - t0
    idx = inputs.random_entries(A.numel(), 32, seed=1)
    h = 1e-6
    gflat = g.view(-1).cpu().numpy()
    rows = []
    t0 = time.perf_counter()
    for i in idx:
        vals = []
        for sgn in (1, -1):
            Ap = A.clone()
            Ap.view(-1)[int(i)] += sgn * h
            env, _, _ = ipeps.ctmrg(Ap, w["chi"], tol=tol, maxit=1000, prec=prec, env=env)
            vals.append(ipeps.energy(Ap, env, ham))
        fd = (vals[0] - vals[1]) / (2 * h)
        rows.append((int(i), float(gflat[i]), fd))
        print(f"[fd] entry {i}: grad {gflat[i]: .10e} fd {fd: .10e} diff {fd - gflat[i]: .2e}", file=sys.stderr,
              flush=True)
    gmax = float(np.abs(gflat).max())
    diffs = [abs(fd - gi) for _, gi, fd in rows]
    rec = {"mode": "fdcheck", "workload": args.workload, "precision": args.prec, "E": E, "ctm_iters": it,
           "ctm_change": err, "seconds_ctmrg": t_ctm, "seconds_gradient": t_grad,
           "seconds_fd": time.perf_counter() - t0, "entries": len(rows), "step": h,
           "max_abs_diff": max(diffs), "max_abs_grad": gmax, "max_rel_diff_vs_max_grad": max(diffs) / gmax,
           "rows": rows}
    print(json.dumps(rec), flush=True)


def run_gemm(args):
    """--mode gemm: one tensor-core GEMM (3xTF32, or the BF16-digit kernel for
    --prec fp64_tc / bf16x3) on n x n x n FP64 operands, timed per kernel class
    with CUDA events (W warm-up calls, K timed calls)."""
    import torch

    import __graft_entry__ as entry

    entry.build()
    from paper_2511_09546_gb300 import ipeps

    n = args.gemm_n
    g = torch.Generator(device="cpu").manual_seed(0)
    A = torch.randn((n, n), generator=g, dtype=torch.float64).cuda()
    B = torch.randn((n, n), generator=g, dtype=torch.float64).cuda()
    C = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    name = args.prec if args.prec != "fp64" else "tf32x3"
    prec = _prec(ipeps, name)
    for _ in range(args.warmup):
        ipeps.gemm(A, B, C=C, prec=prec)
    torch.cuda.synchronize()
    peaks_live = measured_peaks_live()
    ipeps.profile(True)
    for _ in range(args.steps):
        ipeps.gemm(A, B, C=C, prec=prec)
    torch.cuda.synchronize()
    st = ipeps.profile_stats()
    ipeps.profile(False)
    ref_rows = A[:64] @ B
    err = float((C[:64] - ref_rows).abs().max() / ref_rows.abs().max())
    if name.startswith("tf32"):
        kern, pack, products, peak, unit = "tc_gemm", "tc_pack", 3, peaks_live["tf32_tflops"], "tf32"
    else:
        digits = 8 if name == "fp64_tc" else 2
        kern, pack = f"oz{digits}_gemm", "oz_pack"
        products = digits * (digits + 1) // 2
        peak, unit = _peaks().get("bf16_tflops", 1908.5), "bf16"
    gm, pk = st.get(kern, {}), st.get(pack, {})
    logical = gm["flops"] / (gm["ms"] * 1e-3) / 1e12
    rec = {"mode": "gemm", "prec": name, "n": n, "launches": gm.get("count"), "gemm_ms": gm["ms"] / max(1, gm["count"]),
           "pack_ms": pk.get("ms", 0.0) / max(1, pk.get("count", 1)),
           "logical_tflops": logical, "products_per_term": products, f"issued_{unit}_tflops": products * logical,
           f"{unit}_peak_tflops": peak, "issued_frac_of_peak": products * logical / peak,
           "pack_gbs": pk.get("bytes", 0.0) / max(1e-9, pk.get("ms", 0.0) * 1e-3) / 1e9,
           "rel_err_vs_fp64": err, "peaks_live": peaks_live}
    print(json.dumps(rec), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="fp64_tc", choices=PRECS)
    ap.add_argument("--workload", default="heis_d4_chi64")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mode", default="pass", choices=["pass", "optimize", "gemm", "ctmrg", "ttt", "serve", "fdcheck"])
    ap.add_argument("--serve-jobs", type=int, default=64)
    ap.add_argument("--serve-dmax", type=int, default=6)
    ap.add_argument("--serve-iters", type=int, default=3)
    ap.add_argument("--serve-slots", type=int, default=3)
    ap.add_argument("--ttt-maxiter", type=int, default=400)
    ap.add_argument("--ttt-plain-seconds", type=float, default=1200.0)
    ap.add_argument("--gemm-n", type=int, default=8192)
    args = ap.parse_args()
    rank, world, local = _dist()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    modes = {"optimize": run_optimize, "gemm": run_gemm, "ctmrg": run_ctmrg, "ttt": run_ttt, "serve": run_serve,
             "fdcheck": run_fdcheck}
    if args.mode in modes:
        modes[args.mode](args)
        return
    import torch

    if world > 1:
        torch.distributed.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    rec = run_ours(args, rank, world, local)
    if rank == 0:
        if not args.no_cpu_baseline:
            rec["cpu_baseline"] = cpu_baseline(args.workload)
        print(json.dumps(rec), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
