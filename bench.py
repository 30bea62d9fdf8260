#!/usr/bin/env python3
"""Throughput benchmark of the spectral SOG evaluation (energy + forces).

One step = one sog_eval call over the whole hot path (binning, near field,
mid range, long range and its k = 0 mode, assembly) on the workload below,
with inputs resident on the device.  Prints one JSON line.

Workload (default "c2"): N = 1e5 neutral +-1 charges, uniform positions in a
100 x 100 x 100 box, periodic in x and y and free in z, relative tolerance
1e-6, mixed precision (FP32 bulk, FP64 tables / k = 0 mode / reductions).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With --gpus N > 1 (launched by torch.distributed.run) every rank evaluates
its own replica of the workload; there is no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particles/s (energy+forces) at rel. error 1e-6 vs FP64 oracle; % HBM roofline"
WORKLOADS = {
    "c2": dict(N=100000, L=(100.0, 100.0, 100.0), tol=1e-6, seed=1,
               desc="uniform neutral +-1 charges, N=1e5, box 100x100x100 (periodic x,y, free z), tol 1e-6"),
    "c2_1e4": dict(N=100000, L=(100.0, 100.0, 100.0), tol=1e-4, seed=1,
                   desc="uniform neutral +-1 charges, N=1e5, box 100x100x100, tol 1e-4"),
    "c1": dict(N=1000, L=(10.0, 10.0, 10.0), tol=1e-6, seed=1,
               desc="uniform neutral +-1 charges, N=1e3, box 10x10x10, tol 1e-6"),
    "c5": dict(batch=256, seed=5, tol=1e-6, N=None, L=(0.0, 0.0, 0.0),
               desc="256 independent neutral +-1 systems, N log-uniform in [500, 50000], "
                    "density 0.1, Lz/Lx uniform in [0.05, 10], tol 1e-6, one graph launch"),
}
FLUSH_BYTES = 512 << 20          # larger than the 129 MB L2, written between steps
# FP32 operations of the near field: 8 per candidate of the 27-cell
# neighbourhood (3 differences, squared distance, comparison) and 60 per pair
# inside r_c (distance again, reciprocal square root, degree-8 table
# polynomial with its derivative, compensated potential sum, force).
CAND_FLOP = 8
PAIR_FLOP = 60
DOMINANT = "near"   # largest share of GPU time in the kernel launch list


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm = sorted(float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit())
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[3 + k] == "Active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def stage_units(prm, N, stage):
    """Algorithmic work of one launch of a stage and the resource bounding it:
    ("alu", FP32 operations) or ("hbm", bytes), with a description."""
    Ix, Iy, Iz = prm["I"]
    P = prm["P_win"]
    L = prm["L"]
    rho = N / (L[0] * L[1] * L[2])
    pairs = N * 4.0 / 3.0 * math.pi * prm["rc"] ** 3 * rho
    ncell = [max(1, int(math.floor(L[d] / prm["rc"]))) for d in range(3)]
    cand = N * 27.0 * N / (ncell[0] * ncell[1] * ncell[2])
    if stage == "near":
        return ("alu", cand * CAND_FLOP + pairs * PAIR_FLOP,
                "FP32 flop: %.3g candidates x %d + %.3g pairs x %d" % (cand, CAND_FLOP, pairs, PAIR_FLOP))
    if stage == "mid_spread":
        return "alu", N * P ** 3 * 2.0, "FP32 flop: N x P^3 x 2"
    if stage == "mid_gather":
        return "alu", N * P ** 3 * 4.0, "FP32 flop: N x P^3 x 4 (value and x-derivative sums)"
    if stage == "mid_fft":
        half = Iz * Iy * (Ix // 2 + 1)
        return ("hbm", 3 * 2 * half * 8 + half * 4,
                "bytes: 3 passes x (read + write) of the complex half spectrum + scaling table")
    if stage == "long_gather":
        Pl, Pc = prm["P_long"], prm["P_cheb"]
        return "alu", N * Pc * Pl ** 2 * 4.0, "FP32 flop: N x P_cheb x P_long^2 x 4"
    if stage == "long_spread":
        Pc = prm["P_cheb"]
        Ilx, Ily = prm["I_long"]
        return "alu", N * Pc * Ilx * Ily * 2.0, "FP32 flop: N x P_cheb x I_long^2 x 2 (dense planes)"
    if stage in ("long_moments", "long_eval"):
        Pc = prm["P_cheb"]
        Kx, Ky = (prm["I_long"][0] - 1) // 2, (prm["I_long"][1] - 1) // 2
        nh = Ky + Kx * (2 * Ky + 1)
        k = 4.0 if stage == "long_moments" else 8.0
        return ("alu", N * nh * Pc * k,
                "FP32 flop: N x half-plane modes x P_cheb x %d" % k)
    return None, None, None


def roofline_entry(prm, N, stage, t_s, hbm, fp32_peak, smax, src):
    bound, work, desc = stage_units(prm, N, stage)
    if bound == "alu":
        ach = work / t_s / 1e12
        return {"bound": "alu", "kernel": stage, "achieved": ach, "peak": fp32_peak,
                "unit": "TFLOP/s", "frac": ach / fp32_peak, "work_per_launch": desc,
                "peak_source": "152 SMs x 128 FP32 lanes x 2 x %.0f MHz" % smax}
    if bound == "hbm":
        ach = work / t_s / 1e9
        return {"bound": "hbm", "kernel": stage, "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": ach / hbm, "work_per_launch": desc, "peak_source": src}
    return None


def recorded_traffic(stage):
    """DRAM bytes per launch recorded by an ncu capture of the current kernel
    source (profiles/<stage>_traffic.txt: 'source_sha256 <hex>' and
    'dram_bytes <n>'); None when absent or taken on another version."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "%s_traffic.txt" % stage)
    try:
        rec = dict(line.split(None, 1) for line in open(path).read().splitlines() if line.strip()
                   and not line.startswith("#"))
        src = os.path.join(ROOT, "paper_2412_04595_gb300", "csrc", "sog_kernels.cu")
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
        if rec.get("source_sha256", "").strip() != sha:
            return None
        return float(rec["dram_bytes"])
    except Exception:
        return None


def run_ours(args, wl, rank, world):
    import numpy as np
    import torch
    import __graft_entry__ as g
    from paper_2412_04595_gb300 import binding as B, workloads

    g.build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    N, L, tol = wl["N"], wl["L"], wl["tol"]
    prec = B.SOG_PREC_FP64 if args.precision == "fp64" else B.SOG_PREC_MIXED
    np_dt = np.float64 if prec == B.SOG_PREC_FP64 else np.float32
    q, r = workloads.uniform_neutral(N, L, wl["seed"], dtype=np_dt)
    plan = B.Plan(N, L, tol, precision=prec, n_nb=args.n_nb)
    dt = plan.dtype
    qt = torch.tensor(q, device=dev)
    rt = torch.tensor(r, device=dev)
    phi = torch.empty(N, dtype=dt, device=dev)
    F = torch.empty(N, 3, dtype=dt, device=dev)
    E = torch.zeros(1, dtype=torch.float64, device=dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    plan.set_timing(True)
    for _ in range(args.warmup):
        flush.fill_(1)
        plan.eval(qt, rt, phi, E, F, stream=stream)
    torch.cuda.synchronize()
    if plan.check() != 0:
        raise RuntimeError("evaluation reported a data error")
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index)
    clocks.start()
    times = []
    stages = {}
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.eval(qt, rt, phi, E, F, stream=stream)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        for k, v in plan.timing().items():
            stages.setdefault(k, []).append(v)
    torch.cuda.synchronize()
    launches = plan.launches() * args.steps
    clk = clocks.stop()
    total_ms = max_over_ranks(sum(times), dev)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    value = world * N * args.steps / (total_ms * 1e-3)
    stage_ms = {k: sum(v) / len(v) for k, v in stages.items()}

    # end to end through the host entry point (pinned buffers, H2D + D2H inside)
    qh = torch.tensor(q).pin_memory()
    rh = torch.tensor(r).pin_memory()
    phih = torch.empty(N, dtype=dt).pin_memory()
    Fh = torch.empty(N, 3, dtype=dt).pin_memory()
    Eh = torch.empty(1, dtype=torch.float64).pin_memory()
    plan.set_timing(False)
    for _ in range(2):
        plan.eval_host(qh, rh, phih, Eh, Fh)
    e2e_s = 0.0
    for _ in range(args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = plan.eval_host(qh, rh, phih, Eh, Fh)
        e2e_s += time.perf_counter() - t0
        if st != 0:
            raise RuntimeError("sog_eval_host status %d" % st)
    es = q.dtype.itemsize
    e2e = {"value": N * args.steps / e2e_s, "unit": "particles/s",
           "h2d_bytes_per_step": int(N * 4 * es), "d2h_bytes_per_step": int(N * 4 * es + 8)}

    out = dict(plan=plan, stage_ms=stage_ms, value=value, total_ms=total_ms, times=times,
               launches=launches, clocks=clk, e2e=e2e, E=float(Eh[0]), F=Fh.numpy().astype(np.float64),
               phi=phih.numpy().astype(np.float64), q=q, r=r)
    return out


def oracle_run(prm, q, r):
    import oracle
    from oracle import sog as osog
    oracle.build_oracle()
    t0 = time.perf_counter()
    ref = osog.sog_eval(prm, q.astype("float64"), r.astype("float64"))
    return ref, time.perf_counter() - t0, oracle.num_threads()


def max_over_ranks(x: float, device) -> float:
    """Largest value of x over the ranks of the current process group (x
    itself without one); device: where the reduction tensor lives (CUDA for
    NCCL, CPU for gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def emit(d):
    print(json.dumps(d), flush=True)


def run_batched(args, wl, config, rank, world):
    """Batched workload: the systems in one sog_batch_eval per GPU (mixed
    precision), compared with a loop of per-system FP64 evaluations on the
    same GPU.  With several ranks the fixed set of systems is split between
    them (balanced shares, no exchange): strong scaling."""
    import numpy as np
    import torch
    import __graft_entry__ as g
    from paper_2412_04595_gb300 import binding as B, workloads

    g.build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    # positions rounded to FP32 once, so that both arms see the same inputs
    systems = [(qq, rr.astype(np.float32).astype(np.float64), LL)
               for qq, rr, LL in workloads.batched_slabs(wl["batch"], seed=wl["seed"])]
    Ntot = sum(s[0].size for s in systems)          # the whole job, all ranks
    from paper_2412_04595_gb300.sharding import shard_systems
    mine = shard_systems([s[0].size for s in systems], world)[rank]
    systems = [systems[i] for i in mine]
    prec = B.SOG_PREC_FP64 if args.precision == "fp64" else B.SOG_PREC_MIXED
    batch = B.Batch([(s[0].size, s[2]) for s in systems], wl["tol"], precision=prec)
    dt = batch.dtype
    q = [torch.tensor(s[0], dtype=dt, device=dev) for s in systems]
    r = [torch.tensor(s[1], dtype=dt, device=dev) for s in systems]
    phi = [torch.empty(s[0].size, dtype=dt, device=dev) for s in systems]
    F = [torch.empty(s[0].size, 3, dtype=dt, device=dev) for s in systems]
    E = torch.zeros(len(systems), dtype=torch.float64, device=dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        flush.fill_(1)
        batch.eval(q, r, phi, E, F, stream=stream)
    torch.cuda.synchronize()
    st, bad = batch.check()
    if st != 0:
        raise RuntimeError("system %d reported status %d" % (bad, st))
    steps = max(3, min(args.steps, 200))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index)
    clocks.start()
    t = 0.0
    for _ in range(steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        batch.eval(q, r, phi, E, F, stream=stream)
        e1.record(stream)
        e1.synchronize()
        t += e0.elapsed_time(e1)
    clk = clocks.stop()
    t = max_over_ranks(t, dev)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    value = Ntot * steps / (t * 1e-3)
    launches = batch.launches() * steps
    # the plain form: one FP64 plan per system, evaluated one after another
    plans = [B.Plan(s[0].size, s[2], wl["tol"], precision=B.SOG_PREC_FP64) for s in systems]
    q64 = [torch.tensor(s[0], dtype=torch.float64, device=dev) for s in systems]
    r64 = [torch.tensor(s[1], dtype=torch.float64, device=dev) for s in systems]
    phi64 = [torch.empty(s[0].size, dtype=torch.float64, device=dev) for s in systems]
    F64 = [torch.empty(s[0].size, 3, dtype=torch.float64, device=dev) for s in systems]
    E64 = torch.zeros(len(systems), dtype=torch.float64, device=dev)

    def loop64():
        for i, p in enumerate(plans):
            p.eval(q64[i], r64[i], phi64[i], E64[i:i + 1], F64[i], stream=stream)

    for _ in range(2):
        flush.fill_(1)
        loop64()
    torch.cuda.synchronize()
    steps64 = max(3, min(steps, 20))
    t64 = 0.0
    for _ in range(steps64):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        loop64()
        e1.record(stream)
        e1.synchronize()
        t64 += e0.elapsed_time(e1)
    t64 = max_over_ranks(t64, dev)
    value64 = Ntot * steps64 / (t64 * 1e-3)
    relE = (E.double() - E64).abs() / E64.abs()
    # energy error against the energy's own scale (1/2) sum |q_i phi_i|: the
    # relative error of E is large only where the total nearly cancels
    escale = torch.stack([0.5 * (q64[i] * phi64[i]).abs().sum() for i in range(len(systems))])
    errE_scale = (E.double() - E64).abs() / escale
    rmsF = torch.stack([((F[i].double() - F64[i]) ** 2).sum() / (F64[i] ** 2).sum()
                        for i in range(len(systems))]).sqrt()
    for p in plans:
        p.close()
    if rank != 0:
        return
    config = dict(config, N=Ntot, L=None, systems=wl["batch"],
                  parallelism="systems split over %d GPU(s), no exchange" % world)
    emit({"metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": world, "steps": steps,
          "warmup": args.warmup, "ms_per_step": t / steps, "higher_is_better": True,
          "scaling": "strong", "vs_baseline": None,
          "dtype": "f32" if args.precision == "mixed" else "f64", "data": "synthetic",
          "config": config, "gpu_launches": launches, "clocks": clk,
          "plain_fp64_loop": {"value": value64, "unit": "particles/s",
                              "ms_per_step": t64 / steps64,
                              "desc": "one FP64 plan per system, sog_eval one system after another"},
          "speedup_vs_plain_fp64_loop": value / value64,
          "accuracy_vs_fp64_gpu": {"energy_rel_median": float(relE.median()),
                                   "energy_rel_max": float(relE.max()),
                                   "energy_err_over_sum_abs_q_phi_max": float(errE_scale.max()),
                                   "rms_force_median": float(rmsF.median()),
                                   "rms_force_max": float(rmsF.max()),
                                   "note": "per system, same FP32-rounded inputs; the FP64 GPU "
                                           "path matches the FP64 oracle to 1e-10"}})


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1500)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="c2")
    ap.add_argument("--precision", choices=("mixed", "fp64"), default="mixed")
    ap.add_argument("--n-nb", dest="n_nb", type=float, default=120.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    wl = WORKLOADS[args.workload]
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    config = {"workload": wl["desc"], "N": wl["N"], "L": list(wl["L"]), "tol": wl["tol"],
              "precision": args.precision, "n_nb": args.n_nb,
              "l2": "flushed between steps (%d MiB write)" % (FLUSH_BYTES >> 20),
              "parallelism": "replicas x%d" % world}

    if args.impl == "reference":
        # the oracle on the host cores, rank 0 only.  Each step evaluates a
        # bounded sample of the workload: a system of the same kind (uniform
        # neutral charges at the same density and box aspect) with N_s
        # particles, N_s chosen from a calibration run so that the whole
        # warm-up + timed run takes about two minutes.
        if rank != 0:
            return
        import numpy as np
        from oracle import sog as osog
        from paper_2412_04595_gb300 import workloads
        N, L = wl["N"], wl["L"]

        def sample(ns):
            f = (ns / N) ** (1.0 / 3.0)
            Ls = tuple(x * f for x in L)
            q, r = workloads.uniform_neutral(ns, Ls, wl["seed"])
            return osog.select_params(ns, *Ls, wl["tol"], n_nb=args.n_nb), q, r

        n_cal = min(N, 4000)
        prm, q, r = sample(n_cal)
        _, t_cal, cores = oracle_run(prm, q, r)
        budget = 120.0 / (args.steps + args.warmup)
        ns = int(max(500, min(N, n_cal * budget / max(t_cal, 1e-9))))
        ns -= ns % 2
        prm, q, r = sample(ns)
        for _ in range(args.warmup):
            oracle_run(prm, q, r)
        t = 0.0
        for _ in range(args.steps):
            _, dt, cores = oracle_run(prm, q, r)
            t += dt
        value = ns * args.steps / t
        desc = ("FP64 oracle, one evaluation of a %d-particle system of the same kind "
                "(same density and box aspect) per step" % ns)
        emit({"impl": "reference", "metric": METRIC, "value": value, "unit": "particles/s",
              "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
              "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
              "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
              "cpu_baseline": {"value": value, "unit": "particles/s", "cores": cores, "kind": "oracle",
                               "sample": desc},
              "e2e": {"value": value, "unit": "particles/s", "h2d_bytes_per_step": 0,
                      "d2h_bytes_per_step": 0}})
        return

    if "batch" in wl:
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("nccl")
        run_batched(args, wl, config, rank, world)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    res = run_ours(args, wl, rank, world)
    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    import numpy as np
    plan = res["plan"]
    prm = plan.params
    N = wl["N"]
    hbm, smax, src = peaks()
    fp32_peak = 152 * 128 * 2 * smax * 1e6 / 1e12          # TFLOP/s at the max SM clock
    dom = DOMINANT if DOMINANT in res["stage_ms"] else max(res["stage_ms"], key=res["stage_ms"].get)
    roof = roofline_entry(prm, N, dom, res["stage_ms"][dom] * 1e-3, hbm, fp32_peak, smax, src)
    if roof is not None:
        roof["traffic"] = recorded_traffic(dom)
    others = [roofline_entry(prm, N, k, v * 1e-3, hbm, fp32_peak, smax, src)
              for k, v in res["stage_ms"].items() if k != dom and v > 0]
    line = {"metric": METRIC, "value": res["value"], "unit": "particles/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": res["total_ms"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "mixed" else "f64",
            "data": "synthetic", "config": config, "e2e": res["e2e"],
            "gpu_launches": res["launches"], "clocks": res["clocks"], "roofline": roof,
            "roofline_stages": [o for o in others if o is not None],
            "stage_ms": {k: round(v, 5) for k, v in res["stage_ms"].items()},
            "params": {k: prm[k] for k in ("rc", "M", "m", "I", "P_win", "I_long", "P_cheb",
                                           "long_direct")}}
    if not args.no_cpu_baseline:
        from oracle import sog as osog
        oprm = osog.select_params(N, *wl["L"], wl["tol"], n_nb=args.n_nb)
        ref, t_or, cores = oracle_run(oprm, res["q"], res["r"])
        line["cpu_baseline"] = {"value": N / t_or, "unit": "particles/s", "cores": cores,
                                "kind": "oracle",
                                "sample": "the full workload once (FP64 oracle, same inputs and parameters)"}
        Fr = ref["F"]
        line["accuracy_vs_oracle"] = {
            "rel_energy": abs(res["E"] - ref["E"]) / abs(ref["E"]),
            "rms_force": float(math.sqrt(np.mean(np.sum((res["F"] - Fr) ** 2, 1)) /
                                         np.mean(np.sum(Fr ** 2, 1)))),
            # the paper's measure: largest potential error relative to the largest potential
            "rel_linf_potential": float(np.max(np.abs(res["phi"] - ref["phi"])) /
                                        np.max(np.abs(ref["phi"])))}
    emit(line)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
