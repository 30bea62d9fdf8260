#!/usr/bin/env python3
"""Throughput benchmark of the spectral SOG evaluation (energy + forces).

One step = one sog_eval call over the whole hot path (binning, near field,
mid range, long range and its k = 0 mode, assembly) on the workload below,
with inputs resident on the device.  Prints one JSON line.

Default workload ("c3_slab"): a thin slab, N = 1e6 neutral +-1 charges at
uniform positions in a 1000 x 1000 x 10 box, periodic in x and y and free in
z, relative tolerance 1e-6, mixed precision (FP32 bulk; FP64 tables, k = 0
mode and reductions).  It is the largest configuration at the 1e-6 error of
the metric; its long range takes the gridded form (Algorithm 2).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME] [--precision mixed|fp64]

Besides the timed value the line reports: the same workload through an FP64
plan (plain_fp64); accuracy against the FP64 oracle on sampled targets and
against Ewald2D (the true quasi-2D sum) on a few targets; isolated per-stage
times and their rooflines against measured peaks; the end-to-end rate through
the host entry point; and the oracle's rate on a bounded sample of the
workload on the host cores.

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
    "c3_slab": dict(N=1000000, L=(1000.0, 1000.0, 10.0), tol=1e-6, seed=3, kind="uniform",
                    keep_z=True,
                    desc="thin slab: 1e6 uniform neutral +-1 charges, box 1000x1000x10 "
                         "(periodic x,y, free z), tol 1e-6"),
    "c3_tall": dict(N=1000000, L=(50.0, 50.0, 2000.0), tol=1e-6, seed=3, kind="uniform",
                    keep_z=False,
                    desc="tall cell: 1e6 uniform neutral +-1 charges, box 50x50x2000, tol 1e-6"),
    "c4": dict(N=4000000, L=(400.0, 400.0, 100.0), tol=1e-5, seed=3, kind="edl", keep_z=True,
               desc="electric double layer: 4e6 charges, cations ~exp(-z/2) at one wall, anions at "
                    "the other, half uniform bulk, box 400x400x100, tol 1e-5"),
    "c2": dict(N=100000, L=(100.0, 100.0, 100.0), tol=1e-6, seed=1, kind="uniform", keep_z=False,
               desc="uniform neutral +-1 charges, N=1e5, box 100x100x100, tol 1e-6"),
    "c2_1e4": dict(N=100000, L=(100.0, 100.0, 100.0), tol=1e-4, seed=1, kind="uniform",
                   keep_z=False,
                   desc="uniform neutral +-1 charges, N=1e5, box 100x100x100, tol 1e-4"),
    "c1": dict(N=1000, L=(10.0, 10.0, 10.0), tol=1e-6, seed=1, kind="uniform", keep_z=False,
               desc="uniform neutral +-1 charges, N=1e3, box 10x10x10, tol 1e-6"),
    "c5": dict(batch=256, seed=5, tol=1e-6, N=None, L=(0.0, 0.0, 0.0),
               desc="256 independent neutral +-1 systems, N log-uniform in [500, 50000], "
                    "density 0.1, Lz/Lx uniform in [0.05, 10], tol 1e-6, one graph launch"),
}
DEFAULT_WORKLOAD = "c3_slab"
FLUSH_BYTES = 512 << 20          # larger than the 129 MB L2, written between steps
N_ORACLE_TARGETS = 2000          # sampled targets compared with the FP64 oracle
N_TRUTH_TARGETS = 100            # targets compared with Ewald2D
CPU_SAMPLE_SECONDS = 15.0        # oracle work of the CPU baseline's bounded sample
# FP32 operations the near field must do (the per-unit counts of the method,
# not of this implementation): 8 per candidate of the 27-cell neighbourhood
# (3 differences, squared distance, comparison) and 30 per pair inside r_c
# (distance, reciprocal, kernel value and derivative, potential and force).
# neighbour counts whose analytic parameters sog_tune_cutoff times
CUTOFF_CANDIDATES = (80.0, 100.0, 120.0, 140.0, 160.0, 200.0, 240.0, 280.0, 320.0)
CAND_FLOP = 8
PAIR_FLOP = 30


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return 6800.0, "fallback"


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


def make_system(wl, N=None, seed=None):
    """Charges and positions of the workload (FP32-rounded positions, as both
    the mixed plan and the oracle see them).  With N below the workload's,
    a system of the same kind: same density, the slab and double layer keep
    their height, the others their aspect ratio."""
    import numpy as np
    from paper_2412_04595_gb300 import workloads
    N0, L0 = wl["N"], wl["L"]
    N = N0 if N is None else N
    if N == N0:
        L = tuple(L0)
    elif wl["keep_z"]:
        f = (N / N0) ** 0.5
        L = (L0[0] * f, L0[1] * f, L0[2])
    else:
        f = (N / N0) ** (1.0 / 3.0)
        L = tuple(x * f for x in L0)
    gen = workloads.uniform_neutral if wl["kind"] == "uniform" else workloads.edl_neutral
    q, r = gen(N, L, wl["seed"] if seed is None else seed, dtype=np.float32)
    return q, r, L


def near_counts(prm, r, samples=20000, seed=0):
    """Candidate tests and pairs of the near field on the actual positions:
    candidates = sum over cells of (charges in the cell) x (charges in its
    neighbour cells), the cells being the r_c-wide cells of the cell list
    (Sec. 2.2); pairs = N x the mean number of neighbours within r_c of
    `samples` random charges (k-d tree, minimum image in x, y).  None when
    scipy is missing (the uniform-density estimate is used instead)."""
    import numpy as np
    try:
        from scipy.spatial import cKDTree
    except ImportError:
        return None
    L, rc = prm["L"], prm["rc"]
    N = r.shape[0]
    pts = r.astype(np.float64) + np.array([0.5 * L[0], 0.5 * L[1], 0.5 * L[2]])
    pts[:, 0] %= L[0]
    pts[:, 1] %= L[1]
    pts[:, 2] = np.clip(pts[:, 2], 0.0, L[2])
    nc = [max(1, int(math.floor(L[d] / rc))) for d in range(3)]
    ci = [np.minimum((pts[:, d] * (nc[d] / L[d])).astype(np.int64), nc[d] - 1) for d in range(3)]
    H = np.zeros((nc[2], nc[1], nc[0]))
    np.add.at(H, (ci[2], ci[1], ci[0]), 1.0)
    Hn = np.zeros_like(H)
    # periodic x, y: the three neighbouring columns, or every column when
    # there are fewer than three (the kernel's minimum-image case); z: the
    # cells above and below, where they exist
    for dz in ((-1, 0, 1) if nc[2] > 1 else (0,)):
        for dy in ((-1, 0, 1) if nc[1] >= 3 else range(nc[1])):
            for dx in ((-1, 0, 1) if nc[0] >= 3 else range(nc[0])):
                sh = np.roll(np.roll(H, dy, axis=1), dx, axis=2)
                if dz == 1:
                    sh = np.concatenate([np.zeros_like(sh[:1]), sh[:-1]], 0)
                elif dz == -1:
                    sh = np.concatenate([sh[1:], np.zeros_like(sh[:1])], 0)
                Hn += sh
    cand = float((H * Hn).sum())
    tree = cKDTree(pts, boxsize=[L[0], L[1], L[2] + 2.0 * rc + 1.0])
    idx = np.random.default_rng(seed).choice(N, min(N, samples), replace=False)
    nb = tree.query_ball_point(pts[idx], rc, return_length=True) - 1
    return {"cand": cand, "pairs": float(nb.mean()) * N, "sampled": int(idx.size)}


def stage_work(prm, N, stage, es, counts=None):
    """Algorithmic work of one launch of a stage and the resource bounding it:
    ("alu", FP32 operations), ("hbm", bytes) or (None, None), with its
    description.  es: bytes per element of the plan's type.  counts: the
    near field's candidates and pairs on the actual positions (near_counts);
    None: the uniform-density estimate."""
    Ix, Iy, Iz = prm["I"]
    P, Pc, Pl = prm["P_win"], prm["P_cheb"], prm["P_long"]
    L = prm["L"]
    rho = N / (L[0] * L[1] * L[2])
    if stage == "near":
        if counts is not None:
            cand, pairs, how = counts["cand"], counts["pairs"], "counted on the positions"
        else:
            pairs = N * 4.0 / 3.0 * math.pi * prm["rc"] ** 3 * rho
            nc = [max(1, int(math.floor(L[d] / prm["rc"]))) for d in range(3)]
            ext = [min(3, nc[d]) for d in range(3)]
            cand = N * ext[0] * ext[1] * ext[2] * N / (nc[0] * nc[1] * nc[2])
            how = "uniform-density estimate"
        return ("alu", cand * CAND_FLOP + pairs * PAIR_FLOP,
                "FP32 flop: %.4g candidate tests (27-cell neighbourhoods) x %d + %.4g pairs "
                "within r_c x %d (%s)" % (cand, CAND_FLOP, pairs, PAIR_FLOP, how))
    if stage == "binning":
        sets = 1 + (prm["m"] >= 0) + (prm["m"] < prm["M"] and not prm["long_direct"])
        return ("hbm", N * (4 * es + sets * 17 * es),
                "bytes: q, r read; per bin set key, rank, record written and read, sorted record "
                "and permutation written (%d sets)" % sets)
    if stage == "mid_spread":
        return "alu", N * P ** 3 * 2.0, "FP32 flop: N x P^3 x 2"
    if stage == "mid_gather":
        return "alu", N * P ** 3 * 4.0, "FP32 flop: N x P^3 x 4 (value and x-derivative sums)"
    if stage == "mid_fft":
        half = Iz * Iy * (Ix // 2 + 1)
        return ("hbm", 3 * 2 * half * 2 * es + half * es,
                "bytes: 3 passes x (read + write) of the complex half spectrum + scaling table")
    if stage == "long_spread":
        return "alu", N * Pc * Pl * Pl * 2.0, "FP32 flop: N x P_cheb x P_long^2 x 2"
    if stage == "long_gather":
        return "alu", N * Pc * Pl * Pl * 4.0, "FP32 flop: N x P_cheb x P_long^2 x 4"
    if stage == "long_fft":
        Ilx, Ily = prm["I_long"]
        planes = Pc * Ily * (Ilx + 2) * es
        return ("hbm", 6 * planes,
                "bytes: x pass, fused y pass with contraction, backward x pass: "
                "3 x (read + write) of the %d proxy planes" % Pc)
    if stage in ("long_moments", "long_eval"):
        Kx, Ky = (prm["I_long"][0] - 1) // 2, (prm["I_long"][1] - 1) // 2
        nh = Ky + Kx * (2 * Ky + 1)
        k = 4.0 if stage == "long_moments" else 8.0
        return ("alu", N * nh * Pc * k, "FP32 flop: N x half-plane modes x P_cheb x %d" % k)
    if stage == "assemble":
        return ("hbm", N * (16 * 8 + 5 * es),
                "bytes: four parts and their gradients (FP64) read, q read, phi and F written")
    return None, None, None


def roofline_entry(prm, N, stage, t_s, es, peaks, counts=None):
    bound, work, desc = stage_work(prm, N, stage, es, counts)
    if bound == "alu":
        peak, src = peaks["fp32_tflops"] if es == 4 else peaks["fp64_tflops"], peaks["alu_src"]
        ach = work / t_s / 1e12
        return {"bound": "alu", "kernel": stage, "achieved": ach, "peak": peak,
                "unit": "TFLOP/s", "frac": ach / peak, "work_per_launch": desc,
                "launch_ms": t_s * 1e3, "peak_source": src + (" FP32" if es == 4 else " FP64")}
    if bound == "hbm":
        ach = work / t_s / 1e9
        return {"bound": "hbm", "kernel": stage, "achieved": ach, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": ach / peaks["hbm_gbs"], "work_per_launch": desc,
                "launch_ms": t_s * 1e3, "peak_source": peaks["hbm_src"]}
    return None


def recorded_traffic(stage, workload):
    """DRAM bytes per launch recorded by an ncu capture of the current kernel
    sources (profiles/traffic_<stage>_<workload>.txt: 'source_sha256 <hex>'
    and 'dram_bytes <n>'); None when absent or taken on other sources."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic_%s_%s.txt" % (stage, workload))
    try:
        rec = dict(line.split(None, 1) for line in open(path).read().splitlines() if line.strip()
                   and not line.startswith("#"))
        h = hashlib.sha256()
        for f in ("sog_kernels.cu", "sog_fft.cu"):
            h.update(open(os.path.join(ROOT, "paper_2412_04595_gb300", "csrc", f), "rb").read())
        if rec.get("source_sha256", "").strip() != h.hexdigest():
            return None
        return float(rec["dram_bytes"])
    except Exception:
        return None


def timed_steps(fn, steps, stream, flush):
    """Device milliseconds of each of `steps` calls of fn, L2 flushed before
    each, CUDA events on `stream`."""
    import torch
    out = []
    for _ in range(steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        out.append(e0.elapsed_time(e1))
    return out


def run_ours(args, wl, rank, world):
    import numpy as np
    import torch
    import __graft_entry__ as g
    from paper_2412_04595_gb300 import binding as B

    g.build()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    N, L, tol = wl["N"], wl["L"], wl["tol"]
    prec = B.SOG_PREC_FP64 if args.precision == "fp64" else B.SOG_PREC_MIXED
    q, r, _ = make_system(wl)
    q = q.astype(np.float64) if prec == B.SOG_PREC_FP64 else q
    r = r.astype(np.float64) if prec == B.SOG_PREC_FP64 else r
    qt = torch.tensor(q, device=dev)
    rt = torch.tensor(r, device=dev)
    cutoff = None
    n_nb = args.n_nb
    if not args.no_tune_cutoff:
        # Sec. 4.3: the cutoff chosen by the run time of the evaluation (each
        # candidate neighbour count through the analytic selection, timed on
        # this workload; excluded from the timed region, like plan creation)
        t0 = time.perf_counter()
        n_nb, ms = B.sog_tune_cutoff(N, L, tol, qt, rt, CUTOFF_CANDIDATES, reps=3, precision=prec)
        cutoff = {"n_nb": n_nb, "candidates_ms": {"%g" % k: round(v, 4) for k, v in ms.items()},
                  "analytic_default_n_nb": args.n_nb, "seconds": time.perf_counter() - t0,
                  "desc": "sog_tune_cutoff: median evaluation time of each candidate neighbour "
                          "count's analytic parameters; the fastest is used"}
    plan = B.Plan(N, L, tol, precision=prec, n_nb=n_nb)
    dt = plan.dtype
    tune = None
    if not args.no_autotune:
        # tile edges and CTAs per tile timed on this workload (excluded from
        # the timed region, like the plan's creation)
        t0 = time.perf_counter()
        tiles = plan.autotune(qt, rt, reps=3)
        tune = dict(tiles, seconds=time.perf_counter() - t0)
    phi = torch.empty(N, dtype=dt, device=dev)
    F = torch.empty(N, 3, dtype=dt, device=dev)
    E = torch.zeros(1, dtype=torch.float64, device=dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        plan.eval(qt, rt, phi, E, F, stream=stream)

    for _ in range(args.warmup):
        flush.fill_(1)
        step()
    torch.cuda.synchronize()
    if plan.check() != 0:
        raise RuntimeError("evaluation reported a data error")
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index)
    clocks.start()
    times = timed_steps(step, args.steps, stream, flush)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = plan.launches() * args.steps
    total_ms = max_over_ranks(sum(times), dev)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    value = world * N * args.steps / (total_ms * 1e-3)
    phi_h = phi.double().cpu().numpy()
    F_h = F.double().cpu().numpy()
    E_h = float(E.item())

    # isolated stage durations: every stage on this stream, one after another
    plan.set_timing(2)
    stages = {}
    for _ in range(max(3, min(args.steps, 20))):
        flush.fill_(1)
        step()
        torch.cuda.synchronize()
        for k, v in plan.timing().items():
            stages.setdefault(k, []).append(v)
    plan.set_timing(0)
    stage_ms = {k: float(np.median(v)) for k, v in stages.items()}

    # end to end through the host entry point (pinned buffers, H2D + D2H inside)
    qh = torch.tensor(q).pin_memory()
    rh = torch.tensor(r).pin_memory()
    phih = torch.empty(N, dtype=dt).pin_memory()
    Fh = torch.empty(N, 3, dtype=dt).pin_memory()
    Eh = torch.empty(1, dtype=torch.float64).pin_memory()
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
    prm = plan.params

    # the plain FP64 form: the same workload and parameters through an FP64 plan
    plain = None
    if prec != B.SOG_PREC_FP64 and not args.no_plain_fp64:
        p64 = B.Plan(N, L, tol, precision=B.SOG_PREC_FP64, manual=prm)
        q64 = torch.tensor(q.astype(np.float64), device=dev)
        r64 = torch.tensor(r.astype(np.float64), device=dev)
        phi64 = torch.empty(N, dtype=torch.float64, device=dev)
        F64 = torch.empty(N, 3, dtype=torch.float64, device=dev)
        E64 = torch.zeros(1, dtype=torch.float64, device=dev)

        def step64():
            p64.eval(q64, r64, phi64, E64, F64, stream=stream)

        for _ in range(2):
            flush.fill_(1)
            step64()
        torch.cuda.synchronize()
        s64 = max(3, min(args.steps, 10))
        t64 = sum(timed_steps(step64, s64, stream, flush))
        if p64.check() != 0:
            raise RuntimeError("FP64 evaluation reported a data error")
        plain = {"value": N * s64 / (t64 * 1e-3), "unit": "particles/s", "ms_per_step": t64 / s64,
                 "steps": s64, "dtype": "f64",
                 "desc": "the same workload, inputs and parameters through an FP64 plan",
                 "phi": phi64.cpu().numpy(), "F": F64.cpu().numpy(), "E": float(E64.item())}
        p64.close()
    md = None
    if not args.no_md:
        md = md_rate(B, plan, q, r, dev, stream, flush)
    plan.close()
    return dict(prm=prm, stage_ms=stage_ms, value=value, total_ms=total_ms, launches=launches,
                md=md, tune=tune, cutoff=cutoff,
                clocks=clk, e2e=e2e, E=E_h, F=F_h, phi=phi_h, q=q, r=r, plain=plain, es=es)


def md_rate(B, plan, q, r, dev, stream, flush, steps=50, sort_every=10):
    """Velocity-Verlet steps through sog_md_step on the workload (the plan
    reused, particles re-sorted into cell order every sort_every steps):
    steps per second, L2 flushed before each timed block of sort_every steps."""
    import numpy as np
    import torch
    N = plan.N
    rng = np.random.default_rng(11)
    qt = torch.tensor(q, device=dev)
    rt = torch.tensor(r, device=dev)
    vt = torch.tensor(rng.normal(0.0, 0.05, (N, 3)).astype(q.dtype), device=dev)
    F = torch.empty(N, 3, dtype=plan.dtype, device=dev)
    E = torch.zeros(1, dtype=torch.float64, device=dev)
    order = torch.arange(N, dtype=torch.int32, device=dev)
    plan.eval(qt, rt, None, E, F, stream=stream)
    md = B.MD(plan)
    md.step(qt, rt, vt, F, 1e-4, nsteps=2 * sort_every, E=E, sort_every=sort_every, order=order,
            stream=stream)
    torch.cuda.synchronize()
    blocks = max(1, steps // sort_every)
    ms = sum(timed_steps(lambda: md.step(qt, rt, vt, F, 1e-4, nsteps=sort_every, E=E,
                                         sort_every=sort_every, order=order, stream=stream),
                         blocks, stream, flush))
    st = plan.check()
    md.close()
    if st != 0:
        raise RuntimeError("MD steps reported status %d" % st)
    n = blocks * sort_every
    return {"steps_per_s": n / (ms * 1e-3), "particle_steps_per_s": N * n / (ms * 1e-3),
            "ms_per_step": ms / n, "sort_every": sort_every, "steps": n,
            "desc": "sog_md_step: velocity Verlet (kick, drift, evaluation, kick), plan reused, "
                    "particles re-sorted into cell order every %d steps" % sort_every}


def rel_errors(phi, F, ref_phi, ref_F):
    """The paper's measure (largest potential error over the largest
    potential) and the RMS force error relative to the RMS force."""
    import numpy as np
    linf = float(np.max(np.abs(phi - ref_phi)) / np.max(np.abs(ref_phi)))
    rmsF = float(math.sqrt(np.mean(np.sum((F - ref_F) ** 2, 1)) / np.mean(np.sum(ref_F ** 2, 1))))
    return linf, rmsF


def sampled_targets(r, n, seed=7):
    """n random targets plus the particles nearest the walls and box edges."""
    import numpy as np
    N = r.shape[0]
    pick = set(np.random.default_rng(seed).choice(N, min(n, N), replace=False).tolist())
    for col in range(3):
        o = np.argsort(r[:, col])
        pick.update(o[:4].tolist())
        pick.update(o[-4:].tolist())
    return np.array(sorted(pick), dtype=np.int64)


def accuracy(res, wl):
    """Errors of the GPU results against the FP64 oracle (same parameters,
    sampled targets) and against Ewald2D (the true quasi-2D sum)."""
    import numpy as np
    import oracle
    from oracle import sog as osog
    oracle.build_oracle()
    q = res["q"].astype(np.float64)
    r = res["r"].astype(np.float64)
    tgt = sampled_targets(r, N_ORACLE_TARGETS)
    t0 = time.perf_counter()
    ref = osog.sog_eval(res["prm"], q, r, tgt)
    t_or = time.perf_counter() - t0
    linf, rmsF = rel_errors(res["phi"][tgt], res["F"][tgt], ref["phi"], ref["F"])
    out = {"vs_oracle": {"targets": int(tgt.size), "rel_linf_potential": linf, "rms_force": rmsF,
                         "oracle_seconds": t_or,
                         "desc": "FP64 oracle with the plan's parameters on sampled targets "
                                 "(random plus those nearest the walls and box edges)"}}
    if res["plain"] is not None:
        l64, f64 = rel_errors(res["plain"]["phi"][tgt], res["plain"]["F"][tgt], ref["phi"], ref["F"])
        out["vs_oracle"]["plain_fp64_rel_linf_potential"] = l64
        out["vs_oracle"]["plain_fp64_rms_force"] = f64
        out["rel_energy_vs_plain_fp64"] = abs(res["E"] - res["plain"]["E"]) / abs(res["plain"]["E"])
    tt = tgt[:: max(1, tgt.size // N_TRUTH_TARGETS)][:N_TRUTH_TARGETS]
    L = res["prm"]["L"]
    t0 = time.perf_counter()
    ph_true, g_true = osog.ewald2d(q, r, L, tt, alpha=1.5 / min(L[0], L[1]))
    t_ew = time.perf_counter() - t0
    lt, ft = rel_errors(res["phi"][tt], res["F"][tt], ph_true, -q[tt, None] * g_true)
    out["vs_truth"] = {"targets": int(tt.size), "rel_linf_potential": lt, "rms_force": ft,
                       "ewald_seconds": t_ew, "tol": wl["tol"],
                       "desc": "Ewald2D (Parry's sum, the paper's reference) on sampled targets; "
                               "rel_linf_potential is the paper's error measure"}
    return out


def cpu_baseline(wl, args):
    """The FP64 oracle on the host cores on a bounded sample: one evaluation
    of a system of the same kind (same density and shape) with N_s charges,
    N_s chosen from a calibration run so that it takes about
    CPU_SAMPLE_SECONDS."""
    import oracle
    from oracle import sog as osog
    oracle.build_oracle()

    def run(ns):
        q, r, L = make_system(wl, ns)
        prm = osog.select_params(ns, *L, wl["tol"], n_nb=args.n_nb)
        t0 = time.perf_counter()
        osog.sog_eval(prm, q.astype("float64"), r.astype("float64"))
        return time.perf_counter() - t0

    # calibrate twice: the grid work grows like N, the oracle's direct near
    # field like N^2, so the second estimate is taken from a larger system
    ns = min(wl["N"], 4000)
    t = run(ns)
    for _ in range(2):
        nxt = int(max(1000, min(wl["N"], ns * CPU_SAMPLE_SECONDS / max(t, 1e-9))))
        nxt -= nxt % 2
        if abs(nxt - ns) < 0.2 * ns:
            break
        ns = nxt
        t = run(ns)
    return ns, t, oracle.num_threads()


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


def measured_peaks():
    from paper_2412_04595_gb300 import binding as B
    hbm, hsrc = hbm_peak()
    return {"hbm_gbs": hbm, "hbm_src": hsrc,
            "fp32_tflops": B.sog_measure_fma_peak(B.SOG_PREC_MIXED),
            "fp64_tflops": B.sog_measure_fma_peak(B.SOG_PREC_FP64),
            "alu_src": "measured on this GPU by sog_measure_fma_peak (independent FMA chains)"}


def run_reference(args, wl, config, rank):
    """The oracle on the host cores (rank 0 only): each step one evaluation
    of a bounded sample of the workload, a system of the same kind with N_s
    charges, N_s chosen so that the whole run takes about two minutes."""
    if rank != 0:
        return
    import oracle
    from oracle import sog as osog
    oracle.build_oracle()
    if "batch" in wl:
        wl = dict(WORKLOADS["c2"], desc=wl["desc"])

    def sample(ns):
        q, r, L = make_system(wl, ns)
        return osog.select_params(ns, *L, wl["tol"], n_nb=args.n_nb), q, r

    def run(prm, q, r):
        t0 = time.perf_counter()
        osog.sog_eval(prm, q.astype("float64"), r.astype("float64"))
        return time.perf_counter() - t0

    budget = 120.0 / (args.steps + args.warmup)
    ns = min(wl["N"], 4000)
    t = run(*sample(ns))
    for _ in range(2):
        nxt = int(max(500, min(wl["N"], ns * budget / max(t, 1e-9))))
        nxt -= nxt % 2
        if abs(nxt - ns) < 0.2 * ns:
            break
        ns = nxt
        t = run(*sample(ns))
    prm, q, r = sample(ns)
    for _ in range(args.warmup):
        run(prm, q, r)
    t = sum(run(prm, q, r) for _ in range(args.steps))
    value = ns * args.steps / t
    cores = oracle.num_threads()
    desc = ("FP64 oracle, one evaluation of a %d-charge system of the same kind "
            "(same density and shape) per step" % ns)
    emit({"impl": "reference", "metric": METRIC, "value": value, "unit": "particles/s",
          "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
          "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
          "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
          "cpu_baseline": {"value": value, "unit": "particles/s", "cores": cores, "kind": "oracle",
                           "sample": desc},
          "e2e": {"value": value, "unit": "particles/s", "h2d_bytes_per_step": 0,
                  "d2h_bytes_per_step": 0}})


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--precision", choices=("mixed", "fp64"), default="mixed")
    ap.add_argument("--n-nb", dest="n_nb", type=float, default=120.0,
                    help="neighbour count of the analytic cutoff (used with --no-tune-cutoff)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-plain-fp64", action="store_true")
    ap.add_argument("--no-md", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-tune-cutoff", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    wl = WORKLOADS[args.workload]
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    config = {"workload": wl["desc"], "name": args.workload, "N": wl["N"],
              "L": list(wl["L"]), "tol": wl["tol"], "precision": args.precision,
              "n_nb": args.n_nb, "l2": "flushed between steps (%d MiB write)" % (FLUSH_BYTES >> 20),
              "parallelism": "replicas x%d" % world}
    if not args.no_tune_cutoff and "batch" not in wl:
        config["n_nb"] = ("selected by run time among %s (Sec. 4.3; sog_tune_cutoff)"
                          % ", ".join("%g" % c for c in CUTOFF_CANDIDATES))

    if args.impl == "reference":
        run_reference(args, wl, config, rank)
        return

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if "batch" in wl:
        run_batched(args, wl, config, rank, world)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    res = run_ours(args, wl, rank, world)
    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    prm = res["prm"]
    N = wl["N"]
    peaks = measured_peaks()
    counts = near_counts(prm, res["r"]) if res.get("r") is not None else None
    rooflines = [roofline_entry(prm, N, k, v * 1e-3, res["es"], peaks, counts)
                 for k, v in res["stage_ms"].items() if v > 0]
    rooflines = [x for x in rooflines if x is not None]
    # the dominant kernel: the stage with the longest isolated duration
    roof = max(rooflines, key=lambda x: x["launch_ms"]) if rooflines else None
    if roof is not None:
        roof["traffic"] = recorded_traffic(roof["kernel"], args.workload)
        roof["timing"] = ("isolated stage duration: CUDA events around the stage's kernels, "
                          "stages run one after another on the bench's stream, median of steps")
    line = {"metric": METRIC, "value": res["value"], "unit": "particles/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": res["total_ms"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "mixed" else "f64",
            "data": "synthetic", "config": config, "e2e": res["e2e"],
            "gpu_launches": res["launches"], "clocks": res["clocks"], "roofline": roof,
            "roofline_stages": [x for x in rooflines if x is not roof],
            "stage_ms_isolated": {k: round(v, 5) for k, v in res["stage_ms"].items()},
            "peaks": {k: v for k, v in peaks.items()},
            "params": {k: prm[k] for k in ("rc", "M", "m", "I", "P_win", "I_long", "P_long",
                                           "P_cheb", "long_direct")}}
    if res["md"] is not None:
        line["md"] = res["md"]
    if res["tune"] is not None:
        line["autotuned_tiles"] = res["tune"]
    if res["cutoff"] is not None:
        line["cutoff_selection"] = res["cutoff"]
    if res["plain"] is not None:
        line["plain_fp64"] = {k: v for k, v in res["plain"].items() if k not in ("phi", "F", "E")}
        line["speedup_vs_plain_fp64"] = res["value"] / (world * res["plain"]["value"])
    if not args.no_accuracy:
        line["accuracy"] = accuracy(res, wl)
    if not args.no_cpu_baseline:
        ns, t, cores = cpu_baseline(wl, args)
        line["cpu_baseline"] = {"value": ns / t, "unit": "particles/s", "cores": cores,
                                "kind": "oracle",
                                "sample": "one FP64 oracle evaluation of a %d-charge system of the "
                                          "same kind (same density and shape), %.1f s; the "
                                          "oracle's near field is a direct O(N^2) sum" % (ns, t)}
    emit(line)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
