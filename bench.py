"""Benchmark: GS2-preconditioned restarted GMRES on one GB300.

One step = one full solve A x = b from x0 = 0 of the 3D nonsymmetric
convection-diffusion system on a 192^3 grid (first-order upwind, rotating
wind, lognormal cell Peclet numbers, mass term 1; n = 7,077,888,
nnz = 49,324,032, FP64 CSR, b = A x_true, x_true ~ U[-1,1] from the seed),
GMRES(30) right preconditioned by one symmetric GS2 sweep with one inner JR
sweep (SGS2(1,1)), relative residual 1e-8.  Inputs are synthetic (the
paper's model problems, re-synthesised).  The timed region runs with
profiling off; the per-kernel table and the dominant kernel's roofline come
from a second, identical pass.  Extras on the same line: the same workload
with FP32 and FP16 inner sweeps, the 128^3 Laplacian with the same
measurement, the paper's baselines, packs, serving and the elasticity
workload.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
on the host cores on a bounded sample of the same workload instead.
With torchrun (N > 1) every rank solves its own copy on its own GPU
(replicas; the method has no data-path exchange on one matrix per GPU).
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GS2 sweep HBM GB/s (% peak); GMRES solves/s, p50/p99 latency vs plain FP64"
def workload(grid, n, nnz):
    """The headline workload's description at grid^3 (192^3 by default)."""
    return (f"3D upwind convection-diffusion {grid}^3 (n={n:,}, nnz={nnz:,}), rotating "
            "wind, cell Peclet lognormal in [0.1, 10], CSR FP64, b = A x_true, "
            "x_true ~ U[-1,1]; GMRES(30) + SGS2(1,1) FP64, rel. residual 1e-8")


def l2_note(n, nnz):
    """Whether the per-step working set exceeds the 129 MB L2 (the timed
    steps are not separated by an L2 flush)."""
    a_mb = (12 * nnz + 4 * (n + 1)) / 1e6
    tri_mb = (12 * (nnz - n) / 2 + 4 * (n + 1)) / 1e6
    basis_mb = 8 * n * 31 / 1e6
    total = a_mb + 2 * tri_mb + basis_mb
    what = (f"per-step working set (A {a_mb:.0f} MB, D^-1L/D^-1U 2x{tri_mb:.0f} MB, Krylov "
            f"basis {basis_mb:.0f} MB)")
    if total > 129:
        return f"no flush: {what} exceeds the 129 MB L2"
    return f"no flush: {what} fits in the 129 MB L2 (a small-grid run)"
COUNTS_FILE = os.path.join(ROOT, "tests", "golden", "oracle_counts.txt")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.txt")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--grid", type=int, default=192,
                    help="N of the N^3 convection-diffusion grid")
    ap.add_argument("--no-cpu-table", action="store_true",
                    help="skip the oracle's per-configuration sweep and solve table")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the baseline/precision comparison solves")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle sample")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the elasticity 64^3 and convection-diffusion 192^3 runs")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer e2e timing")
    ap.add_argument("--no-serve", action="store_true", help="skip the request-stream run")
    ap.add_argument("--no-autotune", action="store_true", help="keep the heuristic tile shapes")
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests of the served stream")
    ap.add_argument("--serve-rates", default="50,200,1000",
                    help="open-loop Poisson arrival rates (requests/s), comma list")
    ap.add_argument("--serve-forms",
                    default="fp64,fp32,fp32_sweep,fp16_sweep,fp32_sweep_packed,"
                            "fp32_sweep_packed_lanes",
                    help="server forms (inner-sweep precision, packing, small-request "
                         "slots), comma list")
    ap.add_argument("--serve-sweep-forms",
                    default="fp64,fp32_sweep_packed,fp32_sweep_packed_lanes",
                    help="forms that also run the open-loop rate sweep, comma list")
    ap.add_argument("--no-profile", action="store_true",
                    help="do not time kernels with events inside the timed region")
    ap.add_argument("--only-extras", default="",
                    help="comma list: run only these extras (precision, laplacian128, "
                         "comparisons, hybrid, small_system, packs, workloads, serving)")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def stored_count(key):
    """Full-solve iteration counts written by tests/golden/make_oracle_counts.py
    (the oracle only)."""
    if not os.path.exists(COUNTS_FILE):
        return None
    with open(COUNTS_FILE) as f:
        for line in f:
            if line.startswith(key + " "):
                return int(line.split("iters=")[1].split()[0])
    return None


def stored_traffic(kernel, algorithmic_bytes_per_launch, workload=None):
    """Per-launch DRAM bytes of a kernel: the ratio of DRAM bytes to
    algorithmic bytes captured by ncu on a smaller case of the same kernel
    (profiles/traffic.txt; a capture of the same workload family first),
    scaled to this launch's algorithmic bytes (the kernels stream their
    inputs once, so traffic grows in proportion)."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    found = {}
    with open(TRAFFIC_FILE) as f:
        for line in f:
            if line.startswith("#"):
                continue
            parts = dict(kv.split("=", 1) for kv in line.split() if "=" in kv)
            if parts.get("kernel") == kernel and "dram_over_algorithmic" in parts:
                found.setdefault(parts.get("workload"), float(parts["dram_over_algorithmic"]))
    ratio = found.get(workload, found.get(None))
    return None if ratio is None else round(ratio * algorithmic_bytes_per_launch)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle
# ---------------------------------------------------------------------------

def oracle_sample(pr, key, target_s=12.0):
    """Time the oracle's GMRES(30)+SGS2(1,1) on a bounded sample of about
    `target_s` seconds: a 2-step probe sets how many Arnoldi steps fit; if the
    whole solve fits, it is run to convergence and timed as it is, else that
    many steps are timed and scaled to one full solve by the oracle's own
    full-solve iteration count (stored under `key`).  Returns (solves/s,
    description)."""
    import oracle
    oracle.build()

    def run(max_iters):
        t0 = time.perf_counter()
        _, info = oracle.gmres(pr.A, pr.b, restart=30, tol=1e-8, max_iters=max_iters,
                               pc_kind=oracle.PC_GS2, pc_inner=1,
                               pc_direction=oracle.SYMMETRIC)
        return time.perf_counter() - t0, info

    dt, info = run(2)
    per_iter = dt / max(info.iters, 1)
    full = stored_count(key)
    steps = max(2, int(target_s / per_iter))
    if full and steps >= full:
        dt, info = run(5000)
        return 1.0 / dt, (f"the whole GMRES(30)+SGS2(1,1) solve ({info.iters} Arnoldi steps, "
                          f"{dt:.1f} s)")
    if not full:
        return None, "full-solve count not stored"
    dt, info = run(steps)
    per_iter = dt / max(info.iters, 1)
    return 1.0 / (per_iter * full), (f"{info.iters} Arnoldi steps of the same GMRES(30)+"
                                     f"SGS2(1,1) solve ({dt:.1f} s), scaled by the oracle's "
                                     f"full-solve count {full}")


def sweep_cpu_vs_gpu(gs2, torch, pr, h, stream):
    """One SGS2(1,1) relaxation sweep from x = 0 on the benchmark matrix (the
    work of one preconditioner application): the oracle's sequential build on
    one core, the same oracle built with -fopenmp on every host core (row
    loops spread, bitwise the same result; inner products and exact-GS
    recurrences stay sequential), and the GPU (gs2_apply, CUDA events on the
    handle's stream, mean of 20 after 3 untimed).  Each CPU figure is the mean
    of the sweeps that fit in about 2 s (at least one, after one untimed)."""
    import oracle
    x0 = np.zeros(pr.n)
    res = {"sweep": "SGS2(1,1) from x = 0, FP64, gs2_apply vs the oracle's ora_gs2"}
    ref = None
    for omp in (False, True):
        key = "oracle_all_cores" if omp else "oracle_1_core"
        try:
            oracle.build(openmp=omp)
        except Exception as e:  # no OpenMP in the host compiler
            res[key] = {"unavailable": str(e).splitlines()[0][:200]}
            continue
        run = lambda: oracle.gs2(pr.A, pr.b, x0, 1, 1, 1.0, 1.0, oracle.SYMMETRIC,  # noqa: E731
                                 openmp=omp)
        ref = run()
        reps, t0 = 0, time.perf_counter()
        while reps < 1 or (time.perf_counter() - t0 < 2.0 and reps < 20):
            run()
            reps += 1
        res[key] = {"ms": round(1000 * (time.perf_counter() - t0) / reps, 2),
                    "threads": oracle.threads(openmp=omp), "sweeps_timed": reps}
    b = torch.from_numpy(pr.b).cuda()
    x = torch.zeros(pr.n, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        for _ in range(3):
            x.zero_()
            gs2.gs2_apply(h, b, x, 1, 1, 1.0, "symmetric")
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        ms = 0.0
        for _ in range(20):
            x.zero_()
            e0.record(stream)
            gs2.gs2_apply(h, b, x, 1, 1, 1.0, "symmetric")
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
    res["gpu"] = {"ms": round(ms / 20, 4)}
    if ref is not None:
        xr = torch.from_numpy(ref).cuda()
        res["gpu"]["rel_diff_vs_oracle"] = float(torch.linalg.norm(x - xr) /
                                                 torch.linalg.norm(xr))
    return res


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2104_01196_gb300 import problems as P
    pr = P.convdiff3d(args.grid)
    key = f"convdiff3d_{args.grid}_gmres30_sgs2_1_1"
    values, sample = [], ""
    for s in range(args.warmup + args.steps):
        v, sample = oracle_sample(pr, key, target_s=5.0)
        if s >= args.warmup and v is not None:
            values.append(v)
    value = float(np.mean(values)) if values else None
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 / value if value else None, "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload(args.grid, pr.n, pr.nnz), "grid": args.grid},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                         "sample": f"per step: {sample}"},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


FP64_PEAK_TFLOPS = 2 * 2 * 152 * 2.07e9 / 1e12  # 2 FMA/clk/SM x 2 flop x 152 SMs x 2.07 GHz


def kernel_flops(name, st, n, nnz=None):
    """FP64 flops of a kernel's timed launches, from its algorithmic bytes
    (the CGS2 passes read 8n bytes per basis vector)."""
    L, B = st["launches"], st["bytes"]
    if name == "cgs2_dots":        # bytes 8n(jc+1), 2 jc n flops
        return 2.0 * n * (B / (8.0 * n) - L)
    if name == "cgs2_upd_dots":    # bytes 8n(jc+2), 4 jc n flops
        return 4.0 * n * (B / (8.0 * n) - 2 * L)
    if name == "cgs2_upd_norm":    # bytes 8n(jc+2), 2 (jc+1) n flops
        return 2.0 * n * (B / (8.0 * n) - L)
    return None


def kernel_table(stats, n, hbm, nnz=None):
    out = {}
    for name, s in stats.items():
        if not s["launches"] or s["total_ms"] <= 0:
            continue
        gbs = s["bytes"] / (s["total_ms"] / 1000.0) / 1e9
        row = {"launches": s["launches"], "ms": round(s["total_ms"], 3), "share": None,
               "gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm, 3)}
        fl = kernel_flops(name, s, n, nnz)
        if fl is not None:
            tf = fl / (s["total_ms"] / 1000.0) / 1e12
            row["fp64_tflops"] = round(tf, 3)
            row["fp64_frac"] = round(tf / FP64_PEAK_TFLOPS, 3)
        out[name] = row
    tot = sum(v["ms"] for v in out.values())
    for v in out.values():
        v["share"] = round(v["ms"] / tot, 3) if tot else None
    return out


def roofline(name, s, n, hbm, peak_kind, grid, nnz=None):
    per_launch_bytes = s["bytes"] / s["launches"]
    per_launch_ms = s["total_ms"] / s["launches"]
    gbs = per_launch_bytes / (per_launch_ms / 1000.0) / 1e9
    fl = kernel_flops(name, s, n, nnz)
    traffic = stored_traffic(name, per_launch_bytes)
    tf = None if fl is None else fl / s["launches"] / (per_launch_ms / 1000.0) / 1e12
    # the bound reported is the resource the kernel uses the larger share of
    if tf is not None and tf / FP64_PEAK_TFLOPS >= gbs / hbm:
        return {"bound": "alu", "kernel": name, "achieved": round(tf, 4),
                "peak": round(FP64_PEAK_TFLOPS, 4), "unit": "TFLOP/s",
                "frac": round(tf / FP64_PEAK_TFLOPS, 3), "traffic": traffic,
                "algorithmic_flops_per_launch": fl / s["launches"],
                "algorithmic_bytes_per_launch": per_launch_bytes,
                "hbm_gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm, 3),
                "peak_source": "FP64 FMA rate: 2 FMA/clk/SM x 152 SMs x 2.07 GHz "
                               "(nominal 1.25 TFLOP/s); HBM from MEASURED_PEAKS.json "
                               f"({peak_kind})",
                "launches_timed": s["launches"]}
    return {"bound": "hbm", "kernel": name, "achieved": round(gbs, 1), "peak": hbm,
            "unit": "GB/s", "frac": round(gbs / hbm, 3), "traffic": traffic,
            "algorithmic_bytes_per_launch": per_launch_bytes,
            "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})",
            "launches_timed": s["launches"]}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def slowest_rank(dist, local_ms, device):
    """Max over ranks of a rank's timed-region length (ms)."""
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, steps, slowest_ms):
    """Solves per second of the whole job: every rank (a replica with its own
    system on its own GPU) completes `steps` solves within the slowest
    rank's time."""
    return world * steps / (slowest_ms / 1000.0)


def timed_solves(torch, stream, solve, steps):
    """Device time of `steps` back-to-back solves on `stream` (CUDA events on
    that stream around the whole run and around every solve); returns
    (total ms, per-solve ms, infos)."""
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    infos = []
    with torch.cuda.stream(stream):
        t0.record(stream)
        for k in range(steps):
            ev[k][0].record(stream)
            infos.append(solve())
            ev[k][1].record(stream)
        t1.record(stream)
    torch.cuda.synchronize()
    return t0.elapsed_time(t1), [a.elapsed_time(b) for a, b in ev], infos


def profiled(h, torch, stream, solve, steps, hbm, n, nnz, peak_kind="measured"):
    """The kernel table of one solve (an event pair around every launch),
    then a second pass of `steps` identical solves with only the dominant
    kernel bracketed: its roofline.  Kept out of the timed region."""
    with torch.cuda.stream(stream):
        h.profile_filter(None)
        h.profile(True)
        h.profile_reset()
        solve()
    stream.synchronize()
    table = kernel_table(h.profile_read(), n, hbm, nnz)
    h.profile(False)
    top = max(table, key=lambda k: table[k]["ms"]) if table else None
    roof = None
    if top:
        h.profile_filter(top)
        h.profile(True)
        with torch.cuda.stream(stream):
            solve()  # captures the Arnoldi-step graph with the event nodes
        stream.synchronize()
        h.profile_reset()
        with torch.cuda.stream(stream):
            for _ in range(steps):
                solve()
        stream.synchronize()
        st = h.profile_read()
        h.profile(False)
        h.profile_filter(None)
        if top in st and st[top]["launches"]:
            roof = roofline(top, st[top], n, hbm, peak_kind, None, nnz)
    return table, roof


def run_ours(args):
    import torch

    import paper_2104_01196_gb300 as gs2
    from paper_2104_01196_gb300 import build as B
    from paper_2104_01196_gb300 import problems as P

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0 or not os.path.exists(B.LIB):
        B.build()
    if dist:
        dist.barrier()
    gs2.load()

    pr = P.convdiff3d(args.grid)
    n, nnz = pr.n, pr.nnz
    stream = torch.cuda.Stream()
    h = gs2.gs2_setup(pr.A, precisions=("fp32", "fp16", "fp32_sweep", "fp16_sweep"),
                      stream=stream.cuda_stream)
    if not args.no_autotune:
        h.autotune()  # tile shapes of A and the triangles (setup time, untimed)
    pc = gs2.params("gs2", 1, 1, direction="symmetric")
    if not args.no_autotune:
        h.autotune_gmres(30, pc)  # solve structure: separate launches or cycle graphs
    shapes = {k: v for k, v in h.stats().items()
              if k.startswith(("tpr", "rpt", "sell", "offset", "solve_mode"))}
    with torch.cuda.stream(stream):
        b = torch.from_numpy(pr.b).cuda()
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
    stream.synchronize()

    def solver(prm):
        def solve():
            x.zero_()
            return gs2.gmres_solve(h, b, x, 30, 1e-8, 5000, prm)
        return solve
    solve = solver(pc)

    # warm-up (graph capture, workspaces); no profiling anywhere before or in
    # the timed region
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            info = solve()
    stream.synchronize()
    if info.status != 0:
        raise RuntimeError(f"warm-up solve failed: {info}")
    hbm, peak_kind = peaks()

    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    launches0 = gs2.launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    total_ms, step_ms, infos = timed_solves(torch, stream, solve, args.steps)
    if dist:
        dist.barrier()
    launches = gs2.launch_count() - launches0
    clocks = sampler.stop() if sampler else None
    for inf in infos:
        if inf.status != 0:
            raise RuntimeError(f"timed solve failed: {inf}")
    if dist:
        total_ms = slowest_rank(dist, total_ms, "cuda")
    ms_per_step = total_ms / args.steps
    value = whole_job_rate(world, args.steps, total_ms)
    iters = [inf.iters for inf in infos]
    xt = torch.from_numpy(pr.x_true).cuda()
    err = float(torch.linalg.norm(x - xt) / torch.linalg.norm(xt))
    x64 = x.clone()

    out = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload(args.grid, n, nnz), "grid": args.grid, "n": n,
                   "nnz": nnz, "restart": 30, "tol": 1e-8, "precond": "SGS2(1,1) FP64",
                   "tile_shapes": shapes,
                   "parallelism": f"replicas x{world}",
                   "l2": l2_note(n, nnz)},
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                       "p99": float(np.percentile(step_ms, 99)),
                       "per_step": [round(t, 3) for t in step_ms]},
        "iters": iters,
        "oracle_iters": stored_count(f"convdiff3d_{args.grid}_gmres30_sgs2_1_1"),
        "rel_err_vs_x_true": err,
        "true_relres": infos[-1].true_relres,
        "gpu_launches": int(launches),
        "clocks": clocks,
    }

    # ---- e2e: the public C-ABI call with host (pinned) buffers ------------
    # the library copies b and x0 to the device, solves and copies x back
    # inside every timed call; all `steps` solves are timed
    out["e2e"] = None
    if not args.no_e2e:
        bh = torch.from_numpy(pr.b.copy()).pin_memory().numpy()
        xh = torch.zeros(n, dtype=torch.float64).pin_memory().numpy()
        gs2.gmres_solve(h, bh, xh, 30, 1e-8, 5000, pc)
        e2e_t = []
        for _ in range(args.steps):
            xh[:] = 0.0
            t0 = time.perf_counter()
            inf = gs2.gmres_solve(h, bh, xh, 30, 1e-8, 5000, pc)
            e2e_t.append(time.perf_counter() - t0)
            assert inf.status == 0
        tot = float(np.sum(e2e_t))
        if dist:
            tot = slowest_rank(dist, tot, "cuda")
        out["e2e"] = {"value": world * args.steps / tot, "unit": "solves/s",
                      "h2d_bytes_per_step": 16 * n, "d2h_bytes_per_step": 8 * n,
                      "steps": args.steps,
                      "note": "gmres_solve with pinned host b and x: H2D of b and x0, "
                              "solve, D2H of x inside each timed call (wall clock)"}

    # ---- roofline: a second, identical pass with the dominant kernel ------
    # bracketed by events (and the per-kernel table of one solve before it)
    if not args.no_profile:
        kernels, roof = profiled(h, torch, stream, solve, args.steps, hbm, n, nnz, peak_kind)
        out["roofline"] = roof
        out["kernels"] = kernels
        out["sweep_kernels"] = {k: kernels[k] for k in ("resid", "inner64", "spmv")
                                if k in kernels}

    only = set(filter(None, args.only_extras.split(",")))

    def want(name, off=False):
        return rank == 0 and world == 1 and not off and (name in only if only else True)

    # ---- the same workload with lower-precision inner sweeps --------------
    if want("precision", args.no_extras):
        res = {}
        for prec in ("fp32", "fp16", "fp32_sweep", "fp16_sweep"):
            pp = gs2.params("gs2", 1, 1, direction="symmetric", precision=prec)
            sp = solver(pp)
            with torch.cuda.stream(stream):
                sp()
            stream.synchronize()
            tot, per, inf = timed_solves(torch, stream, sp, args.steps)
            row = {"solves_per_s": args.steps / (tot / 1000.0), "ms_per_solve": tot / args.steps,
                   "iters": inf[-1].iters, "status": inf[-1].status,
                   "oracle_iters": stored_count(
                       f"convdiff3d_{args.grid}_gmres30_sgs2_1_1_{prec}"),
                   "true_relres": inf[-1].true_relres,
                   "rel_err_vs_x_true": float(torch.linalg.norm(x - xt) / torch.linalg.norm(xt)),
                   "rel_err_vs_fp64_solution": float(torch.linalg.norm(x - x64) /
                                                     torch.linalg.norm(x64)),
                   "speedup_vs_fp64": (args.steps / (tot / 1000.0)) / value}
            if not args.no_profile:
                tab, _ = profiled(h, torch, stream, sp, 0, hbm, n, nnz)
                row["kernels"] = {k: v for k, v in tab.items()
                                  if k.startswith(("inner", "resid", "spmv", "rhat", "to32"))}
            res[prec] = row
        out["precision"] = res
    h.close()

    if want("laplacian128", args.no_extras):
        out["laplacian128"] = laplacian_line(gs2, torch, P, args, hbm)
    if want("comparisons", args.no_extras):
        lap = P.poisson3d(128)
        out["comparisons"] = comparisons(gs2, torch, lap, stream,
                                         torch.from_numpy(lap.b).cuda())
        if want("hybrid", args.no_extras):
            out["hybrid"] = hybrid(gs2, torch, lap, stream, torch.from_numpy(lap.b).cuda())
        del lap
    if want("serving", args.no_serve):
        out["serving"] = serving(gs2, torch, args.serve_requests,
                                 [float(r) for r in args.serve_rates.split(",") if r],
                                 [f for f in args.serve_forms.split(",") if f],
                                 [f for f in args.serve_sweep_forms.split(",") if f])
    if want("small_system", args.no_extras):
        out["small_system"] = small_system(gs2, torch)
    if want("packs", args.no_extras):
        out["packs"] = packs(gs2, torch)
    if want("workloads", args.no_extras or args.no_workloads):
        out["workloads"] = full_workloads(gs2, torch)
    if rank == 0 and world == 1 and not args.no_cpu:
        v, sample = oracle_sample(pr, f"convdiff3d_{args.grid}_gmres30_sgs2_1_1")
        hh = gs2.gs2_setup(pr.A, stream=stream.cuda_stream)
        out["cpu_baseline"] = {"value": v, "unit": "solves/s", "cores": 1, "kind": "oracle",
                               "sample": sample,
                               "sweep_1_vs_all_cores": sweep_cpu_vs_gpu(gs2, torch, pr, hh,
                                                                        stream)}
        hh.close()
        if not args.no_cpu_table:
            out["cpu_baseline"]["table"] = cpu_table(gs2, torch, P)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def laplacian_line(gs2, torch, P, args, hbm):
    """The 3D 7-point Laplacian 128^3 with GMRES(30) + SGS2(1,1) FP64, the
    same measurement as the headline: device-timed solves with profiling
    off, then the kernel table and the dominant kernel's roofline from a
    second pass."""
    pr = P.poisson3d(128)
    stream = torch.cuda.Stream()
    h = gs2.gs2_setup(pr.A, stream=stream.cuda_stream)
    if not args.no_autotune:
        h.autotune()
    pc = gs2.params("gs2", 1, 1, direction="symmetric")
    with torch.cuda.stream(stream):
        b = torch.from_numpy(pr.b).cuda()
        x = torch.zeros(pr.n, dtype=torch.float64, device="cuda")

    def solve():
        x.zero_()
        return gs2.gmres_solve(h, b, x, 30, 1e-8, 5000, pc)
    with torch.cuda.stream(stream):
        for _ in range(3):
            solve()
    stream.synchronize()
    tot, per, infos = timed_solves(torch, stream, solve, args.steps)
    res = {"workload": "3D 7-point Laplacian 128^3 (n=2,097,152, nnz=14,581,760), "
                       "GMRES(30) + SGS2(1,1) FP64, 1e-8",
           "solves_per_s": args.steps / (tot / 1000.0), "ms_per_solve": tot / args.steps,
           "iters": infos[-1].iters,
           "oracle_iters": stored_count("poisson3d_128_gmres30_sgs2_1_1"),
           "true_relres": infos[-1].true_relres}
    if not args.no_profile:
        tab, roof = profiled(h, torch, stream, solve, args.steps, hbm, pr.n, pr.nnz,
                             peaks()[1])
        res["kernels"] = tab
        res["roofline"] = roof
    h.close()
    return res


def small_system(gs2, torch, reps=20):
    """2D 5-point Poisson 64x64 (n = 4096), GMRES(30) + forward GS2(1,1) to
    1e-8: latency-bound, so timed with the whole solve inside one
    thread-block cluster (the default at this size: the system in the
    cluster's shared memory), as one cooperative launch, with the Arnoldi
    steps of each cycle replayed as a CUDA graph, as separate launches, and
    as the autotuner's choice (device-timed solves per second)."""
    from paper_2104_01196_gb300 import problems as P
    pr = P.poisson2d(64)
    pc = gs2.params("gs2", 1, 1)
    b = torch.from_numpy(pr.b).cuda()
    x = torch.zeros(pr.n, dtype=torch.float64, device="cuda")
    res = {"workload": "2D 5-point Poisson 64x64, GMRES(30) + GS2(1,1) forward, 1e-8"}
    for name, mode in (("one_cluster", 4), ("one_launch", 3), ("graph", 1), ("launches", 2),
                       ("autotuned", 0)):
        h = gs2.gs2_setup(pr.A)
        h.set_graph_mode(mode)
        if mode == 0:
            res["autotuned_mode"] = h.autotune_gmres(30, pc)
        for _ in range(3):
            x.zero_()
            info = gs2.gmres_solve(h, b, x, 30, 1e-8, 4000, pc)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            x.zero_()
            info = gs2.gmres_solve(h, b, x, 30, 1e-8, 4000, pc)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / reps
        res[name] = {"ms_per_solve": round(ms, 3), "solves_per_s": round(1000.0 / ms, 1),
                     "iters": info.iters, "oracle_iters": stored_count("poisson2d_64_gmres30_gs2_1_1"),
                     "true_relres": info.true_relres}
        h.close()
    # CG with SGS2(1,1) on the same SPD system: one cluster, one launch, graphs of 16
    # iterations
    pcs = gs2.params("gs2", 1, 1, direction="symmetric")
    for name, mode in (("cg_one_cluster", 4), ("cg_one_launch", 3), ("cg_graph", 1)):
        h = gs2.gs2_setup(pr.A)
        h.set_graph_mode(mode)
        for _ in range(3):
            x.zero_()
            info = gs2.cg_solve(h, b, x, 1e-8, 4000, pcs)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            x.zero_()
            info = gs2.cg_solve(h, b, x, 1e-8, 4000, pcs)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / reps
        res[name] = {"ms_per_solve": round(ms, 3), "solves_per_s": round(1000.0 / ms, 1),
                     "iters": info.iters, "oracle_iters": stored_count("poisson2d_64_cg_sgs2_1_1"),
                     "true_relres": info.true_relres}
        h.close()
    return res


def packs(gs2, torch, count=128):
    """Many small systems of the request stream's kinds (2D/3D Poisson and 3D
    convection-diffusion, lognormal coefficients), n log-uniform in
    [1e3, 3.2e4], GMRES(30) + SGS2(1,1) to 1e-8, several ways: one
    gmres_solve after another, gs2_batch_solve (one stream per system), one
    pack (gs2_pack_gmres: every row kernel covers all systems, per-system
    Krylov state; each restart cycle one graph replay) with FP64, FP32 and
    whole-sweep FP32 preconditioning, and the pack as one cooperative launch
    (every system's blocks run its whole solve).  Matrices are set up before the clock starts; each way is timed
    once after an untimed run, wall clock around the call(s) with device
    vectors.  The pack's per-system iteration counts are compared with the
    separate solves'."""
    from paper_2104_01196_gb300 import problems as P
    recipe = P.request_stream(count, rate_hz=1.0, n_lo=1e3, n_hi=3.2e4, build=False)
    probs = [P.variable_coefficient_problem(kind, N, seed) for _, kind, N, seed in recipe]
    res = {"systems": count, "n_total": int(sum(p.n for p in probs)),
           "n_range": [int(min(p.n for p in probs)), int(max(p.n for p in probs))]}
    pc = gs2.params("gs2", 1, 1, direction="symmetric")
    streams = [torch.cuda.Stream() for _ in probs]
    hs = [gs2.gs2_setup(p.A, stream=s.cuda_stream) for p, s in zip(probs, streams)]
    bs = [torch.from_numpy(p.b).cuda() for p in probs]
    xs = [torch.zeros(p.n, dtype=torch.float64, device="cuda") for p in probs]
    torch.cuda.synchronize()

    def clock(fn):
        fn()  # untimed: graphs, workspaces
        for x in xs:
            x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return out, time.perf_counter() - t0

    seq, dt = clock(lambda: [gs2.gmres_solve(h, b, x, 30, 1e-8, 4000, pc)
                             for h, b, x in zip(hs, bs, xs)])
    res["sequential"] = {"solves_per_s": round(count / dt, 1), "s": round(dt, 4),
                         "failed": sum(i.status != 0 for i in seq)}
    bat, dt = clock(lambda: gs2.gs2_batch_solve(hs, bs, xs, 30, 1e-8, 4000, pc))
    res["batch_streams"] = {"solves_per_s": round(count / dt, 1), "s": round(dt, 4),
                            "failed": sum(i.status != 0 for i in bat)}
    for h in hs:
        h.close()
    pack = gs2.pack_setup([p.A for p in probs], precisions=("fp32", "fp32_sweep"))
    b = torch.cat(bs)
    x = torch.zeros(pack.n, dtype=torch.float64, device="cuda")
    for prec in ("fp64", "fp32", "fp32_sweep", "one_launch_fp64"):
        pack.set_graph_mode(3 if prec.startswith("one_launch") else 0)
        pcp = gs2.params("gs2", 1, 1, direction="symmetric",
                         precision=prec.replace("one_launch_", ""))

        def run():
            x.zero_()
            return gs2.pack_gmres(pack, b, x, 30, 1e-8, 4000, pcp)
        infos, dt = clock(run)
        worst = max(i.true_relres for i in infos)
        res[f"pack_{prec}"] = {
            "solves_per_s": round(count / dt, 1), "s": round(dt, 4),
            "failed": sum(i.status != 0 for i in infos), "worst_true_relres": worst,
            "iters_max_abs_diff_vs_sequential": int(max(abs(a.iters - q.iters)
                                                        for a, q in zip(infos, seq)))}
    pack.close()
    # a pack of 32 tiny systems (n in [500, 2000]; ~35K rows in all, about
    # one row per thread of the co-resident blocks): replayed cycle graphs,
    # the whole pack in one cooperative launch, and one thread-block cluster
    # per system
    recipe = P.request_stream(32, rate_hz=1.0, n_lo=5e2, n_hi=2e3, seed=P.SEED_BASE + 500,
                              build=False)
    tiny = [P.variable_coefficient_problem(kind, N, seed) for _, kind, N, seed in recipe]
    tp = gs2.pack_setup([q.A for q in tiny])
    tb = torch.cat([torch.from_numpy(q.b).cuda() for q in tiny])
    tx = torch.zeros(tp.n, dtype=torch.float64, device="cuda")
    pc1 = gs2.params("gs2", 1, 1, direction="symmetric")
    row = {"systems": len(tiny), "n_total": int(tp.n)}
    for name, mode in (("graphs", 1), ("one_launch", 3), ("one_cluster", 4)):
        tp.set_graph_mode(mode)

        def run():
            tx.zero_()
            return gs2.pack_gmres(tp, tb, tx, 30, 1e-8, 4000, pc1)
        infos, dt = clock(run)
        row[name] = {"solves_per_s": round(len(tiny) / dt, 1), "ms": round(1000 * dt, 3),
                     "failed": sum(i.status != 0 for i in infos),
                     "iters_max": int(max(i.iters for i in infos))}
    tp.close()
    res["tiny_pack"] = row
    return res


def full_workloads(gs2, torch):
    """The Q1 elasticity configuration at full size (64^3 nodes), device-timed
    once per setting (after an untimed restart cycle): SGS2(1, n_j) at the
    omega its few inner sweeps need (n_j = 2: 0.8, n_j = 3: 0.9; with
    omega = 1 it stagnates, as the paper's elasticity tables show), FP64 and
    FP32 triangle values (GMRES FP64), each beside the oracle's count for the
    same setting and precision; and stationary JR at omega = 1, which
    diverges on it.  (The 192^3 convection-diffusion configuration is the
    headline, with its precision variants.)"""
    from paper_2104_01196_gb300 import problems as P
    out = {}

    def timed(h, b, x, pc, max_iters):
        x.zero_()
        gs2.gmres_solve(h, b, x, 30, 1e-8, 30, pc)  # warm: one restart cycle
        x.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        info = gs2.gmres_solve(h, b, x, 30, 1e-8, max_iters, pc)
        e1.record()
        e1.synchronize()
        return info, e0.elapsed_time(e1)

    pr = P.elasticity3d(64)
    h = gs2.gs2_setup(pr.A, precisions=("fp32",))
    b = torch.from_numpy(pr.b).cuda()
    x = torch.zeros(pr.n, dtype=torch.float64, device="cuda")
    res = {"n": pr.n, "nnz": int(len(pr.A[1]))}
    x64 = {}
    for nj, om in ((2, 0.8), (3, 0.9)):
        for prec in ("fp64", "fp32"):
            stem = f"sgs2_1_{nj}_w{om}"
            vname = f"{stem}_{prec}"
            pc = gs2.params("gs2", 1, nj, omega=om, direction="symmetric", precision=prec)
            info, ms = timed(h, b, x, pc, 5000)
            key = f"elasticity3d_64_gmres30_{stem}" + ("" if prec == "fp64" else f"_{prec}")
            res[vname] = {"status": info.status, "iters": info.iters,
                          "oracle_iters": stored_count(key), "ms": round(ms, 2),
                          "true_relres": info.true_relres}
            # FP32 values: error against the FP64-value solution of the same
            # system (itself within the parity bound of the oracle)
            if prec == "fp64":
                x64[stem] = x.clone()
            else:
                res[vname]["rel_err_vs_fp64_solution"] = float(
                    torch.linalg.norm(x - x64[stem]) / torch.linalg.norm(x64[stem]))
    # stationary JR, omega = 1 (the paper's elasticity tables): the residual grows
    x.zero_()
    r0 = float(torch.linalg.norm(b))
    gs2.jr_apply(h, b, x, 50, 1.0)
    y = torch.zeros_like(x)
    gs2.gs2_spmv(h, x, y)
    growth = float(torch.linalg.norm(b - y)) / r0
    res["jr_stationary_w1.0_50_sweeps_residual_growth"] = \
        growth if math.isfinite(growth) else None
    h.close()
    out["elasticity3d_64"] = res
    return out


def cpu_table(gs2, torch, P, reps=10, solve_budget_s=30.0):
    """The oracle on the host cores for every single-GPU configuration (2D
    Poisson 64^2, 3D Laplacian 128^3, Q1 elasticity 64^3, convection-diffusion
    192^3): each sweep type as the median of `reps` runs on one core and,
    where its loop is row-parallel, on every core (the -fopenmp build of the
    same source, bitwise the same result), with the GPU's mean over `reps`
    beside it; and one full GMRES(30) solve on one core with the
    configuration's preconditioner -- run to convergence when it fits in
    `solve_budget_s`, else that many Arnoldi steps timed and scaled by the
    oracle's stored full-solve count (labelled "extrapolated")."""
    import platform

    import oracle
    oracle.build()
    oracle.build(openmp=True)
    model = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    res = {"nproc": os.cpu_count(), "cpu": model, "threads_all_cores": oracle.threads(True),
           "configs": {}}
    confs = [
        ("poisson2d_64", lambda: P.poisson2d(64), 1, 1.0, oracle.FORWARD,
         "poisson2d_64_gmres30_gs2_1_1"),
        ("poisson3d_128", lambda: P.poisson3d(128), 1, 1.0, oracle.SYMMETRIC,
         "poisson3d_128_gmres30_sgs2_1_1"),
        ("elasticity3d_64", lambda: P.elasticity3d(64), 2, 0.8, oracle.SYMMETRIC,
         "elasticity3d_64_gmres30_sgs2_1_2_w0.8"),
        ("convdiff3d_192", lambda: P.convdiff3d(192), 1, 1.0, oracle.SYMMETRIC,
         "convdiff3d_192_gmres30_sgs2_1_1"),
    ]

    def med(fn):
        fn()
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            fn()
            ts.append(time.perf_counter() - t0)
        return round(1000 * float(np.median(ts)), 3)

    for name, mk, nj, om, dirn, key in confs:
        pr = mk()
        A, bb = pr.A, pr.b
        x0 = P.uniform_pm1(99, pr.n)
        row = {"n": pr.n, "nnz": int(len(A[1])), "sweeps_ms": {}}
        sweeps = {
            "spmv": (lambda o: oracle.spmv(A, x0, openmp=o), True),
            "jr_1": (lambda o: oracle.jr(A, bb, x0, 1, 1.0, openmp=o), True),
            "resid_scale_update_gs2_fwd_1_0": (
                lambda o: oracle.gs2(A, bb, x0, 1, 0, 1.0, 1.0, oracle.FORWARD, openmp=o), True),
            "gs2_fwd_1_1": (
                lambda o: oracle.gs2(A, bb, x0, 1, 1, 1.0, 1.0, oracle.FORWARD, openmp=o), True),
            "sgs2_1_1": (
                lambda o: oracle.gs2(A, bb, x0, 1, 1, 1.0, 1.0, oracle.SYMMETRIC, openmp=o), True),
            "sgs_exact": (lambda o: oracle.gs(A, bb, x0, 1, 1.0, oracle.SYMMETRIC), False),
        }
        h = gs2.gs2_setup(A)
        bd = torch.from_numpy(bb).cuda()
        x0d = torch.from_numpy(x0).cuda()
        xd = torch.zeros_like(x0d)
        gpu = {
            "spmv": lambda: gs2.gs2_spmv(h, x0d, xd),
            "jr_1": lambda: (xd.copy_(x0d), gs2.jr_apply(h, bd, xd, 1, 1.0)),
            "resid_scale_update_gs2_fwd_1_0": lambda: (xd.copy_(x0d),
                                                       gs2.gs2_apply(h, bd, xd, 1, 0, 1.0, 0)),
            "gs2_fwd_1_1": lambda: (xd.copy_(x0d), gs2.gs2_apply(h, bd, xd, 1, 1, 1.0, 0)),
            "sgs2_1_1": lambda: (xd.copy_(x0d), gs2.gs2_apply(h, bd, xd, 1, 1, 1.0, 2)),
            "sgs_exact": lambda: (xd.copy_(x0d), gs2.gs_apply(h, bd, xd, 1, 1.0, 2)),
        }
        for sname, (fn, par) in sweeps.items():
            r = {"oracle_1_core_ms": med(lambda: fn(False))}
            if par:
                r["oracle_all_cores_ms"] = med(lambda: fn(True))
            g = gpu[sname]
            g()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                g()
            e1.record()
            e1.synchronize()
            r["gpu_ms"] = round(e0.elapsed_time(e1) / reps, 4)
            row["sweeps_ms"][sname] = r
        h.close()
        # one full GMRES solve on one core (or a scaled sample of it)
        kw = dict(pc_kind=oracle.PC_GS2, pc_inner=nj, pc_omega=om, pc_direction=dirn)
        t0 = time.perf_counter()
        _, info = oracle.gmres(A, bb, restart=30, tol=1e-8, max_iters=2, **kw)
        per = (time.perf_counter() - t0) / max(info.iters, 1)
        full = stored_count(key)
        if full and per * full <= solve_budget_s:
            t0 = time.perf_counter()
            _, info = oracle.gmres(A, bb, restart=30, tol=1e-8, max_iters=5000, **kw)
            dt = time.perf_counter() - t0
            row["gmres_1_core"] = {"s": round(dt, 2), "iters": info.iters, "extrapolated": False}
        elif full:
            steps = max(2, int(solve_budget_s / per))
            t0 = time.perf_counter()
            _, info = oracle.gmres(A, bb, restart=30, tol=1e-8, max_iters=steps, **kw)
            dt = time.perf_counter() - t0
            row["gmres_1_core"] = {"s": round(dt / info.iters * full, 2), "iters": full,
                                   "extrapolated": True,
                                   "sample": f"{info.iters} Arnoldi steps in {dt:.1f} s"}
        res["configs"][name] = row
        del pr, A, bb
    return res


def _make_request(rec):
    """One request of the stream (spawned worker): its CSR and right-hand side."""
    from paper_2104_01196_gb300 import problems as P
    _, kind, N, seed = rec
    pr = P.variable_coefficient_problem(kind, N, seed)
    return pr.A, pr.b


SERVE_FORMS = {
    # name: (sweep precision, rows up to which requests are packed, slots
    # kept for requests of at most 65,536 rows)
    "fp64": ("fp64", 0, 0),
    "fp32": ("fp32", 0, 0),
    "fp16": ("fp16", 0, 0),
    "fp32_packed": ("fp32", 1 << 16, 0),
    "fp32_sweep": ("fp32_sweep", 0, 0),
    "fp16_sweep": ("fp16_sweep", 0, 0),
    "fp32_sweep_packed": ("fp32_sweep", 1 << 16, 0),
    "fp32_sweep_packed_lanes": ("fp32_sweep", 1 << 16, 2),
}


def serving(gs2, torch, count, rates, forms, sweep_forms, workers=0):
    """The request stream of the serving configuration: `count` requests,
    each a 2D/3D Poisson or 3D convection-diffusion system (type uniform),
    n log-uniform in [1e3, 2e6], lognormal(0,1) coefficients, GMRES(30) +
    SGS2(1,1) to 1e-8, served by the continuous-batching server (8 slots,
    admission by device memory).  Per form (inner sweeps FP64, FP32, FP16, or
    FP32 with requests of at most 65,536 rows admitted together as packs,
    optionally with two of the slots kept for those requests):
    the server saturated (every request submitted at once: solves/s and
    submit-to-done latency); for the forms in `sweep_forms` also open-loop
    Poisson arrivals at each rate in `rates` (the stream's seeded
    inter-arrival gaps rescaled; p50/p99 latency over all requests and per
    size tercile, throughput achieved).
    The requests are generated once, before any clock starts, by spawned
    worker processes; the server copies each request's inputs at submit."""
    import multiprocessing as mp

    from paper_2104_01196_gb300 import problems as P
    recipe = P.request_stream(count, rate_hz=1.0, build=False)
    t0 = time.perf_counter()
    nw = workers or max(1, min(16, (os.cpu_count() or 2) - 1))
    with mp.get_context("spawn").Pool(nw) as pool:
        reqs = pool.map(_make_request, recipe, chunksize=4)
    gen_s = time.perf_counter() - t0
    ns = np.array([len(A[0]) - 1 for A, _ in reqs])
    gaps = np.diff(np.concatenate([[0.0], [r[0] for r in recipe]]))  # rate 1/s
    terc = np.quantile(ns, [1 / 3, 2 / 3])
    tercile = np.digitize(ns, terc)  # 0, 1, 2
    res = {"requests": count, "n_total": int(ns.sum()), "n_range": [int(ns.min()), int(ns.max())],
           "size_terciles_rows": [[int(ns.min()), int(terc[0])], [int(terc[0]), int(terc[1])],
                                  [int(terc[1]), int(ns.max())]],
           "generate_s": round(gen_s, 1), "workers": nw}

    def pct(v):
        return {"p50": round(float(np.percentile(v, 50)), 2),
                "p99": round(float(np.percentile(v, 99)), 2)} if len(v) else None

    for name in forms:
        prec, pack_rows, small_slots = SERVE_FORMS[name]
        pc = gs2.params("gs2", 1, 1, direction="symmetric", precision=prec)
        srv = gs2.Server(restart=30, tol=1e-8, max_iters=10000, precond=pc, max_slots=8,
                         prep_threads=4, pack_rows=pack_rows, pack_max=32,
                         small_rows=1 << 16, small_slots=small_slots)
        row = {}
        # saturated: everything queued at once
        t0 = time.perf_counter()
        tickets = [srv.submit(A, b) for A, b in reqs]
        lat, iters, bad, worst = [], [], 0, 0.0
        for t in tickets:
            info, _, ms = srv.wait(t, 0, timeout=3600.0)
            lat.append(ms)
            iters.append(info.iters)
            if info.status != 0:
                bad += 1
            else:
                worst = max(worst, info.true_relres)
        dt = time.perf_counter() - t0
        sat = count / dt
        st = srv.stats()
        row["saturated"] = {"solves_per_s": round(sat, 2), "s": round(dt, 2),
                            "latency_ms": pct(lat), "failed": bad,
                            "worst_true_relres": worst, "max_active": st["max_active"],
                            "iters_total": int(np.sum(iters)),
                            "iters_median": int(np.median(iters)),
                            "iters_max": int(np.max(iters))}
        for rate in (rates if name in sweep_forms else []):
            arrivals = np.cumsum(gaps / rate)
            t0 = time.perf_counter()
            tickets = []
            for a, (A, b) in zip(arrivals, reqs):
                delay = a - (time.perf_counter() - t0)
                if delay > 0:
                    time.sleep(delay)
                tickets.append(srv.submit(A, b))
            lat = np.array([srv.wait(t, 0, timeout=3600.0)[2] for t in tickets])
            dt = time.perf_counter() - t0
            row[f"open_loop_{rate:g}_per_s"] = {
                "offered_per_s": rate, "achieved_per_s": round(count / dt, 2),
                "s": round(dt, 2), "latency_ms": pct(lat),
                "latency_ms_by_size_tercile": [pct(lat[tercile == k]) for k in range(3)]}
        srv.close()
        res[name] = row
    base = res.get("fp64", {}).get("saturated", {}).get("solves_per_s")
    if base:
        res["saturated_speedup_vs_fp64"] = {
            k: round(res[k]["saturated"]["solves_per_s"] / base, 3)
            for k in forms if k != "fp64"}
    return res


def hybrid(gs2, torch, pr, stream, b):
    """The hybrid (block-Jacobi) preconditioners of the paper's distributed
    runs on the same workload, P row blocks standing in for P processes:
    the global JR(4,1), the local JR(1,4), hybrid SGS2(1,1) and hybrid exact
    SGS (local triangular solves by level sets); GMRES(30)
    iterations and device time per solve for each P (one untimed solve
    first, which also builds the blocks' matrices)."""
    res = {"workload": "GMRES(30) to 1e-8 on the 128^3 Laplacian, P contiguous row blocks"}
    h = gs2.gs2_setup(pr.A, stream=stream.cuda_stream)
    with torch.cuda.stream(stream):
        x = torch.zeros(pr.n, dtype=torch.float64, device="cuda")
        for parts in (1, 8, 64, 512):
            row = {}
            for name, p in (("jr_4_1_global", gs2.params("jr", 4, parts=parts)),
                            ("jr_1_4_local", gs2.params("jr", 1, parts=parts, local=4)),
                            ("sgs2_1_1", gs2.params("gs2", 1, 1, direction="symmetric",
                                                    parts=parts)),
                            ("sgs_levels", gs2.params("gs", 1, direction="symmetric",
                                                      parts=parts))):
                x.zero_()
                gs2.gmres_solve(h, b, x, 30, 1e-8, 5000, p)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                x.zero_()
                e0.record(stream)
                info = gs2.gmres_solve(h, b, x, 30, 1e-8, 5000, p)
                e1.record(stream)
                e1.synchronize()
                okey = {"jr_4_1_global": "jr_4_1", "jr_1_4_local": "jr_1_4",
                        "sgs2_1_1": "sgs2_1_1", "sgs_levels": "sgs"}[name]
                row[name] = {"status": info.status, "iters": info.iters,
                             "oracle_iters": stored_count(
                                 f"poisson3d_128_gmres30_hybrid_{okey}_P{parts}"),
                             "ms": round(e0.elapsed_time(e1), 2)}
            res[f"P={parts}"] = row
    h.close()
    return res


# the oracle's stored full-solve counts of the comparison solves
ORACLE_KEYS = {
    "sgs2_1_2": "poisson3d_128_gmres30_sgs2_1_2",
    "sgs2_1_3": "poisson3d_128_gmres30_sgs2_1_3",
    "compact_sgs2_1_2": "poisson3d_128_gmres30_compact_sgs2_1_2",
    "sgs2_1_1_fp32": "poisson3d_128_gmres30_sgs2_1_1_fp32",
    "sgs2_1_1_fp16": "poisson3d_128_gmres30_sgs2_1_1_fp16",
    "gs_levels_sym": "poisson3d_128_gmres30_sgs_exact",
    "mtsgs": "poisson3d_128_gmres30_mtsgs",
    "amg_sgs2_1_1": "poisson3d_128_gmres30_amg_sgs2_1_1",
    "jr3_w1.0": "poisson3d_128_gmres30_jr3_w1.0",
    "jr3_w0.8": "poisson3d_128_gmres30_jr3_w0.8",
    "cg_sgs2_1_1": "poisson3d_128_cg_sgs2_1_1",
    "cg_amg_sgs2_1_1": "poisson3d_128_cg_amg_sgs2_1_1",
}


def comparisons(gs2, torch, pr, stream, b):
    """One solve each of the paper's baselines and the precision variants on
    the same workload (untimed by the headline; device-timed here), and CG
    with SGS2 and with the AMG cycle (the Laplacian is SPD; Sec. 9 runs CG
    with SGS2)."""
    res = {}
    variants = {
        "sgs2_1_2": gs2.params("gs2", 1, 2, direction="symmetric"),
        "sgs2_1_3": gs2.params("gs2", 1, 3, direction="symmetric"),
        "compact_sgs2_1_2": gs2.params("gs2", 1, 2, direction="symmetric", form="compact"),
        "sgs2_1_1_fp32": gs2.params("gs2", 1, 1, direction="symmetric", precision="fp32"),
        "sgs2_1_1_fp16": gs2.params("gs2", 1, 1, direction="symmetric", precision="fp16"),
        "gs_levels_sym": gs2.params("gs", 1, direction="symmetric"),
        "mtsgs": gs2.params("mtgs", 1, direction="symmetric"),
        "amg_sgs2_1_1": gs2.params("amg", 1, 1, direction="symmetric"),
        "jr3_w1.0": gs2.params("jr", 3, omega=1.0),
        "jr3_w0.8": gs2.params("jr", 3, omega=0.8),
        "cg_sgs2_1_1": gs2.params("gs2", 1, 1, direction="symmetric"),
        "cg_amg_sgs2_1_1": gs2.params("amg", 1, 1, direction="symmetric"),
    }
    h = gs2.gs2_setup(pr.A, precisions=("fp32", "fp16", "fp32_sweep", "fp16_sweep"),
                      stream=stream.cuda_stream)
    t0 = time.perf_counter()
    h.amg_setup()  # smoothed-aggregation hierarchy (host setup, once per matrix)
    res["amg_setup_s"] = round(time.perf_counter() - t0, 3)
    res["amg_levels"] = [list(lv) for lv in h.amg_info()]
    with torch.cuda.stream(stream):
        x = torch.zeros(pr.n, dtype=torch.float64, device="cuda")
        # the FP64 SGS2(1,1) solution, the reference of the precision variants
        x_ref = torch.zeros_like(x)
        gs2.gmres_solve(h, b, x_ref, 30, 1e-8, 3000,
                        gs2.params("gs2", 1, 1, direction="symmetric"))
        for name, p in variants.items():
            # (the Laplacian is SPD: the cg_ variants run CG with the
            # symmetric preconditioner instead of GMRES)
            def solve():
                if name.startswith("cg_"):
                    return gs2.cg_solve(h, b, x, 1e-8, 3000, p)
                return gs2.gmres_solve(h, b, x, 30, 1e-8, 3000, p)
            x.zero_()
            solve()  # warm (levels, workspace)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            x.zero_()
            e0.record(stream)
            info = solve()
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            err = float(torch.linalg.norm(x - torch.from_numpy(pr.x_true).cuda()) /
                        math.sqrt(pr.n))
            res[name] = {"status": info.status, "iters": info.iters,
                         "oracle_iters": stored_count(ORACLE_KEYS.get(name, "")),
                         "ms": round(ms, 2), "solves_per_s": round(1000.0 / ms, 3),
                         "true_relres": info.true_relres, "rms_err_vs_x_true": err}
            if name in ("sgs2_1_1_fp32", "sgs2_1_1_fp16") and x_ref is not None:
                res[name]["rel_err_vs_fp64_solution"] = float(
                    torch.linalg.norm(x - x_ref) / torch.linalg.norm(x_ref))
    h.close()
    return res


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
