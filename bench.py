#!/usr/bin/env python
"""Throughput of the MPR gap-filling hot path on GB300: site-updates/s.

One step = one whole gap-filling job through the C ABI on a synthetic Gaussian field with the
exponential covariance of the paper's Sec. 3 (m = 50, sigma = 10, kappa = 0.2) at L = 4096 with
90 % of the sites removed: mapping + initial state, temperature tuning, 2000 equilibration and
200 sampling sweeps, prediction. A site-update is one hybrid move (Metropolis + over-relaxation)
of one prediction site; the library counts them exactly (tuning probes included).

  value  : inputs resident in device memory (mpr_create_dev / mpr_predict_dev)
  e2e    : host buffers (pinned) through mpr_create / mpr_predict, copies inside the timing
  --impl reference : the FP64 CPU oracle on this host's cores, on a bounded sample of sweeps

Runs as one process per GPU under torchrun for N > 1: independent problems per rank (no data
exchange), max time over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# MUFU lanes per SM per clock when the probe cannot run (nominal, times the device's own SM count
# and maximum clock): 16 for each of sin, cos, ex2 and rcp
MUFU_FALLBACK_PER_CLK = {"sin": 16, "cos": 16, "ex2": 16, "rcp": 16}
STORE_BYTES = {"D": 8, "S": 4, "H": 2, "B": 2}
# Temperature of the oracle's timed sweeps when no tuned value is at hand (--impl reference): the
# temperature the tuning reaches on the default workload (4096^2, p = 0.9, field seed 1, mask
# seed 101), T = 0.0649; the measured arm times its cpu_baseline at its own tuned T.
WORKLOAD_T = 0.065


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["mine", "reference"], default="mine")
    ap.add_argument("--L", type=int, default=4096)
    ap.add_argument("--p", type=float, default=0.9)
    ap.add_argument("--setup", default="HDS", help="precision X_S X_E X_F (Sec. 2), e.g. HDS, SDS")
    ap.add_argument("--acc", default="f64", choices=["f64", "kahan"])
    ap.add_argument("--equil", type=int, default=2000)
    ap.add_argument("--samples", type=int, default=200)
    ap.add_argument("--tune-eq", type=int, default=200, help="sweeps per tuning probe before measuring")
    ap.add_argument("--tune-meas", type=int, default=50, help="measured sweeps per tuning probe")
    ap.add_argument("--ddd-sweeps", type=int, default=10, help="FP64 sweeps timed for the speedup")
    ap.add_argument("--no-ddd-job", action="store_true",
                    help="skip the FP64 (DDD) job on the same problem that gives the accuracy gap")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of the oracle sample")
    ap.add_argument("--workload", choices=["single", "batch"], default="single",
                    help="single: one L x L field; batch: many uneven problems in one launch")
    ap.add_argument("--batch-n", type=int, default=256)
    ap.add_argument("--no-autotune", action="store_true", help="batch: default launch shape")
    ap.add_argument("--sweep-kernel", type=int, default=-1, choices=[-1, 0, 1],
                    help="FP32 sweep kernel: -1 automatic (timed per job), 0 tile per block, 1 TMA-fed")
    ap.add_argument("--proposal", default="",
                    help="bounded Metropolis proposals 'WIDTH,TARGET' (mpr_set_proposal); default uniform")
    ap.add_argument("--ref-T", type=float, default=WORKLOAD_T,
                    help="--impl reference: temperature of the oracle's timed sweeps")
    ap.add_argument("--no-extra-configs", action="store_true",
                    help="skip the short runs of the batch workload (config 4) and the 16384^2 "
                         "field (config 5) that the default line reports beside the main number")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    return ap.parse_args()


# ------------------------------------------------------------------------------------------------
# distributed plumbing (barrier + max over ranks only; nothing of the method crosses ranks)
# ------------------------------------------------------------------------------------------------

class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch
            import torch.distributed as dist

            backend = "nccl" if torch.cuda.is_available() else "gloo"
            if backend == "nccl":
                torch.cuda.set_device(self.local)
            dist.init_process_group(backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, v: float) -> float:
        if not self.pg:
            return v
        import torch

        dev = "cuda" if torch.cuda.is_available() else "cpu"
        t = torch.tensor([v], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def sum(self, v: float) -> float:
        if not self.pg:
            return v
        import torch

        dev = "cuda" if torch.cuda.is_available() else "cpu"
        t = torch.tensor([v], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ------------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[5 + k] == "Active"})
        pw = [float(r[3]) for r in self.rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "power_w_max": max(pw) if pw else None, "samples": len(self.rows)}


# ------------------------------------------------------------------------------------------------
# the measured arm
# ------------------------------------------------------------------------------------------------

KERNEL_SOURCES = {
    "mpr::sweep_f32_kernel": ("mpr_tile_f32.cuh", "mpr_sweep_f32.cuh", "mpr_device.cuh"),
    "mpr::sweep_f32_tma_kernel": ("mpr_tile_f32.cuh", "mpr_sweep_tma.cu", "mpr_tma.cuh",
                                  "mpr_device.cuh"),
    "mpr::sweep_kernel": ("mpr_sweep.cu", "mpr_device.cuh"),
}


def sweep_kernel_id(kernel: str = "mpr::sweep_f32_kernel") -> str:
    """Hash of a sweep kernel's sources: ties stored ncu counters to the code they came from."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1910_08448_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def stored_counters(kernel_id: str, kernel: str, workload: str):
    """ncu counters of this kernel version on this workload (profiles/dram_traffic.json), or {}:
    DRAM bytes per launch and the share of issue slots the kernel kept busy."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return {}
    e = d.get(workload)
    if not e or e.get("kernel_id") != kernel_id or e.get("kernel") != kernel:
        return {}
    return e


# kernel that ran the plain passes, by mpr_info.sweep_kernel
SWEEP_KERNELS = {-1: "mpr::sweep_kernel", 0: "mpr::sweep_f32_kernel", 1: "mpr::sweep_f32_tma_kernel"}


def mufu_rates(local_rank: int, sm_mhz_max: float, sm_count: int):
    """Special-function throughput (ops/s) measured by the probe that build() compiles
    (paper_1910_08448_gb300/probe/mufu_rate.cu), on this rank's GPU; nominal lanes x clock if it
    cannot run."""
    exe = os.path.join(ROOT, "paper_1910_08448_gb300", "_build", "mufu_rate")
    env = dict(os.environ, CUDA_VISIBLE_DEVICES=str(local_rank))
    if "CUDA_VISIBLE_DEVICES" in os.environ:
        vis = os.environ["CUDA_VISIBLE_DEVICES"].split(",")
        env["CUDA_VISIBLE_DEVICES"] = vis[local_rank] if local_rank < len(vis) else vis[0]
    try:
        r = subprocess.run([exe], capture_output=True, text=True, timeout=60, env=env)
        d = json.loads(r.stdout.strip().splitlines()[-1])
        rates = {k: d[f"{k}_per_s"] for k in ("sin", "cos", "ex2", "rcp")}
        if all(v > 0 for v in rates.values()):
            return rates, "probe"
    except (OSError, ValueError, KeyError, IndexError, subprocess.SubprocessError):
        pass
    return {k: sm_count * v * sm_mhz_max * 1e6 for k, v in MUFU_FALLBACK_PER_CLK.items()}, "nominal"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return d.get("hbm_gbs", 6800.0), d.get("sm_max_mhz", 2070.0), "measured"
    except (OSError, ValueError):
        return 6800.0, 2070.0, "fallback"


def run_mine(args, dist: Dist):
    import numpy as np
    import torch

    import mpr_inputs
    import paper_1910_08448_gb300 as mpr

    dev = torch.device("cuda", dist.local)
    torch.cuda.set_device(dev)
    mpr.load()
    L, p = args.L, args.p
    pr = mpr_inputs.make_problem(L, L, p, field_seed=1 + dist.rank, mask_seed=101 + dist.rank,
                                 periodic=L > 4096, device=dev)
    zt = torch.from_numpy(pr.z).to(dev)
    mt = torch.from_numpy(pr.mask).to(dev)
    out = torch.empty_like(zt)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2
    seed = 7 + dist.rank
    proposal = tuple(float(v) for v in args.proposal.split(",")) if args.proposal else None

    # phase boundaries of a job: CUDA events on the handle's stream (the legacy default stream,
    # torch's current stream here), so tuning, equilibration and sampling are reported apart
    PHASES = ("setup", "tune", "equil", "sample", "predict")

    def mark(marks):
        if marks is not None:
            e = torch.cuda.Event(enable_timing=True)
            e.record()
            marks.append(e)

    def step_device(profile=False, marks=None):
        mark(marks)
        h = mpr.mpr_create_dev(zt, mt)
        try:
            mpr.mpr_set_options(h, args.setup, seed=seed, acc=args.acc)
            if args.sweep_kernel >= 0:
                mpr.mpr_set_sweep_kernel(h, args.sweep_kernel)
            if proposal:
                mpr.mpr_set_proposal(h, *proposal)
            mpr.mpr_set_tuning(h, n_eq=args.tune_eq, n_meas=args.tune_meas)
            if profile:
                mpr.mpr_set_profiling(h, True)
            mark(marks)
            T, _ = mpr.mpr_tune_temperature(h)
            mark(marks)
            mpr.mpr_run(h, args.equil, 0)      # the same chain as one mpr_run(equil, samples)
            mark(marks)
            mpr.mpr_run(h, 0, args.samples)
            mark(marks)
            mpr.mpr_predict_dev(h, out)
            info = mpr.mpr_get_info(h)
        finally:
            mpr.mpr_destroy(h)
        mark(marks)
        return info

    for _ in range(args.warmup):
        step_device()
    torch.cuda.synchronize()

    # ---- timed: K steps, inputs resident, L2 flushed between steps outside the events ----
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    infos = []
    marks = [[] for _ in range(args.steps)]
    dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dist.local) as clk:
        t_wall = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record()
            infos.append(step_device(profile=True, marks=marks[k]))
            ev[k][1].record()
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    dist.barrier()
    torch.cuda.synchronize()
    ms_local = sum(a.elapsed_time(b) for a, b in ev)
    ms = dist.max(ms_local)
    updates_local = float(sum(i["site_updates"] for i in infos))
    updates = dist.sum(updates_local)
    value = updates / (ms / 1e3)
    launches = int(sum(i["kernel_launches"] for i in infos))
    phases_ms = {name: sum(m[i].elapsed_time(m[i + 1]) for m in marks) / args.steps
                 for i, name in enumerate(PHASES)}

    # ---- dominant kernel: sweep half-pass, device time from CUDA events inside the steps ----
    sweep_ms = sum(i["prof_sweep_ms"] for i in infos)
    sweep_launches = sum(i["prof_sweep_launches"] for i in infos)
    t_launch = (sweep_ms / 1e3) / max(sweep_launches, 1)
    N = L * L
    b = STORE_BYTES[args.setup[0]]
    bytes_launch = (N / 2) * (b * (2 + p) + 1 / 8)
    hbm_gbs, sm_mhz_max, src = peaks()
    # MUFU work of one pass: every site's sin/cos once (staged as a neighbour); per prediction
    # site its own sin/cos, the proposal's sin/cos, one ex2 and one rcp. Each at its own measured
    # rate; expressed in sin-equivalent operations at the sin rate.
    rates, mufu_src = mufu_rates(dist.local, sm_mhz_max,
                                 torch.cuda.get_device_properties(dev).multi_processor_count)
    r_sc = min(rates["sin"], rates["cos"])
    t_mufu = (N / 2) * (2 / r_sc + p * (4 / r_sc + 1 / rates["ex2"] + 1 / rates["rcp"]))
    mufu_launch = t_mufu * r_sc
    mufu_peak = r_sc
    t_hbm = bytes_launch / (hbm_gbs * 1e9)
    kname = SWEEP_KERNELS[infos[-1]["sweep_kernel"]]
    kid = sweep_kernel_id(kname)
    workload = f"L{L}_p{p}_{args.setup}" + ("_bounded" if proposal else "")
    counters = stored_counters(kid, kname, workload)
    traffic = counters.get("bytes_per_launch")
    if t_hbm >= t_mufu:
        roof = {"bound": "hbm", "achieved": bytes_launch / t_launch / 1e9, "peak": hbm_gbs,
                "unit": "GB/s"}
    else:
        roof = {"bound": "alu", "achieved": mufu_launch / t_launch / 1e9,
                "peak": mufu_peak / 1e9, "unit": "Gop/s (MUFU, sin-equivalent)"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof.update({"traffic": traffic,
                 # what limits this kernel: instruction issue (ncu smsp__issue_active, same kernel
                 # version), next to the MUFU and HBM fractions
                 "issue_active_ncu": counters.get("issue_active"),
                 "peak_source": src if roof["bound"] == "hbm" else mufu_src,
                 "kernel": kname,
                 "launch_us": t_launch * 1e6, "algorithmic_bytes_per_launch": bytes_launch,
                 "algorithmic_mufu_per_launch": mufu_launch, "kernel_id": kid,
                 "hbm_frac": bytes_launch / t_launch / 1e9 / hbm_gbs,
                 "mufu_frac": mufu_launch / t_launch / mufu_peak,
                 "mufu_rates_per_s": rates, "mufu_rates_source": mufu_src})

    # ---- FP64 (DDD) GPU path on the same lattice: speedup of the sweep kernel ----
    T_last = infos[-1]["T"]
    ddd = None
    if args.ddd_sweeps > 0:
        h = mpr.mpr_create_dev(zt, mt)
        try:
            mpr.mpr_set_options(h, "DDD", seed=seed)
            mpr.mpr_set_temperature(h, T_last)
            mpr.mpr_set_profiling(h, True)
            mpr.mpr_run(h, 2, 0)
            i0 = mpr.mpr_get_info(h)
            mpr.mpr_run(h, args.ddd_sweeps, 0)
            i1 = mpr.mpr_get_info(h)
        finally:
            mpr.mpr_destroy(h)
        ddd_s = (i1["prof_sweep_ms"] - i0["prof_sweep_ms"]) / 1e3
        ddd_rate = (i1["site_updates"] - i0["site_updates"]) / ddd_s
        fast_rate = infos[-1]["n_pred"] / (2 * t_launch)
        ddd = {"fp64_sweep_site_updates_per_s": ddd_rate,
               "sweep_site_updates_per_s": fast_rate, "speedup_vs_fp64_gpu": fast_rate / ddd_rate}

    # ---- the same job in FP64 (DDD) on the same problem and seed, outside the timed region: the
    # reference of the metric's accuracy clause (MAE of the reduced-precision job within 1 % of
    # the FP64 job's) ----
    ddd_job = None
    if not args.no_ddd_job and args.setup != "DDD":
        out_d = torch.empty_like(zt)
        h = mpr.mpr_create_dev(zt, mt)
        try:
            mpr.mpr_set_options(h, "DDD", seed=seed)
            if proposal:
                mpr.mpr_set_proposal(h, *proposal)
            mpr.mpr_set_tuning(h, n_eq=args.tune_eq, n_meas=args.tune_meas)
            t0 = time.perf_counter()
            T_d, _ = mpr.mpr_tune_temperature(h)
            mpr.mpr_run(h, args.equil, args.samples)
            mpr.mpr_predict_dev(h, out_d)
            info_d = mpr.mpr_get_info(h)
            torch.cuda.synchronize()
            t_d = time.perf_counter() - t0
        finally:
            mpr.mpr_destroy(h)
        ddd_job = {"zhat": out_d.cpu().numpy(), "T": T_d, "e_bond_mean": info_d["e_bond_mean"],
                   "seconds": t_d, "site_updates": info_d["site_updates"]}

    # ---- end to end through the host API: pinned inputs, H2D + D2H inside the timing ----
    e2e = None
    if not args.no_e2e:
        zp = torch.from_numpy(pr.z).pin_memory()
        mp = torch.from_numpy(pr.mask).pin_memory()
        zhat_host = torch.empty_like(zp).pin_memory()
        zn, mn, on = zp.numpy(), mp.numpy(), zhat_host.numpy()
        import ctypes

        lib = mpr.load()
        e_ms, e_upd = 0.0, 0
        dist.barrier()
        for k in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h = mpr.mpr_create(zn, mn)
            try:
                mpr.mpr_set_options(h, args.setup, seed=seed, acc=args.acc)
                if args.sweep_kernel >= 0:
                    mpr.mpr_set_sweep_kernel(h, args.sweep_kernel)
                if proposal:
                    mpr.mpr_set_proposal(h, *proposal)
                mpr.mpr_set_tuning(h, n_eq=args.tune_eq, n_meas=args.tune_meas)
                mpr.mpr_tune_temperature(h)
                mpr.mpr_run(h, args.equil, args.samples)
                mpr._check(lib.mpr_predict(h, on.ctypes.data_as(ctypes.c_void_p)))
                e_upd += mpr.mpr_get_info(h)["site_updates"]
            finally:
                mpr.mpr_destroy(h)
            torch.cuda.synchronize()
            e_ms += (time.perf_counter() - t0) * 1e3
        e_ms = dist.max(e_ms)
        e_upd = dist.sum(float(e_upd))
        e2e = {"value": e_upd / (e_ms / 1e3), "unit": "site-updates/s",
               "h2d_bytes_per_step": int(pr.z.nbytes + pr.mask.nbytes),
               "d2h_bytes_per_step": int(pr.z.nbytes), "ms_per_step": e_ms / args.steps}

    # ---- accuracy of this run against the truth (prediction sites) ----
    zhat = out.cpu().numpy()
    pred = pr.mask == 0
    err = (zhat - pr.z)[pred]
    acc_rep = {"mae": float(np.mean(np.abs(err))), "rmse": float(np.sqrt(np.mean(err ** 2))),
               "T": T_last, "e_bond_mean": infos[-1]["e_bond_mean"],
               "e_sample": infos[-1]["e_sample"]}
    if ddd_job is not None:
        err_d = (ddd_job["zhat"] - pr.z)[pred]
        mae_d = float(np.mean(np.abs(err_d)))
        rmse_d = float(np.sqrt(np.mean(err_d ** 2)))
        acc_rep.update({
            "mae_fp64_gpu": mae_d, "rmse_fp64_gpu": rmse_d, "T_fp64_gpu": ddd_job["T"],
            "e_bond_fp64_gpu": ddd_job["e_bond_mean"],
            # relative gaps of this setup's job to the FP64 job (same problem, seed and sweeps)
            "mae_gap": acc_rep["mae"] / mae_d - 1.0, "rmse_gap": acc_rep["rmse"] / rmse_d - 1.0,
            "e_bond_gap": acc_rep["e_bond_mean"] / ddd_job["e_bond_mean"] - 1.0,
            "fp64_job_seconds": ddd_job["seconds"],
            "fp64_job_site_updates_per_s": ddd_job["site_updates"] / ddd_job["seconds"]})

    return {
        "value": value, "ms": ms, "updates": updates, "launches": launches, "roof": roof,
        "ddd": ddd, "e2e": e2e, "clocks": clk.summary(), "accuracy": acc_rep,
        "wall_s": t_wall, "site_updates_per_step": updates_local / args.steps,
        "sweeps_per_step": infos[-1]["sweep"], "n_pred": infos[-1]["n_pred"], "problem": pr,
        "phases_ms": phases_ms,
    }


def run_batch(args, dist):
    """Config 4: args.batch_n independent problems (side log-uniform 64..1024, aspect up to 4:1,
    p in {0.33, 0.66, 0.9}, kappa in [0.05, 0.5]) filled by one persistent launch per step
    (tuning + equilibration + sampling of every problem) plus the predictions to host memory."""
    import numpy as np
    import torch

    import mpr_inputs
    import paper_1910_08448_gb300 as mpr

    dev = torch.device("cuda", dist.local)
    torch.cuda.set_device(dev)
    mpr.load()
    probs = mpr_inputs.make_batch(args.batch_n, seed=1 + dist.rank)
    outs = [torch.empty(p.z.shape, dtype=torch.float64).pin_memory().numpy() for p in probs]
    lib = mpr.load()
    import ctypes

    b = mpr.mpr_batch_create([p.z for p in probs], [p.mask for p in probs], args.setup,
                             seed=7 + dist.rank, acc=args.acc)
    try:
        mpr.mpr_batch_set_tuning(b, n_eq=args.tune_eq, n_meas=args.tune_meas)
        if args.no_autotune:
            rows, cols, bps, mode = 32, 128, 0, 2
            mpr.mpr_batch_set_launch(b, rows, cols, bps, mode)
        else:
            rows, cols, bps, mode = mpr.mpr_batch_autotune(b, 10)

        fills = []

        def step():
            T, st = mpr.mpr_batch_fill(b, args.equil, args.samples)
            fills.append(mpr.mpr_batch_get_stats(b))
            for i, o in enumerate(outs):
                mpr._check(lib.mpr_batch_predict(b, i, o.ctypes.data_as(ctypes.c_void_p)))
            return T, st

        def updates():
            return sum(mpr.mpr_batch_get_info(b, i)["site_updates"] for i in range(len(probs)))

        for _ in range(args.warmup):
            step()
        dist.barrier()
        torch.cuda.synchronize()
        u0 = updates()
        with ClockSampler(dist.local) as clk:
            t0 = time.perf_counter()
            for _ in range(args.steps):
                T, st = step()
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
        dist.barrier()
        u1 = updates()
        launches = mpr.mpr_batch_get_info(b, 0)["kernel_launches"]
        sweeps = [mpr.mpr_batch_get_info(b, i)["sweep"] for i in range(len(probs))]
        # a fill with every problem at a fixed temperature: no tuning tail, equal sweeps
        u_a = updates()
        mpr.mpr_batch_fill(b, 200, 0, T=np.full(len(probs), 0.3))
        fixed = mpr.mpr_batch_get_stats(b)
        fixed_rate = (updates() - u_a) / (fixed["fill_ms"] / 1e3)
    finally:
        mpr.mpr_batch_destroy(b)
    ms = dist.max(dt * 1e3)
    upd = dist.sum(float(u1 - u0))
    maes = []
    for p, o in zip(probs, outs):
        pred = p.mask == 0
        maes.append(float(np.mean(np.abs(o - p.z)[pred])))
    return {"value": upd / (ms / 1e3), "ms": ms, "tile": [rows, cols], "blocks_per_sm": bps, "mode": mode,
            "clocks": clk.summary(), "n_problems": len(probs),
            "sites": int(sum(p.z.size for p in probs)),
            "pred_sites": int(sum(int((p.mask == 0).sum()) for p in probs)),
            "mean_mae": float(np.mean(maes)), "tune_status_nonzero": int(np.count_nonzero(st)),
            "T_range": [float(np.min(T)), float(np.max(T))], "launches": launches,
            "last_fill": fills[-1], "fixed_T_fill": dict(fixed, site_updates_per_s=fixed_rate),
            "sweeps_per_problem": [int(np.min(sweeps)), int(np.median(sweeps)), int(np.max(sweeps))]}


def run_extra_configs(args, dist):
    """Short runs of the two other workloads that are not the metric's own, reported as sub-objects
    of the default line: the batch of 256 uneven problems (config 4, HDS, tune + 2000 + 200 per
    problem, one step after one warm-up step) and the 16384^2 field (config 5, SDS, FP64
    accumulators, tune + 500 + 100, one step after one warm-up step). Each is timed like its own
    bench line (python bench.py --workload batch; python bench.py --L 16384 --setup SDS --equil
    500 --samples 100), with fewer steps."""
    import copy

    out = {}
    a = copy.copy(args)
    a.workload, a.steps, a.warmup = "batch", 1, 1
    b = run_batch(a, dist)
    out["batch"] = {"config": "4: 256 problems, side log-uniform 64..1024, aspect <= 4:1, "
                              "p in {0.33,0.66,0.9}, kappa in [0.05,0.5]; tune + 2000 + 200",
                    "setup": a.setup, "value": b["value"], "unit": "site-updates/s",
                    "ms_per_step": b["ms"], "steps": 1, "warmup": 1,
                    "tile_rows_x_cols": b["tile"], "blocks_per_sm": b["blocks_per_sm"],
                    "mode": ["persistent cooperative kernel", "persistent kernel in a one-node graph",
                             "graph with device-side while loop"][b["mode"]],
                    "pred_sites": b["pred_sites"], "sites": b["sites"],
                    "mean_mae": b["mean_mae"],
                    "fixed_T_site_updates_per_s": b["fixed_T_fill"]["site_updates_per_s"],
                    "clocks": b["clocks"]}
    a = copy.copy(args)
    a.L, a.setup, a.equil, a.samples = 16384, "SDS", 500, 100
    a.steps, a.warmup, a.no_e2e, a.no_ddd_job, a.ddd_sweeps = 1, 1, True, True, 0
    r = run_mine(a, dist)
    out["config5"] = {"config": "5: 16384x16384, 90% removed, SDS (FP32 spins, FP64 energy and "
                                "accumulators); tune + 500 + 100",
                      "value": r["value"], "unit": "site-updates/s", "ms_per_step": r["ms"],
                      "steps": 1, "warmup": 1,
                      "roofline": {k: r["roof"][k] for k in ("bound", "achieved", "peak", "unit",
                                                             "frac", "hbm_frac", "mufu_frac",
                                                             "launch_us", "kernel")},
                      "mae": r["accuracy"]["mae"], "T": r["accuracy"]["T"],
                      "clocks": r["clocks"]}
    return out


def oracle_sample(L, p, setup, seconds, seed=7, pr=None, T=None):
    """The FP64 oracle, as it stands, on a bounded number of sweeps of the same workload at the
    job's temperature T."""
    import mpr_inputs
    import oracle

    oracle.build()
    if pr is None:
        pr = mpr_inputs.make_problem(L, L, p, field_seed=1, mask_seed=101)
    o = oracle.Oracle(L, L, seed=seed, ubits=32 if setup[2] == "D" else 23)
    phi, _, _ = o.map(pr.z, pr.mask)
    phi = o.init(phi, pr.mask)
    n_pred = int((pr.mask == 0).sum())
    t0 = time.perf_counter()
    T = WORKLOAD_T if T is None else T
    phi, _, _ = o.run(phi, pr.mask, T, 0, 1)
    t1 = time.perf_counter() - t0
    n = max(1, int(seconds / max(t1, 1e-9)) - 1)
    t0 = time.perf_counter()
    o.run(phi, pr.mask, T, 1, n)
    t = time.perf_counter() - t0
    return {"value": n * n_pred / t, "unit": "site-updates/s", "cores": 1, "kind": "oracle",
            "sample": f"{n} hybrid sweeps of the {L}x{L} p={p} lattice at T={T:.4g} "
                      f"({n * n_pred} site-updates, {t:.1f} s, 1 thread)"}


def _oracle_worker(args):
    """One oracle replica for the all-cores sample: its own chain (seed) on the shared problem."""
    zpath, mpath, L, setup, seed, n, T, barrier, queue = args
    import numpy as np

    import oracle

    z = np.load(zpath)
    mask = np.load(mpath)
    o = oracle.Oracle(L, L, seed=seed, ubits=32 if setup[2] == "D" else 23)
    phi, _, _ = o.map(z, mask)
    phi = o.init(phi, mask)
    n_pred = int((mask == 0).sum())
    phi, _, _ = o.run(phi, mask, T, 0, 1)   # warm-up sweep (page-in), untimed
    barrier.wait()
    t0 = time.monotonic()
    o.run(phi, mask, T, 1, n)
    queue.put((n * n_pred, t0, time.monotonic()))


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_sample_cores(L, p, setup, seconds, pr, workers=None, seed=7, T=None):
    """The oracle as it stands on every host core at once: one independent replica (own chain) per
    process, all started together behind a barrier; value = all site-updates / the wall time from
    the first start to the last finish (CLOCK_MONOTONIC is shared by the processes). Processes
    are spawned, never forked, so a CUDA context in the parent is not inherited."""
    import multiprocessing as mp
    import shutil
    import tempfile

    import numpy as np

    import oracle

    oracle.build()
    T = WORKLOAD_T if T is None else T
    single = oracle_sample(L, p, setup, min(seconds, 6.0), seed=seed, pr=pr, T=T)
    workers = workers or host_cores()
    # memory guard: each replica holds the data and about two copies of the state (FP64); use at
    # most a quarter of the host's available memory
    need = L * L * (3 * 8 + 1) + (64 << 20)
    try:
        with open("/proc/meminfo") as fh:
            avail = next(int(ln.split()[1]) * 1024 for ln in fh if ln.startswith("MemAvailable:"))
        workers = min(workers, max(1, int(0.25 * avail / need)))
    except (OSError, StopIteration, ValueError):
        workers = min(workers, 4)
    if workers <= 1:
        return single
    # one replica's sweeps take about its single-thread time (more under memory contention)
    n_pred = int((pr.mask == 0).sum())
    t_sweep = n_pred / single["value"]
    n = max(1, int(seconds / t_sweep / 2))
    tmp = tempfile.mkdtemp(prefix="mpr_oracle_")
    try:
        zpath, mpath = os.path.join(tmp, "z.npy"), os.path.join(tmp, "mask.npy")
        np.save(zpath, np.asarray(pr.z, np.float64))
        np.save(mpath, np.asarray(pr.mask, np.uint8))
        ctx = mp.get_context("spawn")
        barrier = ctx.Barrier(workers)
        queue = ctx.Queue()
        procs = [ctx.Process(target=_oracle_worker,
                             args=((zpath, mpath, L, setup, seed + 1 + i, n, T, barrier, queue),))
                 for i in range(workers)]
        for pr_ in procs:
            pr_.start()
        res = [queue.get(timeout=600) for _ in procs]
        for pr_ in procs:
            pr_.join(timeout=60)
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
    upd = sum(r[0] for r in res)
    wall = max(r[2] for r in res) - min(r[1] for r in res)
    return {"value": upd / wall, "unit": "site-updates/s", "cores": workers, "kind": "oracle",
            "sample": f"{workers} processes, each {n} hybrid sweeps of its own chain on the {L}x{L} "
                      f"p={p} lattice at T={T:.4g} ({upd} site-updates in {wall:.1f} s wall)",
            "single_thread": {"value": single["value"], "sample": single["sample"]}}


def main():
    args = parse()
    dist = Dist()
    metric = f"site-updates/s at L={args.L} p={args.p}"
    workload = (f"MPR gap filling, {args.L}x{args.L} Gaussian field (exp. covariance, kappa=0.2), "
                f"{int(args.p * 100)}% removed: tune + {args.equil} equil + {args.samples} samples")
    config = {"workload": workload, "L": args.L, "p": args.p, "setup": args.setup,
              "acc": args.acc, "equil": args.equil, "samples": args.samples,
              "tune_probe_sweeps": [args.tune_eq, args.tune_meas],
              "l2": "flushed between steps (512 MB write)"}
    if args.proposal:
        config["proposal"] = args.proposal   # bounded Metropolis proposals: width, target

    if args.impl == "reference":
        if dist.rank == 0:
            import torch  # noqa: F401  (same process layout as the measured arm)

            import mpr_inputs

            pr = mpr_inputs.make_problem(args.L, args.L, args.p, field_seed=1, mask_seed=101)
            vals = []
            # warm-up steps: one single-thread sample each (pages the oracle and the data in)
            for k in range(args.warmup):
                oracle_sample(args.L, args.p, args.setup, 2.0, pr=pr, T=args.ref_T)
            for k in range(args.steps):
                vals.append(oracle_sample_cores(args.L, args.p, args.setup, args.cpu_seconds / 2,
                                                pr, T=args.ref_T))
            v = statistics.mean(r["value"] for r in vals)
            line = {"metric": metric, "value": v, "unit": "site-updates/s", "n_gpus": args.gpus,
                    "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
                    "impl": "reference", "dtype": "f64", "data": "synthetic", "config": config,
                    "cpu_baseline": {"value": v, "unit": "site-updates/s",
                                     "cores": vals[-1]["cores"], "kind": "oracle",
                                     "sample": vals[-1]["sample"],
                                     "single_thread": vals[-1].get("single_thread")},
                    "e2e": {"value": v, "unit": "site-updates/s", "h2d_bytes_per_step": 0,
                            "d2h_bytes_per_step": 0},
                    "vs_baseline": None}
            print(json.dumps(line), flush=True)
        dist.close()
        return

    if args.workload == "batch":
        res = run_batch(args, dist)
        if dist.rank == 0:
            line = {
                "metric": f"site-updates/s, batch of {res['n_problems']} problems",
                "value": res["value"], "unit": "site-updates/s", "n_gpus": dist.world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["ms"] / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"{res['n_problems']} independent problems, side "
                                       "log-uniform 64..1024, aspect <= 4:1, p in {0.33,0.66,0.9}, "
                                       "kappa in [0.05,0.5]; one launch per step (tune + "
                                       f"{args.equil} equil + {args.samples} samples) + predictions",
                           "setup": args.setup, "acc": args.acc, "sites": res["sites"],
                           "pred_sites": res["pred_sites"],
                           "autotuned_tile_rows_x_cols": res["tile"],
                           "autotuned_blocks_per_sm": res["blocks_per_sm"],
                           "autotuned_mode": ["persistent cooperative kernel",
                                              "persistent kernel in a one-node graph",
                                              "graph with device-side while loop"][res["mode"]],
                           "l2": "inputs larger than L2 (pooled state of all problems)"},
                "clocks": res["clocks"], "gpu_launches": res["launches"],
                "accuracy": {"mean_mae": res["mean_mae"], "T_range": res["T_range"],
                             "tune_not_converged": res["tune_status_nonzero"]},
                "launch_stats": {"last_fill": res["last_fill"], "fixed_T_fill": res["fixed_T_fill"],
                                 "sweeps_per_problem_min_med_max_cumulative": res["sweeps_per_problem"]},
            }
            print(json.dumps(line), flush=True)
        dist.close()
        return

    res = run_mine(args, dist)
    extra = {}
    if dist.world == 1 and args.workload == "single" and not args.no_extra_configs and args.L == 4096:
        extra = run_extra_configs(args, dist)
    cpu = None
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu:
        cpu = oracle_sample_cores(args.L, args.p, args.setup, args.cpu_seconds, res["problem"],
                                  T=res["accuracy"]["T"])
    if dist.rank == 0:
        line = {
            "metric": metric, "value": res["value"], "unit": "site-updates/s",
            "n_gpus": dist.world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": res["ms"] / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": {"D": "f64", "S": "f32", "H": "f16+f32"}[args.setup[2]],
            "data": "synthetic", "config": config,
            "roofline": res["roof"], "cpu_baseline": cpu, "e2e": res["e2e"],
            "gpu_launches": res["launches"], "clocks": res["clocks"],
            "fp64_gpu": res["ddd"], "accuracy": res["accuracy"],
            "site_updates_per_step": res["site_updates_per_step"],
            "sweeps_per_step": res["sweeps_per_step"], "wall_s_timed": res["wall_s"],
            # device time per job by phase (CUDA events): set-up, tuning, equilibration, sampling,
            # prediction and release
            "phases_ms": res["phases_ms"],
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    dist.close()


if __name__ == "__main__":
    main()
