#!/usr/bin/env python
"""Benchmark: smoothed time steps per second of the temporally parallel RTS
smoother (Alg. pkf filter pass with log-likelihood + Alg. prts smoother pass)
on the 2D constant-velocity tracking model (nx=4, ny=2, dt=0.1, q=1,
R=0.25 I) at T = 2^20, one sequence per GPU (weak scaling: every rank
smooths its own sequence; there is no data-path collective).

One step = one kf_rts_smooth call on one T-step sequence resident in HBM.
The L2 cache is flushed (256 MB write) between timed steps, outside the
timed events.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

FP32_LANES_PER_SM = 128      # Blackwell SM: 4 SMSPs x 32 FP32 lanes
N_SM = 152                   # GB300
SM_MAX_MHZ = 2070.0


# ------------------------------------------------------------------ work model
# FMA counts of the operator code (kf_math.cuh), derived in the design doc, with
# n = nx, m = ny, S = n(n+1)/2; an FMA counts 2 flops.

def lemma1_flops(n):
    S = n * (n + 1) // 2
    fma = 5 * n ** 3 + 3 * S * n + 5 * n * n + (n - 1) * (3 * n * n - n) // 2
    return 2 * fma + (3 * n * n - n) // 2 + n


def lemma2_flops(n):
    S = n * (n + 1) // 2
    return 2 * (2 * n ** 3 + n * n + S * n)


def rts_build_flops(n):
    S = n * (n + 1) // 2
    fma = n ** 3 + (S * n + sum(j for i in range(n) for j in range(i + 1))) + n * n * (n - 1) + 2 * n * n + S * n
    return 2 * fma + (S - n) + 2 * n * n + 2 * n


def filter_step_flops(n, m, loglik=True):
    # a work-efficient scan applies the operator ~2 times per element
    f = 2 * lemma1_flops(n) + 4 * n * m
    if loglik:
        f += 2 * (m * n + m * m + m + 2 * n * n + n) + n
    return f


def rts_step_flops(n):
    return 2 * lemma2_flops(n) + rts_build_flops(n)


def step_bytes(n, m, w):
    S = n * (n + 1) // 2
    filt = (m + n + S) * w                  # read y, write filter mean + packed cov
    rts = (n + S) * w + (n + n * n) * w     # read them back, write smoothed mean + full cov
    return filt, rts


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ reference (oracle) arm

def run_reference(args, rank, world):
    import oracle
    if rank != 0:
        return
    model = W.cv_model()
    Ts = min(args.T, 1 << 18)          # bounded sample of the workload per step
    y = W.simulate(model, Ts, seed=1)
    if args.precision != "fp64":
        y = y.astype(np.float32).astype(np.float64)

    def step():
        mf, Pf, ll = oracle.kf(model, y)
        oracle.rts(model, mf, Pf)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = args.steps * Ts / dt
    cpu = {"value": value, "unit": "smoothed steps/s", "cores": 1, "kind": "oracle",
           "sample": "sequential FP64 C Kalman filter + RTS smoother over %d steps of the workload per step" % Ts}
    print(json.dumps({
        "impl": "reference", "metric": "smoothed steps/s", "value": value, "unit": "smoothed steps/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded simulation of the model)",
        "config": workload_config(args, world), "cpu_baseline": cpu,
        "e2e": {"value": value, "unit": "smoothed steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def workload_config(args, world):
    return {"workload": "2D constant-velocity tracking (nx=4, ny=2, dt=0.1, q=1, R=0.25 I), one sequence of "
                        "T=2^%d per GPU, filter (with log-likelihood) + RTS smoother" % int(np.log2(args.T)),
            "T": args.T, "nx": 4, "ny": 2, "op": args.op, "scan": args.scan, "precision": args.precision,
            "parallelism": "one independent sequence per GPU (%d GPU)" % world,
            "l2": "flushed (256 MB write) between timed steps, outside the timed events"}


# ------------------------------------------------------------------ our arm

def cpu_baseline(args):
    import oracle
    model = W.cv_model()
    Ts = min(args.T, 1 << 20)
    y = W.simulate(model, Ts, seed=7).astype(np.float32).astype(np.float64)
    done, t0 = 0, time.perf_counter()
    while True:
        mf, Pf, _ = oracle.kf(model, y)
        oracle.rts(model, mf, Pf)
        done += Ts
        if time.perf_counter() - t0 > 10.0:
            break
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": "smoothed steps/s", "cores": 1, "kind": "oracle",
            "sample": "sequential FP64 C oracle (Kalman filter + RTS) over %d x %d steps of the same model, "
                      "%.1f s on one host core" % (done // Ts, Ts, dt)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "fp32_fp64solve"])
    ap.add_argument("--op", default="rts", choices=["rts", "tf"])
    ap.add_argument("--scan", default="dlb")
    ap.add_argument("--T", type=int, default=1 << 20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile", action="store_true",
                    help="warm-up and timed steps only (no soak, end-to-end pass, CPU baseline or FMA probe): "
                         "the form run under ncu")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import paper_2511_10363_gb300 as kf
    from paper_2511_10363_gb300 import build as kbuild

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    kbuild.build()

    model = W.cv_model()
    nx, ny, T = 4, 2, args.T
    dt = kf.dtype_of(args.precision)
    w = 8 if args.precision == "fp64" else 4
    y_host = torch.tensor(W.simulate(model, T, seed=1 + rank), dtype=dt).pin_memory()
    y = y_host.to("cuda")
    ms = torch.empty((T, nx), dtype=dt, device="cuda")
    Ps = torch.empty((T, nx, nx), dtype=dt, device="cuda")
    ll = torch.empty(1, dtype=torch.float64, device="cuda")
    ws = torch.empty(kf.kf_workspace_size(args.op, nx, ny, T, args.precision, args.scan), dtype=torch.uint8,
                     device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    fn = kf.kf_rts_smooth if args.op == "rts" else kf.kf_two_filter_smooth
    mdl = kf.Model(model)

    def step():
        fn(mdl, y, args.precision, args.scan, ms_out=ms, Ps_out=Ps, loglik=True, workspace=ws)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if kf.kf_sync_status() != 0:
        raise RuntimeError("kernel status error in warm-up")

    clocks = ClockSampler(local)
    if not args.profile:
        clocks.start()
        # untimed soak so that the clock sampler sees the GPU under this load
        t_soak = time.perf_counter()
        while time.perf_counter() - t_soak < 1.5:
            step()
            torch.cuda.synchronize()
    kf.kf_timing_reset()
    kf.kf_timing_enable(1)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()
        starts[k].record()
        step()
        ends[k].record()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    kf.kf_timing_enable(0)
    ck = clocks.stop()
    status = kf.kf_sync_status()
    if status != 0:
        raise RuntimeError("kernel status %d in the timed region" % status)
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = float(sum(step_ms))
    kinds = {"filter_scan": 0, "rts_scan": 1, "tf_scan": 2}
    kern = {}
    launches = 0
    for name, kd in kinds.items():
        n_l, t_ms = kf.timing_read(kd)
        launches += n_l
        if n_l:
            kern[name] = {"launches": n_l, "avg_ms": t_ms / n_l}
    for kd in (3, 4, 5):
        n_l, _ = kf.timing_read(kd)
        launches += n_l

    t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    max_ms = float(t.item())
    value = world * args.steps * T / (max_ms * 1e-3)

    if args.profile:
        if rank == 0:
            print(json.dumps({"metric": "smoothed steps/s", "value": value, "unit": "smoothed steps/s",
                              "profile_run": True, "kernels": kern, "gpu_launches": launches,
                              "config": workload_config(args, world)}))
        if dist:
            dist.destroy_process_group()
        return

    # ---- end to end through the public API with pinned host buffers
    ms_h = torch.empty((T, nx), dtype=dt).pin_memory()
    Ps_h = torch.empty((T, nx, nx), dtype=dt).pin_memory()
    ll_h = torch.empty(1, dtype=torch.float64).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ek = max(3, min(args.steps, 20))
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(ek):
        kf.rts_smooth_host(mdl, y_host, args.precision, args.scan, ms_h, Ps_h, ll_h, workspace=ws, op=args.op,
                           y_dev=y, ms_dev=ms, Ps_dev=Ps, ll_dev=ll)
    e1.record()
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    te = torch.tensor([e2e_ms], dtype=torch.float64, device="cuda")
    if dist:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e_value = world * ek * T / (float(te.item()) * 1e-3)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel
    fb, rb = step_bytes(nx, ny, w)
    f_flops = filter_step_flops(nx, ny)
    r_flops = rts_step_flops(nx)
    fma_peak = kf.measure_fma_peak(fp64=(args.precision == "fp64"))
    if args.precision == "fp64":
        alu_peak = fma_peak   # no vendor unit count for the FP64 pipe of this part: measured
        peak_src = "measured DFMA throughput (kf_measure_fma_peak)"
    else:
        alu_peak = N_SM * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6
        peak_src = "152 SMs x 128 FP32 lanes x 2 flops x 2070 MHz"
    hbm_peak = 6780.7e9
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            hbm_peak = float(json.load(f)["hbm_gbs"]) * 1e9
    except Exception:
        pass
    for name, fl, by in (("filter_scan", f_flops, fb), ("rts_scan", r_flops, rb)):
        if name in kern:
            k = kern[name]
            tsec = k["avg_ms"] * 1e-3
            k["alg_flops_per_step"] = fl
            k["alg_bytes_per_step"] = by
            k["tflops"] = fl * T / tsec / 1e12
            k["gbs"] = by * T / tsec / 1e9
            k["bound"] = "alu" if fl / by > alu_peak / hbm_peak else "hbm"
            k["frac"] = (k["tflops"] * 1e12 / alu_peak) if k["bound"] == "alu" else (k["gbs"] * 1e9 / hbm_peak)
    dom = max(kern, key=lambda n: kern[n]["avg_ms"])
    d = kern[dom]
    if d["bound"] == "alu":
        roof = {"kernel": dom, "bound": "alu", "achieved": d["tflops"], "peak": alu_peak / 1e12, "unit": "TFLOP/s",
                "frac": d["frac"], "traffic": None,
                "peak_source": peak_src + "; measured FFMA throughput %.1f TFLOP/s" % (fma_peak / 1e12)}
    else:
        roof = {"kernel": dom, "bound": "hbm", "achieved": d["gbs"], "peak": hbm_peak / 1e9, "unit": "GB/s",
                "frac": d["frac"], "traffic": None, "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    step_roof = 1.0 / (max(f_flops / alu_peak, fb / hbm_peak) + max(r_flops / alu_peak, rb / hbm_peak))

    out = {
        "metric": "smoothed steps/s", "value": value, "unit": "smoothed steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": max_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp64": "f64", "fp32_fp64solve": "f32+f64solve"}[args.precision],
        "data": "synthetic (seeded simulation of the model)", "config": workload_config(args, world),
        "roofline": roof,
        "kernels": kern,
        "step_roofline": {"steps_per_s": step_roof, "frac": value / world / step_roof},
        "e2e": {"value": e2e_value, "unit": "smoothed steps/s", "h2d_bytes_per_step": T * ny * w,
                "d2h_bytes_per_step": T * (nx + nx * nx) * w + 8},
        "gpu_launches": launches,
        "clocks": ck,
    }
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args)
    print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
