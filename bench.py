#!/usr/bin/env python
"""Benchmark of the Fast-QMMD hot path on GB300.

One step = one XL-BOMD (Fast-QMMD) step of the 2048-atom water-like system
(682 O + 1366 H, n = 4094 orbitals, 1.0 g/cc, seed 0): half kick + drift,
the n update of Eq. Verl_n, H[n], D by SP2 (tensor-core projections + FP64
refinement), Mulliken charges, forces and energy, half kick.  Every stage
runs in libtbmd's CUDA kernels; state stays on the device.

value = SP2 D-matrix throughput: algorithmic flops of the purification
(2 n^3 per projection, main phase + refinement, counted from the device
reports of every timed step) / timed wall time of the whole steps.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Multi-GPU: independent replicas (one system per rank, no collective in the
data path); value = all ranks' flops / max-over-ranks time.
"""

from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SP2 D-matrix TFLOP/s (% peak) & XL-BOMD steps/s vs FP64 path; p50/p99 latency"
WORKLOAD = ("water-like orthogonal SCC-TB, 2048 atoms (682 O + 1366 H), n=4094 orbitals, "
            "1.0 g/cc periodic cube, seed 0; one XL-BOMD (Fast-QMMD) step per step")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="tf32x3", choices=["tf32", "tf32x3", "bf16", "bf16x3"])
    ap.add_argument("--refine", type=int, default=3)
    ap.add_argument("--natoms", type=int, default=2048,
                    help="atoms of the water-like system (2048 = the headline workload)")
    ap.add_argument("--scf-iters", type=int, default=12)
    ap.add_argument("--no-check", action="store_true", help="skip the accuracy check against the oracle")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64-path step")
    return ap.parse_args()


# ---------------------------------------------------------------- utilities

def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        d["source"] = "measured"
        return d
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- CPU oracle

def cpu_oracle_sample(max_seconds: float = 20.0) -> dict:
    """The oracle's FP64 SP2 (NumPy/BLAS) on the same 4094-orbital H, timed on
    the host cores for a bounded number of projections."""
    import numpy as np
    from workloads import ModelParams, config2_system
    from oracle import tb, density
    P = ModelParams()
    s = config2_system()
    H = tb.build_H(tb.build_h(s.R, s.types, s.box, P), tb.build_gamma(s.R, s.box, P), s.types,
                   np.zeros(s.natoms))
    n = H.shape[0]
    nocc = s.n_occ(P)
    density.sp2(H, nocc, max_iter=1)  # warm-up (BLAS threads, page-in)
    k = 1
    while True:
        t0 = time.perf_counter()
        r = density.sp2(H, nocc, max_iter=k, tol=0.0)
        dt = time.perf_counter() - t0
        if dt * 2 > max_seconds or k >= 16:
            break
        k *= 2
    flops = 2.0 * n ** 3 * r.iters
    return {"value": flops / dt / 1e12, "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{r.iters} FP64 SP2 projections (NumPy matmul) of the n={n} config-2 H, {dt:.1f} s"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np
    from workloads import ModelParams, config2_system
    from oracle import tb, density
    P = ModelParams()
    s = config2_system()
    H = tb.build_H(tb.build_h(s.R, s.types, s.box, P), tb.build_gamma(s.R, s.box, P), s.types,
                   np.zeros(s.natoms))
    n = H.shape[0]
    nocc = s.n_occ(P)
    per_step = 2  # projections per reference step (bounded sample of the SP2 D construction)

    def step():
        density.sp2(H, nocc, max_iter=per_step, tol=0.0)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    flops = 2.0 * n ** 3 * per_step * args.steps
    val = flops / dt / 1e12
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{per_step} FP64 SP2 projections (NumPy) of the n={n} H per step"},
            "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm

def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1203_6836_gb300 import build, tbmd
    from paper_1203_6836_gb300.device import DeviceSystem, MDState, sp2_opts, xl_params, report_to_dict
    from workloads import ModelParams, XLParams, config2_system, thermal_velocities

    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    ctx = tbmd.Context()
    P = ModelParams()
    TP = tbmd.tb_params.from_model(P)
    XL = XLParams()
    from workloads import water_system
    s = config2_system(seed=rank) if args.natoms == 2048 else water_system(args.natoms, density=1.0, seed=rank)
    M = s.masses(P)
    v0 = thermal_velocities(M, 300.0, seed=100 + rank)
    ds = DeviceSystem(s.R, s.types, s.box)
    n = ds.norb
    opts = sp2_opts(args.precision, max_iter=100, tol=1e-10, refine=args.refine)
    st = MDState(ds, v0, M, s.n_occ(P), XL.K, opts)
    xp = xl_params(XL.dt, XL.kappa, XL.alpha, XL.c)
    stream = torch.cuda.current_stream()
    scf_it = tbmd.xlbomd_init(ctx, TP, st.st, xp, opts, 1e-6, args.scf_iters)

    for _ in range(args.warmup):
        tbmd.xlbomd_step(ctx, TP, st.st, xp, opts)
    rep_sz = st.report.numel()
    reports = torch.empty(args.steps, rep_sz, dtype=torch.uint8, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    sampler = ClockSampler(local)
    tbmd.tb_ctx_set_profiling(ctx, True)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    sampler.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    ev[0].record(stream)
    for k in range(args.steps):
        tbmd.xlbomd_step(ctx, TP, st.st, xp, opts)
        reports[k].copy_(st.report, non_blocking=True)
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    main_ms = tbmd.tb_ctx_sp2_launch_times(ctx, 0)
    ref_ms = tbmd.tb_ctx_sp2_launch_times(ctx, 1)
    tbmd.tb_ctx_set_profiling(ctx, False)
    step_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[args.steps])
    reps = [report_to_dict(reports[k]) for k in range(args.steps)]
    proj = sum(r["iters"] + r["refine_iters"] for r in reps)
    flops = 2.0 * float(n) ** 3 * proj
    if world > 1:
        t = torch.tensor([total_ms, flops], dtype=torch.float64, device="cuda")
        tmax = t[0:1].clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        dist.all_reduce(t[1:2], op=dist.ReduceOp.SUM)
        total_ms, flops = float(tmax.item()), float(t[1].item())
    value = flops / (total_ms * 1e-3) / 1e12
    last = reps[-1]

    # ---- dominant kernel: tensor-core projection of the last timed step
    peaks = measured_peaks()
    tf = args.precision.startswith("tf32")
    ratio = 0.5 if tf else 1.0  # nominal tf32 : bf16 dense tensor rate
    peak = peaks["bf16_tflops_sustained"] * ratio
    work = main_ms[:last["iters"]]
    avg_ms = sum(work) / len(work) if work else float("nan")
    achieved = 2.0 * float(n) ** 3 / (avg_ms * 1e-3) / 1e12
    mmas = 3 if args.precision.endswith("x3") else 1
    ref_work = ref_ms[:last["refine_iters"]]
    ref_avg = sum(ref_work) / len(ref_work) if ref_work else float("nan")

    result = {}
    if rank == 0:
        # ---- end to end through the C ABI with host buffers
        pin = dict(dtype=torch.float64, pin_memory=True)
        hR = torch.empty(st.R.shape, **pin).copy_(st.R)
        hv = torch.empty(st.v.shape, **pin).copy_(st.v)
        hF = torch.empty(st.F.shape, **pin).copy_(st.F)
        hn = torch.empty(st.n_hist.shape, **pin).copy_(st.n_hist)
        hq = torch.empty(st.q.shape, **pin).copy_(st.q)
        hE = torch.empty(st.energies.shape, **pin)
        e2e_steps = max(2, min(args.steps, 5))
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e2e_proj = 0
        for _ in range(e2e_steps):
            for d, h in ((st.R, hR), (st.v, hv), (st.F, hF), (st.n_hist, hn), (st.q, hq)):
                d.copy_(h, non_blocking=True)
            tbmd.xlbomd_step(ctx, TP, st.st, xp, opts)
            hE.copy_(st.energies, non_blocking=True)
            for d, h in ((st.R, hR), (st.v, hv), (st.F, hF), (st.n_hist, hn), (st.q, hq)):
                h.copy_(d, non_blocking=True)
            stream.synchronize()
            e2e_proj += st.report.cpu().numpy().view(np.int32)[1] + st.report.cpu().numpy().view(np.int32)[2]
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = e0.elapsed_time(e1)
        h2d = sum(t.numel() * 8 for t in (hR, hv, hF, hn, hq))
        d2h = h2d + hE.numel() * 8
        e2e_val = 2.0 * float(n) ** 3 * e2e_proj / (e2e_ms * 1e-3) / 1e12

        # ---- the plain FP64 GPU path: one step
        fp64 = None
        if not args.no_fp64:
            o64 = sp2_opts("fp64", max_iter=100, tol=1e-10, refine=0)
            st64 = MDState(ds, v0, M, s.n_occ(P), XL.K, o64)
            for name in ("R", "v", "F", "n_hist", "q"):
                getattr(st64, name).copy_(getattr(st, name))
            st64.st.step = st.st.step
            torch.cuda.synchronize()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            tbmd.xlbomd_step(ctx, TP, st64.st, xp, o64)
            a1.record(stream)
            torch.cuda.synchronize()
            r64 = report_to_dict(st64.report)
            ms64 = a0.elapsed_time(a1)
            fp64 = {"steps_per_s": 1e3 / ms64, "ms_per_step": ms64, "sp2_projections": r64["iters"],
                    "tflops": 2.0 * float(n) ** 3 * r64["iters"] / (ms64 * 1e-3) / 1e12}
            del st64

        # ---- accuracy of D, q, energy vs the oracle (same inputs: R0, n = 0)
        check = None
        if not args.no_check:
            from oracle import tb, density, observables
            Ho = tb.build_H(tb.build_h(s.R, s.types, s.box, P), tb.build_gamma(s.R, s.box, P), s.types,
                            np.zeros(s.natoms))
            ref = density.density_T0(Ho, int(s.n_occ(P)))
            f64 = dict(dtype=torch.float64, device="cuda")
            H = torch.empty(n, n, **f64)
            G = torch.empty(s.natoms, s.natoms, **f64)
            ds0 = DeviceSystem(s.R, s.types, s.box)
            tbmd.tb_build_H(ctx, TP, ds0.sys, ds0.R, None, H, G)
            D = torch.empty_like(H)
            from paper_1203_6836_gb300.device import DensitySolver
            sol = DensitySolver(ctx, n, opts)
            sol(H, s.n_occ(P), D)
            q = torch.empty(s.natoms, **f64)
            tbmd.mulliken(ctx, TP, ds0.sys, D, q)
            torch.cuda.synchronize()
            Dg = D.cpu().numpy()
            qo = observables.mulliken(ref.D, s.types, P)
            h0 = tb.build_h(s.R, s.types, s.box, P)
            check = {"D_fro_per_sqrt_n": float(np.linalg.norm(Dg - ref.D) / np.sqrt(n)),
                     "q_max_abs": float(np.abs(q.cpu().numpy() - qo).max()),
                     "band_energy_abs_eV": float(abs(2 * np.sum(h0 * Dg) - 2 * np.sum(h0 * ref.D))),
                     "gap_eV": float(ref.gap), "inputs": "R of config 2, n = 0"}

        cpu = None
        if not args.no_cpu and world == 1:
            cpu = cpu_oracle_sample()

        result = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": f"{args.precision}+f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": args.precision, "refine_iters": args.refine,
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                       "l2": "no flush: per-step working set (H, D 134 MB each, X buffers) exceeds the 129 MB L2",
                       "scf_init_iters": scf_it},
            "steps_per_s": 1e3 * args.steps / total_ms * world,
            "latency_ms": {"p50": statistics.median(step_ms),
                           "p99": sorted(step_ms)[min(len(step_ms) - 1, int(0.99 * len(step_ms)))]},
            "sp2": {"projections_per_step": proj / args.steps, "last_step": {k: last[k] for k in (
                "status", "iters", "refine_iters", "trace", "idem_trace")}},
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": f"k_sp2_step_tc<{args.precision}>",
                         "peak_source": f"{peaks['source']} bf16_tflops_sustained x {ratio} ({'tf32' if tf else 'bf16'})",
                         "mma_per_product": mmas, "mma_frac": achieved * mmas / peak,
                         "avg_launch_ms": avg_ms},
            "refine_kernel": {"kind": "emulated FP64 (28 exact bf16 slice products)" if opts.refine_mode == 0
                              else "FP64 FMA",
                              "avg_launch_ms": ref_avg,
                              "tflops": 2.0 * float(n) ** 3 / (ref_avg * 1e-3) / 1e12 if ref_work else None},
            "fp64_path": fp64,
            "accuracy_vs_oracle": check,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_val, "unit": "TFLOP/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "steps": e2e_steps},
            "gpu_launches": None,
            "clocks": clocks,
        }
        # kernel launches per step: main phase (max_iter + 1 + split) + FP64 refinement
        # (refine + 2) + bounds/init/finalize + H build (2) + Mulliken + forces + MD (3)
        per_step = (100 + 2) + (2 * args.refine + 2) + 3 + 2 + 1 + 1 + 3
        result["gpu_launches"] = per_step * args.steps
        print(json.dumps(result), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
