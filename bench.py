#!/usr/bin/env python
"""Benchmark of Fourier-accelerated steepest-descent Landau gauge fixing.

Workload (one step = one complete gauge fixing): an SU(3) 32^4 lattice in FP64
with 12-real link storage, alpha = 0.08, run until theta < 1e-15, on synthetic
rough-gauge configurations of roughness eps in {0.15, 0.3, 0.5} (stand-ins for
the paper's three Wilson-action couplings), cycled over the steps.  The metric
is iterations per second over the timed steps (all ranks together) and the
time-to-theta of each configuration.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

The reference arm times the FP64 CPU oracle on the host cores on the same
workload (one oracle iteration per step).  Under torchrun each rank fixes its
own configurations (independent replicas, weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "SD iters/s & time-to-theta<1e-15, 32^4 SU(3), FP64 vs mixed; % of HBM peak"
# GB300 dense FP64 from unit counts and clocks: 152 SMs x 2 FP64 FMAs per cycle per SM
# (1.25 TFLOP/s nominal at the 2070 MHz maximum SM clock) x 2 flops x 2.07 GHz
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07
EPS = (0.15, 0.3, 0.5)
SEEDS = (3201, 3202, 3203)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--dims", default="32,32,32,32")
    ap.add_argument("--alpha", type=float, default=0.08)
    ap.add_argument("--tol", type=float, default=1e-15)
    ap.add_argument("--max-iter", type=int, default=20000)
    ap.add_argument("--cpu-iters", type=int, default=20, help="oracle iterations of the CPU-baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-diff", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-links18", action="store_true")
    ap.add_argument("--no-links8", action="store_true")
    ap.add_argument("--no-wilson", action="store_true")
    ap.add_argument("--no-cpu-fix", action="store_true", help="skip the oracle's full-size fix in cpu_baseline")
    ap.add_argument("--no-48", action="store_true", help="skip the 48^4 FP64-vs-mixed leg")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the 58-lattice ensemble leg")
    ap.add_argument("--no-slabs", action="store_true", help="skip the one-GPU measurement of the t-slab path")
    ap.add_argument("--slab-ranks", type=int, default=2,
                    help="--workload slabs in one process: t-slabs emulated on one GPU")
    ap.add_argument("--slab-iters", type=int, default=10, help="iterations per step of --workload slabs")
    ap.add_argument("--workload", default="single",
                    choices=["single", "ensemble", "wilson", "kernels", "probe", "slabs"],
                    help="single: the 32^4 lattice line; ensemble: the batched mixed-precision ensemble; "
                         "wilson: Wilson-action configuration generation (heat bath + overrelaxation); "
                         "kernels: the iteration kernels launched one by one (FP64 and FP32), per-kernel times; "
                         "probe: the FP64 and FP32 FMA rates of the GPU (the FP64 kernels' arithmetic ceiling)")
    ap.add_argument("--no-autotune", action="store_true", help="--workload kernels: default launch shapes")
    ap.add_argument("--zt-form", type=int, default=-1, choices=[-1, 0, 1],
                    help="--workload kernels: z,t kernel form of both precisions (0 pencil-tiled, 1 TMA-staged "
                         "pencils, 4-column pencils; -1 the default or autotuned shape)")
    ap.add_argument("--beta", type=float, default=6.0, help="coupling of --workload wilson")
    ap.add_argument("--switch-tol", type=float, default=1e-6,
                    help="theta that ends the FP32 phase of --workload ensemble (1e-6 as specified; 1e-13 deep)")
    return ap.parse_args()


def bench_config(dims, args, ws):
    """The workload description printed by both arms (same keys, same values)."""
    V = int(np.prod(dims))
    return {"workload": workload(dims), "dims": list(dims), "alpha": args.alpha, "tol": args.tol, "eps": list(EPS),
            "l2": "inputs larger than L2 (%.0f MB of links per configuration)" % (4 * V * 12 * 8 / 1e6),
            "parallelism": "replicas" if ws > 1 else "single"}


def workload(dims):
    return "SU(3) %s FP64 Fourier-accelerated steepest descent, 12-real links, alpha=0.08, theta<1e-15, eps %s" % (
        "x".join(str(d) for d in dims), "/".join(str(e) for e in EPS))


def dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_over_ranks(pg, seconds: float, units: float, device="cuda"):
    """Whole-job figures of independent replicas: the slowest rank's time and the
    units (iterations) summed over ranks."""
    if pg is None:
        return seconds, units
    import torch

    t = torch.tensor([seconds], device=device, dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    n = torch.tensor([units], device=device, dtype=torch.float64)
    pg.all_reduce(n, op=pg.ReduceOp.SUM)
    return float(t.item()), float(n.item())


def configs(dims, rank):
    from paper_1301_3460_gb300 import inputs

    return [inputs.rough_gauge_field(dims, e, s + 1000 * rank) for e, s in zip(EPS, SEEDS)]


# ---------------------------------------------------------------- clocks

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
            return
        # the sampler's start-up (NVML initialisation) must not fall inside the timed region
        t0 = time.time()
        while time.time() - t0 < 15 and self.p.poll() is None:
            if os.path.getsize(self.f.name) > 0:
                break
            time.sleep(0.05)

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.3)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if "Active" in v and "Not" not in v:
                    reasons.add(n)
        if not sm:
            return None
        load = [v for v in sm if mx and v > 0.5 * mx] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- traffic record

KERNEL_SOURCES = ("lgf_common.cuh", "lgf_dft.cuh", "lgf_kernels.cuh")


def csrc_hash():
    """Hash of the sources that define the iteration kernels."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1301_3460_gb300", "csrc")
    for fn in KERNEL_SOURCES:
        with open(os.path.join(d, fn), "rb") as f:
            h.update(fn.encode() + f.read())
    return h.hexdigest()[:16]


def traffic_record(kernel, dims, precision):
    """DRAM bytes per launch of a kernel from the committed ncu summary, if it
    was taken on the current kernel sources; else None."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        rec = json.load(open(p))
    except (OSError, ValueError):
        return None
    if rec.get("csrc_hash") != csrc_hash():
        return None
    key = "%s/%s/fp%d" % (kernel, "x".join(map(str, dims)), precision)
    v = rec.get("per_launch_bytes", {}).get(key)
    return float(v) if v is not None else None


# ---------------------------------------------------------------- arms

def run_reference(args, dims):
    ws, rank, _ = dist()
    if rank != 0:
        return 0
    from oracle import oracle as orc

    U = configs(dims, 0)
    t_all = []
    n_it = 0
    for k in range(args.warmup + args.steps):
        Ui = U[k % len(U)]
        t0 = time.perf_counter()
        r = orc.fix(dims, Ui, alpha=args.alpha, tol=0.0, max_iter=1)
        dt = time.perf_counter() - t0
        U[k % len(U)] = r["U"]
        if k >= args.warmup:
            t_all.append(dt)
            n_it += r["iters"]
    T = sum(t_all)
    value = n_it / T
    cores = orc.threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * T / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(dims, args, 1),
        "cpu_baseline": {"value": value, "unit": "iters/s", "cores": cores, "kind": "oracle",
                         "sample": "one oracle iteration per step on the %s configurations (eps %s)" % (
                             "x".join(map(str, dims)), "/".join(map(str, EPS)))},
        "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, dims):
    import torch

    from paper_1301_3460_gb300 import lgf, roofline

    ws, rank, local = dist()
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU (the library has no CPU path)")
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as tdist

        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = tdist
    lgf.load()
    host = configs(dims, rank)
    V = host[0].shape[1]
    stream = torch.cuda.current_stream()
    dev = [torch.from_numpy(U).to("cuda") for U in host]
    lat = lgf.Lattice(dims, stream=stream)
    lat.set_links(dev[1])
    lat.autotune()  # launch shapes of the FFT kernels, chosen by timing (set-up, not timed)

    def step(i):
        lat.set_links(dev[i % len(dev)])
        return lat.fix(args.alpha, args.tol, args.max_iter)

    # the clock sampler starts before the warm-up, so its start-up overlaps untimed work
    clocks = Clocks(local)
    clocks.start()
    for k in range(args.warmup):
        step(k)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    info = []
    ev[0].record(stream)
    for k in range(args.steps):
        info.append(step(k))
        ev[k + 1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if pg:
        pg.barrier()
    per_step = [ev[k].elapsed_time(ev[k + 1]) / 1000.0 for k in range(args.steps)]
    T = sum(per_step)
    iters = sum(r["iters"] for r in info)
    T, iters = reduce_over_ranks(pg, T, iters)
    value = iters / T
    # kernels of the timed region, per step: lgf_set_links (pack and check, G = 1),
    # then the graph of lgf_fix (packed parts and Delta of the input, then per loop
    # pass the z,t kernel, the inverse x,y + g kernel, the update, Delta and the
    # loop control)
    launches = sum(2 + 2 + 5 * max(r["iters"], 1) for r in info)
    ttt = {}
    for k, r in enumerate(info):
        ttt.setdefault(str(EPS[k % len(EPS)]), dict(iters=r["iters"], ms=1000 * per_step[k], F=r["F"],
                                                     theta=r["theta"], converged=r["converged"]))

    # the same workload in mixed precision (FP32 until theta < 1e-6, then FP64)
    mixed = None
    if not args.no_mixed:
        latm = lgf.Lattice(dims, mixed=True, stream=stream)
        latm.set_links(dev[1])
        latm.autotune()

        def mstep(i):
            latm.set_links(dev[i % len(dev)])
            return latm.fix(args.alpha, args.tol, args.max_iter)

        for k in range(args.warmup):
            mstep(k)
        torch.cuda.synchronize()
        evm = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        minfo = []
        evm[0].record(stream)
        for k in range(args.steps):
            minfo.append(mstep(k))
            evm[k + 1].record(stream)
        torch.cuda.synchronize()
        mper = [evm[k].elapsed_time(evm[k + 1]) / 1000.0 for k in range(args.steps)]
        Tm = sum(mper)
        mit = sum(r["iters"] for r in minfo)
        Tm, mit = reduce_over_ranks(pg, Tm, mit)
        # set_links; FP32 start (copy, parts, Delta); FP32 passes of 7 kernels (with the two
        # refresh kernels); the switch (3) and the FP64 start (2); FP64 passes of 5
        mixed_launches = sum(2 + 3 + 7 * max(r["iters_fp32"], 1) + 5 + 5 * max(r["iters_fp64"], 1) for r in minfo)
        mttt = {}
        for k, r in enumerate(minfo):
            e = str(EPS[k % len(EPS)])
            f64 = ttt.get(e, {}).get("F")
            mttt.setdefault(e, dict(iters_fp32=r["iters_fp32"], iters_fp64=r["iters_fp64"], ms=1000 * mper[k],
                                    F=r["F"], theta=r["theta"], converged=r["converged"],
                                    F_rel_diff_vs_fp64=(abs(r["F"] / f64 - 1) if f64 else None)))
        mixed = {"value": mit / Tm, "unit": "iters/s", "ms_per_step": 1000 * Tm / args.steps,
                 "gpu_launches": mixed_launches,
                 "speedup_time_to_theta_vs_fp64": T / Tm, "time_to_theta": mttt}
        # the FP32 phase run down to theta < 1e-13, where FP32 iterations stop tracking FP64 ones
        latm.set_switch_tol(1e-13)
        deep = {}
        for e, Ud in zip((str(v) for v in EPS), dev):
            latm.set_links(Ud)
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            r = latm.fix(args.alpha, args.tol, args.max_iter)
            f1.record(stream)
            torch.cuda.synchronize()
            f64 = ttt.get(e, {}).get("F")
            deep[e] = dict(iters_fp32=r["iters_fp32"], iters_fp64=r["iters_fp64"], ms=f0.elapsed_time(f1),
                           converged=r["converged"], F_rel_diff_vs_fp64=(abs(r["F"] / f64 - 1) if f64 else None))
        mixed["time_to_theta_switch_1e-13"] = deep
        latm.set_switch_tol(1e-6)
        latm.set_links(dev[1])
        # per-kernel times of the two-kernel FP32 form; the default (persistent) form runs
        # its g builder and update as one launch, timed beside them
        latm.set_fp32_update(2)
        msp = latm.time_kernels(args.alpha, n_iter=8, precision=32)
        mixed["kernels_fp32_persistent"] = {"delta_xyfft": msp["delta_xyfft"], "zt_fft_accel": msp["zt_fft_accel"],
                                            "g_and_update": msp["xyifft_g"] + msp["update"]}
        mixed["fp32_persistent_iteration_ms"] = sum(msp.values())
        latm.set_fp32_update(0)
        latm.set_links(dev[1])
        msm = latm.time_kernels(args.alpha, n_iter=8, precision=32)
        per32 = roofline.per_site(dims, 32, fused32=False)
        mixed["kernels_fp32"] = {k: {"ms": msm[k], "gbs": per32[k]["bytes"] * V / msm[k] / 1e6,
                                     "gflops": per32[k]["flops"] * V / msm[k] / 1e6} for k in msm}
        mixed["fp32_iteration_ms"] = sum(msm.values())
        # the FP32 phase with the update fused with Delta (selectable form), same kernels timed
        latm.set_fp32_update(True)
        msf = latm.time_kernels(args.alpha, n_iter=8, precision=32)
        perf = roofline.per_site(dims, 32, fused32=True)
        mixed["kernels_fp32_fused"] = {k: {"ms": msf[k], "gbs": perf[k]["bytes"] * V / msf[k] / 1e6}
                                       for k in msf}
        mixed["fp32_fused_iteration_ms"] = sum(msf.values())
        latm.set_fp32_update(2)
        # the accelerator's transforms in FP32 inside the FP64 iterations (Delta, theta,
        # F, Gram-Schmidt and update in FP64): whole fixes in FP64 iterations (no FP32
        # phase) and the mixed mode at both switch points, same steps as above
        latm.set_accel_precision(32)
        accel = {}
        for name, sw in (("fp64_iterations", 1e300), ("mixed_switch_1e-06", 1e-6), ("mixed_switch_1e-13", 1e-13)):
            latm.set_switch_tol(sw)
            for k in range(max(1, args.warmup)):
                mstep(k)
            torch.cuda.synchronize()
            eva = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
            ainfo = []
            eva[0].record(stream)
            for k in range(args.steps):
                ainfo.append(mstep(k))
                eva[k + 1].record(stream)
            torch.cuda.synchronize()
            aper = [eva[k].elapsed_time(eva[k + 1]) / 1000.0 for k in range(args.steps)]
            Ta, ait = reduce_over_ranks(pg, sum(aper), sum(r["iters"] for r in ainfo))
            attt = {}
            for k, r in enumerate(ainfo):
                e = str(EPS[k % len(EPS)])
                f64 = ttt.get(e, {}).get("F")
                attt.setdefault(e, dict(iters_fp32=r["iters_fp32"], iters_fp64=r["iters_fp64"], ms=1000 * aper[k],
                                        converged=r["converged"], theta=r["theta"],
                                        F_rel_diff_vs_fp64=(abs(r["F"] / f64 - 1) if f64 else None)))
            accel[name] = {"value": ait / Ta, "unit": "iters/s", "ms_per_step": 1000 * Ta / args.steps,
                           "speedup_time_to_theta_vs_fp64": T / Ta, "time_to_theta": attt}
        latm.set_switch_tol(1e-6)
        latm.set_links(dev[1])
        msa = latm.time_kernels(args.alpha, n_iter=8, precision=64)
        accel["kernels_fp64_iteration"] = {k: {"ms": msa[k]} for k in msa}
        accel["fp64_iteration_ms"] = sum(msa.values())
        mixed["accel_fp32"] = accel
        latm.set_accel_precision(64)
        latm.close()

    # link parametrisation: the same FP64 workload with row 2 kept in memory (18 reals)
    links18 = None
    if not args.no_links18:
        l18 = lgf.Lattice(dims, links18=True, stream=stream)
        l18.set_links(dev[1])
        l18.autotune()
        for k in range(1):
            l18.set_links(dev[k % len(dev)])
            l18.fix(args.alpha, args.tol, args.max_iter)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n18 = 0
        e0.record(stream)
        for k in range(args.steps):
            l18.set_links(dev[k % len(dev)])
            n18 += l18.fix(args.alpha, args.tol, args.max_iter)["iters"]
        e1.record(stream)
        torch.cuda.synchronize()
        T18 = e0.elapsed_time(e1) / 1000.0
        l18.set_links(dev[1])
        ms18 = l18.time_kernels(args.alpha, n_iter=8, precision=64)
        l18.close()
        links18 = {"value": n18 / T18, "unit": "iters/s", "ms_per_step": 1000 * T18 / args.steps,
                   "update_ms": ms18["update"], "kernels_ms": ms18}
        # the 18-real form with the accelerator's transforms in FP32 inside the FP64
        # iterations (a mixed context whose FP32 phase is empty: switch above theta)
        if not args.no_mixed:
            la = lgf.Lattice(dims, mixed=True, links18=True, stream=stream)
            la.set_accel_precision(32)
            la.set_switch_tol(1e300)
            la.set_links(dev[1])
            la.autotune()
            la.set_links(dev[0])
            la.fix(args.alpha, args.tol, args.max_iter)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            na = 0
            e0.record(stream)
            for k in range(args.steps):
                la.set_links(dev[k % len(dev)])
                na += la.fix(args.alpha, args.tol, args.max_iter)["iters"]
            e1.record(stream)
            torch.cuda.synchronize()
            Ta = e0.elapsed_time(e1) / 1000.0
            la.set_links(dev[1])
            msa = la.time_kernels(args.alpha, n_iter=8, precision=64)
            la.close()
            links18["accel_fp32"] = {"value": na / Ta, "unit": "iters/s", "ms_per_step": 1000 * Ta / args.steps,
                                     "iteration_ms": sum(msa.values()), "kernels_ms": msa}

    # the 8-real form: a third of the 12-real link bytes, more FP64 work per load and store
    links8 = None
    if not args.no_links18 and not args.no_links8:
        l8 = lgf.Lattice(dims, links8=True, stream=stream)
        n8, T8, ok8 = 0, 0.0, True
        try:
            for Ud in dev:
                l8.set_links(Ud)
        except lgf.LgfError:
            ok8 = False  # a link too close to the form's singular set |u00| = 1
        if ok8:
            l8.autotune()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for k in range(args.steps):
                l8.set_links(dev[k % len(dev)])
                n8 += l8.fix(args.alpha, args.tol, args.max_iter)["iters"]
            e1.record(stream)
            torch.cuda.synchronize()
            T8 = e0.elapsed_time(e1) / 1000.0
            l8.set_links(dev[1])
            ms8 = l8.time_kernels(args.alpha, n_iter=8, precision=64)
            links8 = {"value": n8 / T8, "unit": "iters/s", "ms_per_step": 1000 * T8 / args.steps,
                      "update_ms": ms8["update"], "kernels_ms": ms8}
        else:
            links8 = {"value": None, "note": "configuration refused: a link the 8-real form cannot hold"}
        l8.close()

    # critical slowing down: plain steepest descent against the accelerated method at 16^4
    plain = None
    if not args.no_plain:
        Lp = (16, 16, 16, 16)
        Up = torch.from_numpy(configs(Lp, rank)[1]).to("cuda")
        plain = {"dims": list(Lp), "eps": EPS[1]}
        for name, acc, alpha in (("accelerated", True, args.alpha), ("plain", False, 0.1)):
            lp = lgf.Lattice(Lp, accelerate=acc, stream=stream)
            lp.set_links(Up)
            lp.fix(alpha, args.tol, 100000)
            lp.set_links(Up)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = lp.fix(alpha, args.tol, 100000)
            e1.record(stream)
            torch.cuda.synchronize()
            plain[name] = {"alpha": alpha, "iters": r["iters"], "ms": e0.elapsed_time(e1), "converged": r["converged"]}
            lp.close()

    # differentiation: forward + backward of a K-step unroll with checkpoints and D(p_min)
    diff = None
    if not args.no_diff:
        from paper_1301_3460_gb300 import autograd as lad

        Kd, every = 10, 5
        lat_d = lgf.Lattice(dims, track_gauge=False, stream=stream)
        for rep in range(2):  # the first pass warms up
            U0 = dev[1].clone().requires_grad_(True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            D, _ = lad.gluon_after_fixing(U0, dims, K=Kd, every=every, lat=lat_d)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            D.backward()
            torch.cuda.synchronize()
            t2 = time.perf_counter()
        lat_d.close()
        diff = {"steps": Kd, "checkpoint_every": every, "fwd_ms": 1000 * (t1 - t0), "bwd_ms": 1000 * (t2 - t1),
                "fwd_bwd_steps_per_s": Kd / (t2 - t0), "D_pmin": float(D.item())}

    # Wilson-action configuration generation at the same extents (beta = 6.0, cold start)
    wilson = None
    if not args.no_wilson:
        lw = lgf.Lattice(dims, track_gauge=False, stream=stream)
        lw.set_unit_links()
        lw.wilson_sweeps(6.0, 7, first_sweep=0, n_heatbath=3, n_overrelax=1)
        wilson = {"beta": 6.0, "start": "cold + 3 x (heat bath + overrelaxation)", "links_per_sweep": 4 * V}
        for lab, nhb, nor in (("heatbath", 1, 0), ("overrelax", 0, 1)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for k in range(args.steps):
                lw.wilson_sweeps(6.0, 7, first_sweep=3 + k, n_heatbath=nhb, n_overrelax=nor)
            e1.record(stream)
            torch.cuda.synchronize()
            msw = e0.elapsed_time(e1) / args.steps
            gf = roofline.WILSON_FLOPS_PER_LINK * 4 * V / msw / 1e6
            wilson[lab] = {"ms_per_sweep": msw, "gflops": gf, "frac_fp64_peak": gf / FP64_PEAK_GFLOPS}
        # the FP32 generator (its own chain; links re-orthonormalised in FP64)
        lw.set_generator_precision(32)
        for lab, nhb, nor in (("heatbath_fp32", 1, 0), ("overrelax_fp32", 0, 1)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for k in range(args.steps):
                lw.wilson_sweeps(6.0, 7, first_sweep=100 + k, n_heatbath=nhb, n_overrelax=nor)
            e1.record(stream)
            torch.cuda.synchronize()
            wilson[lab] = {"ms_per_sweep": e0.elapsed_time(e1) / args.steps}
        lw.set_generator_precision(64)
        wilson["plaquette"] = lw.plaquette()
        # generate -> fix on the device: Wilson-action configurations at three couplings
        # (cold start, 40 x (heat bath + 4 overrelaxation)), then FP64 gauge fixing
        # and the same configurations in mixed precision (FP32 until theta < 1e-6)
        wilson["fix"] = {}
        lm = None if args.no_mixed else lgf.Lattice(dims, mixed=True, stream=stream)
        for beta in (5.7, 6.0, 6.2):
            lw.set_unit_links()
            e0, e1, e2, e3 = (torch.cuda.Event(enable_timing=True) for _ in range(4))
            e0.record(stream)
            lw.wilson_sweeps(beta, 11, first_sweep=0, n_heatbath=40, n_overrelax=4)
            e1.record(stream)
            U_gen = lw.get_links(device="cuda") if lm is not None else None
            e2.record(stream)
            r = lw.fix(args.alpha, args.tol, 20000)
            e3.record(stream)
            torch.cuda.synchronize()
            w = {"generate_ms": e0.elapsed_time(e1), "plaquette": lw.plaquette(), "iters": r["iters"],
                 "fix_ms": e2.elapsed_time(e3), "F": r["F"], "theta": r["theta"], "converged": r["converged"]}
            if lm is not None:
                lm.set_links(U_gen)
                f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                f0.record(stream)
                rm = lm.fix(args.alpha, args.tol, 20000)
                f1.record(stream)
                torch.cuda.synchronize()
                w["mixed"] = {"iters_fp32": rm["iters_fp32"], "iters_fp64": rm["iters_fp64"],
                              "fix_ms": f0.elapsed_time(f1), "F": rm["F"], "converged": rm["converged"],
                              "F_rel_diff_vs_fp64": abs(rm["F"] / r["F"] - 1) if r["F"] else None}
                # FP32 phase down to theta < 1e-13
                lm.set_switch_tol(1e-13)
                lm.set_links(U_gen)
                f0.record(stream)
                rd = lm.fix(args.alpha, args.tol, 20000)
                f1.record(stream)
                torch.cuda.synchronize()
                lm.set_switch_tol(1e-6)
                w["mixed_switch_1e-13"] = {"iters_fp32": rd["iters_fp32"], "iters_fp64": rd["iters_fp64"],
                                        "fix_ms": f0.elapsed_time(f1), "F": rd["F"], "converged": rd["converged"],
                                        "F_rel_diff_vs_fp64": abs(rd["F"] / r["F"] - 1) if r["F"] else None}
            wilson["fix"][str(beta)] = w
        if lm is not None:
            lm.close()
        lw.close()

    # end to end through the C ABI from pinned host memory, copies included: every
    # step copies its input in, fixes it and reads the fixed links back
    # (lgf_get_links to pinned host memory).  The steps alternate between two
    # contexts on two streams, each driven by its own host thread (the library's
    # calls release the GIL); the fixes run one at a time in step order, and a
    # step's copies in (the copy engine into a device buffer, then lgf_set_links)
    # and out overlap the fixes of its neighbours.  The same steps one after
    # another on one context, lgf_set_links reading the pinned input in place,
    # give `serial_value`.
    e2e = None
    if not args.no_e2e:
        import threading

        pin_in = [torch.from_numpy(U).pin_memory() for U in host]
        pin_out = [torch.empty((4, V, 3, 3), dtype=torch.complex128).pin_memory() for _ in range(2)]
        nbytes = pin_in[0].numel() * 16
        cdev = torch.cuda.current_device()

        def copy_out(c, out):
            lgf._check(c._lib.lgf_get_links(c._h, lgf.ctypes.c_void_p(out.data_ptr()), 0), "lgf_get_links")

        torch.cuda.synchronize()
        t0 = time.perf_counter()
        n_ser = 0
        for k in range(args.steps):
            lat.set_links(pin_in[k % len(pin_in)])
            n_ser += lat.fix(args.alpha, args.tol, args.max_iter)["iters"]
            copy_out(lat, pin_out[0])
        torch.cuda.synchronize()
        Ts = time.perf_counter() - t0
        lat2 = lgf.Lattice(dims, stream=torch.cuda.Stream())
        lat2.set_links(dev[1])
        lat2.autotune()
        lat2.fix(args.alpha, args.tol, args.max_iter)  # its graph is built here, outside the timed region
        counts, errs = [0, 0], []
        turn = [0]
        cv = threading.Condition()
        # device landing buffers of the copies in: the copy engine moves the input
        # while the other context's fix runs, then lgf_set_links packs it on the GPU
        land = [torch.empty((4, V, 3, 3), dtype=torch.complex128, device="cuda") for _ in range(2)]

        def e2e_worker(i, c):
            try:
                torch.cuda.set_device(cdev)
                for k in range(i, args.steps, 2):
                    # during the previous step's fix: H2D copy on this context's stream, then the pack
                    with torch.cuda.stream(c._stream):
                        land[i].copy_(pin_in[k % len(pin_in)], non_blocking=True)
                    c.set_links(land[i])
                    with cv:
                        if not cv.wait_for(lambda: turn[0] == k or errs, timeout=600) or errs:
                            return
                    try:
                        counts[i] += c.fix(args.alpha, args.tol, args.max_iter)["iters"]
                    finally:
                        with cv:
                            turn[0] += 1
                            cv.notify_all()
                    copy_out(c, pin_out[i])  # during the next step's fix
            except BaseException as e:  # re-raised on the main thread
                with cv:
                    errs.append(e)
                    cv.notify_all()

        torch.cuda.synchronize()
        t0 = time.perf_counter()
        threads = [threading.Thread(target=e2e_worker, args=(i, c)) for i, c in enumerate((lat, lat2))]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        torch.cuda.synchronize()
        Te = time.perf_counter() - t0
        lat2.close()
        if errs:
            raise errs[0]
        if turn[0] != args.steps:
            raise RuntimeError("end-to-end leg: %d of %d steps ran" % (turn[0], args.steps))
        n_e2e = sum(counts)
        Te, n_e2e = reduce_over_ranks(pg, Te, n_e2e)
        Ts, n_ser = reduce_over_ranks(pg, Ts, n_ser)
        e2e = {"value": n_e2e / Te, "unit": "iters/s", "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
               "contexts": 2, "serial_value": n_ser / Ts}

    # the t-slab decomposition of one lattice (the multi-GPU path) on this GPU: its
    # own kernels and host-driven exchanges, ranks emulated as slabs of one process
    slabs = None
    if not args.no_slabs and pg is None:
        slabs = {"iterations": 10, "ranks": "emulated on one GPU (device copies in place of messages)",
                 "iters_per_s": {str(R): slab_rate(dims, host[1], R, 10) for R in (1, 2)}}

    # 48^4 (radix-3 FFT lengths): FP64 against mixed precision on one configuration
    big48 = None
    if not args.no_48 and not args.no_mixed:
        try:
            big48 = run_48(args, stream, rank)
        except Exception as e:  # the main line stands without this leg
            big48 = {"error": repr(e)}

    # the batched ensemble of uneven lattices in one graph launch, switch 1e-6 and 1e-13
    ens = None
    if not args.no_ensemble and not args.no_mixed:
        try:
            ens = ensemble_leg(args, stream, rank)
        except Exception as e:
            ens = {"error": repr(e)}

    # per-kernel durations (CUDA events around each launch) on the eps = 0.3 configuration
    lat.set_links(dev[1])
    ms = lat.time_kernels(args.alpha, n_iter=8, precision=64)
    per = roofline.per_site(dims, 64)
    kern = max(ms, key=lambda k: ms[k])
    sec = ms[kern] / 1000.0
    flops = per[kern]["flops"] * V
    byts = per[kern]["bytes"] * V
    traffic = traffic_record(kern, dims, 64)
    roof = {"bound": "alu", "kernel": kern, "achieved": flops / sec / 1e9, "peak": FP64_PEAK_GFLOPS,
            "unit": "GFLOP/s", "frac": flops / sec / 1e9 / FP64_PEAK_GFLOPS, "traffic": traffic,
            "peak_source": "GB300 FP64 from unit counts and clock: 152 SMs x 2 FP64 FMA/cycle x 2 flops x 2.07 GHz "
                           "(1.25 TFLOP/s nominal); probe_gflops is the FMA-only probe of this run "
                           "(bench.py --workload probe)",
            "hbm_achieved_gbs": byts / sec / 1e9}
    try:
        roof["probe_gflops"] = lgf.probe_fma(64, 10000)["gflops"]
    except lgf.LgfError:
        roof["probe_gflops"] = None
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        roof["hbm_frac_of_measured"] = roof["hbm_achieved_gbs"] / float(peaks["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        pass
    kernels = {k: {"ms": ms[k], "gflops": per[k]["flops"] * V / ms[k] / 1e6, "gbs": per[k]["bytes"] * V / ms[k] / 1e6}
               for k in ms}
    kernels["fp64_iteration_ms"] = sum(ms.values())
    # the metric's "% of HBM peak": algorithmic bytes of one whole FP64 iteration at the measured rate
    try:
        hbm = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
        it_bytes = roofline.per_iteration(dims, 64)["bytes"]
        hbm_iter = {"bytes_per_iteration": it_bytes, "achieved_gbs": it_bytes * value / 1e9, "peak_gbs": hbm,
                    "frac": it_bytes * value / 1e9 / hbm,
                    "note": "FP64 iteration bound by the FP64 pipe, not by HBM; see roofline"}
        if mixed is not None:
            for key in ("kernels_fp32", "kernels_fp32_fused"):
                for k, v in mixed.get(key, {}).items():
                    v["hbm_frac_of_measured"] = v["gbs"] / hbm
    except (OSError, ValueError, KeyError):
        hbm_iter = None

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        from oracle import oracle as orc

        from paper_1301_3460_gb300 import inputs

        t0 = time.perf_counter()
        r = orc.fix(dims, host[1], alpha=args.alpha, tol=0.0, max_iter=args.cpu_iters)
        dt = time.perf_counter() - t0
        cpu = {"value": r["iters"] / dt, "unit": "iters/s", "cores": orc.threads(), "kind": "oracle",
               "sample": "first %d iterations of the eps=0.3 %s configuration" % (r["iters"], "x".join(map(str, dims)))}
        # whole fixes where the oracle finishes in seconds, and the full-size one derived
        # from the GPU's iteration count
        for Ls, seed in (((8, 8, 8, 8), 1001), ((16, 16, 16, 16), 1601)):
            Us = inputs.rough_gauge_field(Ls, 0.3, seed)
            t0 = time.perf_counter()
            rs = orc.fix(Ls, Us, alpha=args.alpha, tol=args.tol, max_iter=args.max_iter)
            cpu["time_to_theta_%s_s" % "x".join(map(str, Ls))] = {"s": time.perf_counter() - t0, "iters": rs["iters"]}
        # the full-size fix to theta < tol, measured (about 15 s on 16 host cores at 32^4)
        if not args.no_cpu_fix:
            t0 = time.perf_counter()
            rs = orc.fix(dims, host[1], alpha=args.alpha, tol=args.tol, max_iter=args.max_iter)
            cpu["time_to_theta_%s_s" % "x".join(map(str, dims))] = {
                "s": time.perf_counter() - t0, "iters": rs["iters"], "converged": rs["converged"],
                "F_rel_diff_vs_gpu": abs(rs["F"] / ttt[str(EPS[1])]["F"] - 1) if str(EPS[1]) in ttt else None}

    lat.close()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * T / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(dims, args, ws),
            "time_to_theta": ttt, "mixed": mixed, "links18": links18, "links8": links8, "diff": diff,
            "plain_sd_16x4": plain,
            "wilson_generation": wilson, "fix_48x4": big48, "ensemble": ens,
            "slabs": slabs,
            "roofline": roof, "kernels": kernels, "hbm_iteration": hbm_iter, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


ENSEMBLE = ((32, (16, 16, 16, 16)), (16, (24, 24, 24, 24)), (8, (32, 32, 32, 64)), (2, (48, 48, 48, 96)))


def run_48(args, stream, rank):
    """One 48^4 configuration (eps = 0.3, drawn on the GPU) fixed in FP64 and in
    mixed precision (switch 1e-6 and 1e-13), each after an untimed warm-up fix:
    time-to-theta, iterations, F of the mixed runs relative to FP64 and the
    largest link difference (the residual global rotation, reading of Gribov
    copies)."""
    import torch

    from paper_1301_3460_gb300 import inputs, lgf

    L = (48, 48, 48, 48)
    U = inputs.rough_gauge_field_cuda(L, 0.3, 4801 + 1000 * rank)
    out = {"dims": list(L), "eps": 0.3}

    def timed(lat):
        lat.set_links(U)
        lat.fix(args.alpha, args.tol, args.max_iter)  # warm-up (autotuned shapes, graph)
        lat.set_links(U)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = lat.fix(args.alpha, args.tol, args.max_iter)
        e1.record(stream)
        torch.cuda.synchronize()
        return r, e0.elapsed_time(e1)

    with lgf.Lattice(L, stream=stream) as l64:
        l64.set_links(U)
        l64.autotune()
        r64, ms64 = timed(l64)
        U64 = l64.get_links(device="cuda")
    out["fp64"] = {"ms": ms64, "iters": r64["iters"], "F": r64["F"], "converged": r64["converged"],
                   "iters_per_s": 1000.0 * r64["iters"] / ms64}
    with lgf.Lattice(L, mixed=True, stream=stream) as lm:
        lm.set_links(U)
        lm.autotune()
        # mixed precision as specified, then with the accelerator's transforms in FP32
        # inside the FP64 iterations (switch 1e300: every iteration FP64)
        for accel, runs in ((64, ((1e-6, "mixed_switch_1e-06"), (1e-13, "mixed_switch_1e-13"))),
                            (32, ((1e300, "fp64_accel_fp32"), (1e-6, "mixed_accel_fp32_switch_1e-06"),
                                  (1e-13, "mixed_accel_fp32_switch_1e-13")))):
            lm.set_accel_precision(accel)
            for sw, name in runs:
                lm.set_switch_tol(sw)
                rm, msm = timed(lm)
                Um = lm.get_links(device="cuda")
                out[name] = {
                    "ms": msm, "iters_fp32": rm["iters_fp32"], "iters_fp64": rm["iters_fp64"], "F": rm["F"],
                    "converged": rm["converged"], "F_rel_diff_vs_fp64": abs(rm["F"] / r64["F"] - 1),
                    "max_link_diff_vs_fp64": float((Um - U64).abs().max().item()),
                    "speedup_vs_fp64": ms64 / msm}
                del Um
    del U64, U
    torch.cuda.empty_cache()
    return out


def ensemble_leg(args, stream, rank):
    """The 58-lattice ensemble (32 x 16^4, 16 x 24^4, 8 x 32^3x64, 2 x 48^3x96, eps
    uniform in [0.15, 0.5] from seed 5000, member i seeded 5000 + i), mixed
    precision, one graph launch per pass: one warm-up pass (autotuning and graph
    build), then one timed pass at switch 1e-6 and one at 1e-13."""
    import torch

    from paper_1301_3460_gb300 import inputs, lgf

    dims = [d for n, d in ENSEMBLE for _ in range(n)]
    eps = np.random.default_rng(5000).uniform(0.15, 0.5, size=len(dims))
    dev = [inputs.rough_gauge_field_cuda(d, float(e), 5000 + i + 1000 * rank) for i, (d, e) in enumerate(zip(dims, eps))]
    out = {"lattices": len(dims), "sites": int(sum(int(np.prod(d)) for d in dims))}
    with lgf.Batch(dims, mixed=True, stream=stream) as b:
        def one_pass():
            for i, u in enumerate(dev):
                b.set_links(i, u)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = b.fix(args.alpha, args.tol, args.max_iter)
            e1.record(stream)
            torch.cuda.synchronize()
            return r, e0.elapsed_time(e1)

        b.set_switch_tol(1e-6)
        one_pass()  # warm-up
        for accel, sw in ((64, 1e-6), (64, 1e-13), (32, 1e-6), (32, 1e-13)):
            if accel == 32 and sw == 1e-6:
                # the accelerator's transforms in FP32 inside the FP64 iterations
                b.set_accel_precision(32)
                b.set_switch_tol(sw)
                one_pass()  # warm-up of the new graph
            b.set_switch_tol(sw)
            r, ms = one_pass()
            tt = np.array(r["t_retire_ms"])
            out[("switch_%g" if accel == 64 else "accel_fp32_switch_%g") % sw] = {
                "ms": ms, "configs_per_hour": len(dims) / ms * 3.6e6,
                "time_to_theta_ms": {"p50": float(np.percentile(tt, 50)), "p99": float(np.percentile(tt, 99)),
                                     "max": float(tt.max())},
                "all_converged": all(st == lgf.LGF_OK for st in r["status"]),
                "iters_fp32_mean": float(np.mean(r["iters_fp32"])),
                "iters_fp64_mean": float(np.mean(r["iters_fp64"]))}
    del dev
    torch.cuda.empty_cache()
    return out


def run_ensemble(args):
    """32 x 16^4, 16 x 24^4, 8 x 32^3x64, 2 x 48^3x96 in mixed precision, eps uniform
    in [0.15, 0.5] (seed 5000), configuration i seeded 5000 + i, fixed by one graph
    launch per step; metric configs/hour with p50/p99 time-to-theta."""
    import torch

    from paper_1301_3460_gb300 import inputs, lgf

    ws, rank, local = dist()
    torch.cuda.set_device(local)
    dims = [d for n, d in ENSEMBLE for _ in range(n)]
    eps = np.random.default_rng(5000).uniform(0.15, 0.5, size=len(dims))
    t0 = time.time()

    def log(msg):
        sys.stderr.write("[ensemble %.1fs] %s\n" % (time.time() - t0, msg))
        sys.stderr.flush()

    dev = [inputs.rough_gauge_field_cuda(d, float(e), 5000 + i + 1000 * rank) for i, (d, e) in enumerate(zip(dims, eps))]
    log("generated %d lattices" % len(dev))
    stream = torch.cuda.current_stream()
    b = lgf.Batch(dims, mixed=True, stream=stream)
    b.set_switch_tol(args.switch_tol)
    log("batch created")

    def step():
        for i, u in enumerate(dev):
            b.set_links(i, u)
        return b.fix(args.alpha, args.tol, args.max_iter)

    clocks = Clocks(local)
    clocks.start()
    for _ in range(max(1, args.warmup)):
        r = step()
        log("warm-up step: iters %s" % r["iters"][:4])
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = []
    e0.record(stream)
    for _ in range(args.steps):
        res.append(step())
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    T = e0.elapsed_time(e1) / 1000.0
    n_cfg = len(dims) * args.steps
    tt = np.array([t for r in res for t in r["t_retire_ms"]])
    sites = sum(int(np.prod(d)) for d in dims)
    line = {
        "metric": "ensemble configs/hour (p50/p99 time-to-theta<1e-15)", "value": n_cfg / T * 3600.0,
        "unit": "configs/hour", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * T / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32->f64", "data": "synthetic",
        "config": {"workload": "ensemble 32x16^4 + 16x24^4 + 8x32^3x64 + 2x48^3x96, mixed precision, one graph "
                               "launch per step, eps U[0.15,0.5]", "sites": sites, "lattices": len(dims),
                   "switch_tol": args.switch_tol},
        "time_to_theta_ms": {"p50": float(np.percentile(tt, 50)), "p99": float(np.percentile(tt, 99)),
                             "max": float(tt.max())},
        "all_converged": all(s == lgf.LGF_OK for r in res for s in r["status"]),
        "iters": {"fp32_mean": float(np.mean(res[-1]["iters_fp32"])), "fp64_mean": float(np.mean(res[-1]["iters_fp64"]))},
        "clocks": clk,
    }
    b.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_wilson(args, dims):
    """Wilson-action configuration generation: one step = one compound sweep (a
    heat-bath sweep and four overrelaxation sweeps) of every link of the lattice,
    from a cold start thermalised by the warm-up steps."""
    import torch

    from paper_1301_3460_gb300 import lgf, roofline

    ws, rank, local = dist()
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as tdist

        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = tdist
    lgf.load()
    V = int(np.prod(dims))
    stream = torch.cuda.current_stream()
    n_or = 4
    lat = lgf.Lattice(dims, track_gauge=False, stream=stream)
    lat.set_unit_links()
    seed = 1000 + rank
    clocks = Clocks(local)
    clocks.start()
    for k in range(args.warmup):
        lat.wilson_sweeps(args.beta, seed, first_sweep=k, n_heatbath=1, n_overrelax=n_or)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        lat.wilson_sweeps(args.beta, seed, first_sweep=args.warmup + k, n_heatbath=1, n_overrelax=n_or)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    T = e0.elapsed_time(e1) / 1000.0
    T, n = reduce_over_ranks(pg, T, args.steps)
    # the two kernels on their own: heat-bath and overrelaxation sweeps
    kinds = {}
    for lab, nhb, nor in (("heatbath", 1, 0), ("overrelax", 0, 1)):
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for k in range(3):
            lat.wilson_sweeps(args.beta, seed, first_sweep=args.warmup + args.steps + k, n_heatbath=nhb,
                              n_overrelax=nor)
        f1.record(stream)
        torch.cuda.synchronize()
        msw = f0.elapsed_time(f1) / 3
        gf = roofline.WILSON_FLOPS_PER_LINK * 4 * V / msw / 1e6
        kinds[lab] = {"ms_per_sweep": msw, "ms_per_launch": msw / 8, "gflops": gf}
    lat.set_generator_precision(32)
    for lab, nhb, nor in (("heatbath_fp32", 1, 0), ("overrelax_fp32", 0, 1)):
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for k in range(3):
            lat.wilson_sweeps(args.beta, seed, first_sweep=args.warmup + args.steps + 3 + k, n_heatbath=nhb,
                              n_overrelax=nor)
        f1.record(stream)
        torch.cuda.synchronize()
        kinds[lab] = {"ms_per_sweep": f0.elapsed_time(f1) / 3}
    plaq = lat.plaquette()
    lat.close()
    hb = kinds["heatbath"]
    roof = {"bound": "alu", "kernel": "k_wilson (heat bath)", "achieved": hb["gflops"], "peak": FP64_PEAK_GFLOPS,
            "unit": "GFLOP/s", "frac": hb["gflops"] / FP64_PEAK_GFLOPS, "traffic": None,
            "peak_source": "GB300 FP64: 152 SMs x 4 flops/cycle x 2.07 GHz; flops per link exclude the sampler's "
                           "transcendental functions"}
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        from oracle import oracle as orc
        from paper_1301_3460_gb300 import inputs

        Ls = (16, 16, 16, 16)
        Us = inputs.unit_field(Ls)
        t0 = time.perf_counter()
        Us = orc.wilson_sweeps(Ls, Us, args.beta, seed, 1, mode=0)
        Us = orc.wilson_sweeps(Ls, Us, args.beta, seed, n_or, mode=1)
        dt = (time.perf_counter() - t0) * V / int(np.prod(Ls))
        cpu = {"value": 1.0 / dt, "unit": "compound sweeps/s", "cores": 1, "kind": "oracle",
               "sample": "one compound sweep of a 16^4 lattice from a cold start, scaled by volume to %s"
               % "x".join(map(str, dims))}
    if rank == 0:
        line = {
            "metric": "Wilson-action compound sweeps/s (1 heat bath + %d overrelaxation)" % n_or,
            "value": n / T, "unit": "compound sweeps/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * T / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": "SU(3) %s Wilson action beta=%g, checkerboard SU(2)-subgroup heat bath + "
                                   "overrelaxation, 12-real links, cold start" % ("x".join(map(str, dims)), args.beta),
                       "l2": "links larger than L2 (%.0f MB)" % (4 * V * 12 * 8 / 1e6),
                       "parallelism": "replicas" if ws > 1 else "single"},
            "kernels": kinds, "plaquette": plaq, "roofline": roof, "cpu_baseline": cpu,
            "gpu_launches": args.steps * 8 * (1 + n_or), "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


def run_kernels(args, dims):
    """The iteration kernels of one lattice (eps = 0.3, drawn on the GPU) launched
    one by one, FP64 and FP32, --steps iterations after --warmup: median event
    time per launch, algorithmic bytes and flops per second, fraction of the
    measured HBM peak."""
    import torch

    from paper_1301_3460_gb300 import inputs, lgf, roofline

    V = int(np.prod(dims))
    hbm = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    U = inputs.rough_gauge_field_cuda(dims, 0.3, 77)
    out = {"metric": "iteration kernels, median ms per launch", "dims": list(dims), "autotuned": not args.no_autotune}
    with lgf.Lattice(dims, mixed=True) as lat:
        lat.set_links(U)
        if not args.no_autotune:
            lat.autotune()
        if args.zt_form >= 0:
            lat.set_shape(64, nt_xy=128, nt_zt=128, xw=4, zt_form=args.zt_form)
            lat.set_shape(32, nt_xy=128, nt_zt=256, xw=4, zt_form=args.zt_form)
        out["shapes"] = {"fp64": lat.get_shape(64), "fp32": lat.get_shape(32)}
        # FP64, FP32 in the two-kernel form, FP32 with the update fused with Delta,
        # FP64 iterations with the accelerator's transforms in FP32, and the FP32 phase's
        # default form (g builder and update in one persistent launch: both in the
        # g builder's slot)
        for name, prec, form in (("fp64", 64, 0), ("fp32", 32, 0), ("fp32_fused", 32, 1),
                                 ("fp64_accel_fp32", 64, 0), ("fp32_persistent", 32, 2)):
            lat.set_fp32_update(form)
            lat.set_accel_precision(32 if name == "fp64_accel_fp32" else 64)
            if args.warmup:
                lat.time_kernels(args.alpha, n_iter=args.warmup, precision=prec)
            ms = lat.time_kernels(args.alpha, n_iter=max(1, args.steps), precision=prec)
            out[name + "_iteration_ms"] = sum(ms.values())
            if form == 2:
                out[name] = {"delta_xyfft": {"ms": ms["delta_xyfft"]}, "zt_fft_accel": {"ms": ms["zt_fft_accel"]},
                             "g_and_update": {"ms": ms["xyifft_g"] + ms["update"]}}
                continue
            per = roofline.per_site(dims, prec, form == 1, accel32=(name == "fp64_accel_fp32"))
            out[name] = {k: {"ms": ms[k], "gbs": per[k]["bytes"] * V / ms[k] / 1e6,
                             "hbm_frac_of_measured": per[k]["bytes"] * V / ms[k] / 1e6 / hbm,
                             "gflops": per[k]["flops"] * V / ms[k] / 1e6} for k in ms}
        lat.set_fp32_update(2)
    print(json.dumps(out), flush=True)
    return 0


def slab_rate(dims, U, nranks: int, n_iter: int, warm: int = 2) -> float:
    """Iterations per second of the t-slab path with `nranks` slabs emulated on
    this GPU (device copies in place of the messages), over n_iter iterations
    from the input links U (host [4, V, 3, 3])."""
    import torch

    from paper_1301_3460_gb300.slabs import LocalExchange, Slab, fix_slabs

    slabs = [Slab(dims, nranks, r) for r in range(nranks)]
    try:
        Vs = U.shape[1] // nranks
        parts = [torch.from_numpy(np.ascontiguousarray(U[:, r * Vs:(r + 1) * Vs])).cuda() for r in range(nranks)]
        ex = LocalExchange(slabs)
        for s, u in zip(slabs, parts):
            s.set_links(u)
        fix_slabs(ex, tol=0.0, max_iter=warm)
        for s, u in zip(slabs, parts):
            s.set_links(u)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = fix_slabs(ex, tol=0.0, max_iter=n_iter)
        torch.cuda.synchronize()
        T = time.perf_counter() - t0
    finally:
        for s in slabs:
            s.close()
    return r["iters"] / T


def run_slabs(args, dims):
    """One lattice split into t-slabs: under torchrun one slab per GPU over NCCL
    (strong scaling: the lattice is fixed), else --slab-ranks slabs emulated on
    one GPU.  A step is --slab-iters iterations from the eps = 0.3 configuration;
    the host drives the loop (one theta/F reduction and four exchanges per
    iteration)."""
    import torch

    from paper_1301_3460_gb300 import inputs
    from paper_1301_3460_gb300.slabs import DistExchange, LocalExchange, Slab, fix_slabs

    ws, rank, local = dist()
    torch.cuda.set_device(local)
    U = inputs.rough_gauge_field(dims, EPS[1], SEEDS[1])
    if ws > 1:
        import torch.distributed as tdist

        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
        N = ws
        slabs = [Slab(dims, N, rank, stream=torch.cuda.current_stream())]
        ex = DistExchange(slabs[0])
        mine = [rank]
    else:
        N = args.slab_ranks
        slabs = [Slab(dims, N, r) for r in range(N)]
        ex = LocalExchange(slabs)
        mine = list(range(N))
    Vs = U.shape[1] // N
    parts = {r: torch.from_numpy(np.ascontiguousarray(U[:, r * Vs:(r + 1) * Vs])).cuda() for r in mine}

    def step():
        for s, r in zip(slabs, mine):
            s.set_links(parts[r])
        return fix_slabs(ex, tol=0.0, max_iter=args.slab_iters)["iters"]

    for _ in range(args.warmup):
        step()
    if ws > 1:
        tdist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    n = sum(step() for _ in range(args.steps))
    torch.cuda.synchronize()
    T = time.perf_counter() - t0
    if ws > 1:
        t = torch.tensor([T], device="cuda", dtype=torch.float64)
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        T = float(t.item())
    for s in slabs:
        s.close()
    if rank == 0:
        print(json.dumps({
            "metric": "SD iters/s of one %s lattice split into %d t-slabs" % ("x".join(map(str, dims)), N),
            "value": n / T, "unit": "iters/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * T / args.steps, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "t-slab decomposition, FP64, eps 0.3, %d iterations per step" % args.slab_iters,
                       "dims": list(dims), "slabs": N,
                       "ranks": "one per GPU over NCCL" if ws > 1 else "emulated on one GPU"}}), flush=True)
    if ws > 1:
        tdist.destroy_process_group()
    return 0


def run_probe(args):
    """FP64 and FP32 FMA rates (best of --steps launches after --warmup), with the
    SM clock sampled during the launches."""
    import torch

    from paper_1301_3460_gb300 import lgf

    torch.cuda.set_device(0)
    clocks = Clocks(0)
    clocks.start()
    out = {"metric": "FMA rate (an FMA = 2 flops)", "unit": "GFLOP/s", "per_sm_clock_nominal": {
        "fp64": FP64_PEAK_GFLOPS, "note": "152 SMs x 2 FP64 FMA per cycle x 2 flops x 2.07 GHz"}}
    for prec, n in ((64, 10000), (32, 200000)):
        for _ in range(args.warmup):
            lgf.probe_fma(prec, n)
        runs = [lgf.probe_fma(prec, n) for _ in range(max(1, args.steps))]
        best = max(runs, key=lambda r: r["gflops"])
        out["fp%d" % prec] = {"gflops": best["gflops"], "ms": best["ms"], "n_iter": n,
                              "all_gflops": [r["gflops"] for r in runs]}
    out["clocks"] = clocks.stop()
    out["fp64_frac_of_nominal"] = out["fp64"]["gflops"] / FP64_PEAK_GFLOPS
    print(json.dumps(out), flush=True)
    return 0


def main():
    args = parse()
    if args.workload == "probe":
        return run_probe(args)
    if args.workload == "kernels":
        return run_kernels(args, tuple(int(v) for v in args.dims.split(",")))
    if args.workload == "ensemble":
        return run_ensemble(args)
    if args.workload == "wilson":
        dims = tuple(int(v) for v in args.dims.split(","))
        return run_wilson(args, dims)
    if args.workload == "slabs":
        return run_slabs(args, tuple(int(v) for v in args.dims.split(",")))
    dims = tuple(int(v) for v in args.dims.split(","))
    if args.impl == "reference":
        return run_reference(args, dims)
    return run_ours(args, dims)


if __name__ == "__main__":
    sys.exit(main())
