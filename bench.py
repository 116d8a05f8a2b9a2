#!/usr/bin/env python
"""Benchmark of the real-space PAW eigensolver step on GB300.

One step = one Rayleigh-Ritz iteration of the whole hot path on one band block: H psi and
S psi (order-6 FD stencil + local potential + projector overlaps + nonlocal back-add), the
Gram matrices H_nm and S_nm, the subspace diagonalization (Cholesky + Jacobi eigh), and the
band rotation; the rotated bands feed the next step.  Default workload: 96^3 periodic grid
at 0.2 Angstrom, 256 real FP64 bands, 32 atoms x 18 projectors (seeded synthetic inputs).

Prints one JSON line (rank 0).  ``value`` is grid-point x band throughput of whole steps
(Gpt.band/s: K * nb per step / step time / 1e9) with inputs resident in HBM.
``--impl reference`` times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import csv
import io
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

from paper_2310_14776_gb300 import synth  # noqa: E402

METRIC = "H|psi> Gpt\u00b7band/s; Rayleigh-Ritz steps/s and p50/p99 latency vs plain FP64"
UNIT = "Gpt\u00b7band/s"
VALUE_DEF = ("grid points x bands of whole Rayleigh-Ritz steps (apply_H, apply_S, Hermitian Gram H and S, "
             "subspace diag, rotation) per second / 1e9, inputs resident in HBM")
HOST_PSI_MAX = 3e8           # larger band blocks are generated on the device (seeded torch RNG)
FP64_NOMINAL_TFLOPS = 1.25   # GB300 FP64 (vector and tensor), nominal
FP32_PROBE_TFLOPS = 70.1     # GB300 FP32 FMA rate measured by a DFMA/FFMA probe kernel on this machine


# Measured DRAM traffic of the dominant stage's kernels (ncu dram__bytes_read.sum +
# dram__bytes_write.sum of every kernel of one pawfd_gram_hs call at 64^3 x 256 bands).  At a
# fixed band count it grows with the grid points K
# (slicing and digit-plane reads per K block); valid only for that band count and while the
# kernels' sources are the ones that were measured.
_GRAM_SOURCES = {"paper_2310_14776_gb300/csrc/sliced_gram.cuh": "dcad82e720e6d74d785b8eceb2d43563d70a1ea4",
                 "paper_2310_14776_gb300/csrc/tc_gram.cu": "f71758ac3494c927ade28099fe219df55efa207c",
                 "paper_2310_14776_gb300/csrc/nonlocal.cu": "375a13b3bd58e662195fcecdc233878a150e7244",
                 "paper_2310_14776_gb300/csrc/tc_common.cuh": "69b7022593a46a5fea888d3ab59abd564beb1cc9"}
TRAFFIC = {
    ("gram_HS", "fp64", False): {"nb": 256, "per_point": 21819.6, "sources": _GRAM_SOURCES},
    ("gram_HS", "mixed", False): {"nb": 256, "per_point": 11975.8, "sources": _GRAM_SOURCES},
}


# Measured DRAM traffic per launch of the Gram MMA kernel (the mean of the two launches of one
# pawfd_gram_hs call, ncu at 64^3 x 256 bands), per grid
# point: FP64 (1887.1 + 15.0 + 940.7 + 5.5) / 2 MB, mixed (1075.2 + 4.6 + 537.9 + 1.3) / 2 MB.
KERNEL_TRAFFIC = {
    ("gram_mma", "fp64", False): {"nb": 256, "per_point": 1424.15e6 / 262144, "sources": _GRAM_SOURCES},
    ("gram_mma", "mixed", False): {"nb": 256, "per_point": 809.5e6 / 262144, "sources": _GRAM_SOURCES},
}


def kernel_traffic(kernel, precision, cplx, K, nb):
    """DRAM bytes of one launch of the kernel, scaled from the measured small case, or None."""
    import hashlib
    t = KERNEL_TRAFFIC.get((kernel, precision, cplx))
    if t is None or t["nb"] != nb:
        return None
    for path, sha in t["sources"].items():
        with open(os.path.join(ROOT, path), "rb") as f:
            if hashlib.sha1(f.read()).hexdigest() != sha:
                return None
    return t["per_point"] * K


def sg_tiles_area(nb):
    """Output entries the real Hermitian Gram kernel computes: for 192 < nb <= 256 the four
    128 x 96 tiles of the symmetric cover, otherwise the 128 x 96 tiles holding an element with
    row <= column."""
    if 192 < nb <= 256:
        return 4 * 128 * 96
    tr, tcn = (nb + 127) // 128, (nb + 95) // 96
    return sum(max(0, tcn - (128 * r) // 96) for r in range(tr)) * 128 * 96


def stage_traffic(stage, precision, cplx, K, nb, natoms):
    """DRAM bytes of one launch of the stage, scaled from the measured small case, or None."""
    import hashlib
    t = TRAFFIC.get((stage, precision, cplx))
    if t is None or t["nb"] != nb:
        return None
    for path, sha in t["sources"].items():
        with open(os.path.join(ROOT, path), "rb") as f:
            if hashlib.sha1(f.read()).hexdigest() != sha:
                return None
    return t["per_point"] * K


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="pawfd", choices=["pawfd", "reference"])
    p.add_argument("--workload", default="gamma-96c-256b", choices=sorted(synth.WORKLOADS) + ["batch64", "served", "davidson", "density", "poisson", "pw"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--precision", default=None, choices=["fp64", "mixed"],
                   help="fp64 (default for single workloads) or mixed (default for batch64 / served)")
    p.add_argument("--rate", type=float, default=200.0, help="served: arrivals per second")
    p.add_argument("--serve-seconds", type=float, default=60.0, help="served: length of the arrival stream")
    p.add_argument("--serve-warmup", type=float, default=5.0, help="served: arrivals before this are excluded")
    p.add_argument("--real", action="store_true", help="batch64 / served: real (Gamma) instead of Bloch instances")
    p.add_argument("--no-refine", action="store_true", help="mixed: skip the final FP64 refinement measurement")
    p.add_argument("--bands", type=int, default=0,
                   help="single workloads: this many bands instead of the workload's own (profiling cases)")
    p.add_argument("--tc-scratch-mb", type=int, default=8192,
                   help="single workloads and batch64: digit-plane scratch of the tensor-core Gram and rotation "
                        "per context (MB); 0 keeps the library's default block sizes")
    a = p.parse_args()
    if a.precision is None:
        a.precision = "mixed" if a.workload in ("batch64", "served") else "fp64"
    return a


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(seconds, world, dev):
    """The job's timed region: the longest of the ranks' own timed regions (an all-reduce MAX
    over the process group in float64; the identity for one rank)."""
    if world == 1:
        return seconds
    import torch
    import torch.distributed as dist
    t = torch.tensor([seconds], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, seconds):
    """Whole-job throughput in 1e9 units per second: the units all ranks processed (each rank
    the same, weak scaling) over the job's time."""
    return units_per_rank * world / seconds / 1e9


def single_gpu_arm(name):
    """Workloads measured on one GPU only: under a multi-rank launch, rank 0 runs them and the
    other ranks return at once (True when this rank should run)."""
    world, rank, _ = dist_env()
    if world > 1 and rank != 0:
        return False
    if world > 1:
        print("%s: a single-GPU workload; rank 0 runs it alone" % name, file=sys.stderr, flush=True)
    return True


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# ------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.out,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.close()
        rows = list(csv.reader(io.StringIO(open(self.path).read())))
        os.unlink(self.path)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for name, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------
def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_2310_14776_gb300 import api

    world, rank, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = synth.WORKLOADS[args.workload]
    system = w.system()
    nb, K = (args.bands or w.nbands), system.npoints
    cplx = system.complex_wf
    ctx = api.Context(system, max_bands=nb, device=dev, precision=args.precision)
    if args.tc_scratch_mb:
        ctx.set_option("tc_scratch_mb", args.tc_scratch_mb)
    if nb * K <= HOST_PSI_MAX and nb == w.nbands:
        psi_host = w.psi(system)
        if args.precision == "mixed":
            psi_host = psi_host.astype(np.complex64 if cplx else np.float32)
        psi0 = torch.from_numpy(psi_host).to(dev)
        psi_src = "seeded SplitMix64 on the host"
    else:
        psi_host = None
        psi0 = device_bands(ctx, nb, w.seed)
        psi_src = "seeded torch generator on the device (uniform(-1, 1))"
        args.no_e2e = True
    esize = psi0.element_size()
    # the random start, kept for the whole-job timing below when it is small enough to copy
    psi_start = psi0.clone() if nb * K * esize <= 4e9 else None
    psi = [psi0, torch.empty_like(psi0)]
    work = {"Hpsi": ctx.empty_bands(nb), "Spsi": ctx.empty_bands(nb),
            "P": torch.empty((max(ctx.Ip, 1), nb), dtype=ctx.dtype, device=dev),
            "Hnm": torch.empty((nb, nb), dtype=ctx.mat_dtype, device=dev),
            "Snm": torch.empty((nb, nb), dtype=ctx.mat_dtype, device=dev),
            "eps": torch.empty(nb, dtype=torch.float64, device=dev),
            "C": torch.empty((nb, nb), dtype=ctx.mat_dtype, device=dev)}
    stream = torch.cuda.current_stream(dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def step(cur, nxt, marks=None):
        # the calls of pawfd_rr_step, one library call per stage; marks: events between the
        # stages apply_HS | Gram H and S | subspace | rotate
        def mark(i):
            if marks is not None:
                marks[i].record(stream)
        mark(0)
        ctx.apply_hs(cur, Hpsi=work["Hpsi"], Spsi=work["Spsi"], P=work["P"])
        mark(1)
        ctx.gram_hs(cur, work["Hpsi"], work["P"], Hnm=work["Hnm"], Snm=work["Snm"])
        mark(2)
        ctx.subspace_diag(work["Hnm"], work["Snm"], eps=work["eps"], C=work["C"], overwrite=True, check=False)
        mark(3)
        ctx.rotate(cur, work["C"], out=nxt)
        mark(4)

    def whole_step(cur, nxt):
        # the step as one library call (pawfd_rr_step): it also overlaps the rotation's
        # slicing of psi with the subspace solve
        ctx.rr_step(cur, out=nxt, work=work)

    for i in range(args.warmup):
        step(psi[i % 2], psi[(i + 1) % 2])
    ctx.sync()
    eps_first = work["eps"].clone()

    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    launches0 = ctx.launch_count()
    ctx.kernel_timing(True)       # CUDA events around every Gram MMA kernel launch from here
    step_ev = [ev() for _ in range(args.steps + 1)]
    t0, t1 = step_ev[0], step_ev[-1]
    t0.record(stream)
    for i in range(args.steps):
        whole_step(psi[(args.warmup + i) % 2], psi[(args.warmup + i + 1) % 2])
        step_ev[i + 1].record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ctx.sync()
    mma_ms, mma_launches = ctx.kernel_timing(False)
    launches = ctx.launch_count() - launches0
    elapsed = t0.elapsed_time(t1) * 1e-3
    step_ms = [step_ev[i].elapsed_time(step_ev[i + 1]) for i in range(args.steps)]
    drift = float(torch.max(torch.abs(work["eps"] - eps_first)).item())
    # the stage breakdown, from a second (untimed for the value) run of the same steps with
    # one library call per stage and events between them
    marks = [[ev() for _ in range(5)] for _ in range(args.steps)]
    for i in range(args.steps):
        step(psi[(args.warmup + args.steps + i) % 2], psi[(args.warmup + args.steps + i + 1) % 2], marks[i])
    torch.cuda.synchronize(dev)
    ctx.sync()
    latest_idx = (args.warmup + 2 * args.steps) % 2   # the newest rotated bands, and their eps
    eps_latest = work["eps"].clone()
    C_latest = work["C"].clone() if args.precision == "mixed" else None
    # a whole job of ten steps from the random start: its first step takes the far path of the
    # subspace solve (Cholesky reduction, FP32 tridiagonal eigenbasis, FP64 refinement), which
    # the warm-up steps absorb in the timed value; the later steps are near-Ritz steps
    job = None
    if psi_start is not None:
        scratch = psi[1 - latest_idx].clone()
        jev = [ev() for _ in range(11)]
        jev[0].record(stream)
        cur, nxt = psi_start, scratch
        for i in range(10):
            whole_step(cur, nxt)
            jev[i + 1].record(stream)
            cur, nxt = nxt, cur
        torch.cuda.synchronize(dev)
        ctx.sync()
        jms = [jev[i].elapsed_time(jev[i + 1]) for i in range(10)]
        job = {"steps": 10, "job_ms": float(sum(jms)), "first_step_ms": jms[0],
               "later_steps_mean_ms": float(np.mean(jms[1:])),
               "what": "ten pawfd_rr_step calls from the seeded random bands, CUDA events around each"}
        del scratch, psi_start
    elapsed = max_over_ranks(elapsed, world, dev)
    names = ["apply_HS", "gram_HS", "subspace_diag", "rotate"]
    stages = {nm: statistics.mean(m[i].elapsed_time(m[i + 1]) for m in marks) for i, nm in enumerate(names)}

    value = job_throughput(float(nb) * K * args.steps, world, elapsed)
    mixed = args.precision == "mixed"
    peaks = load_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    bf16 = peaks.get("bf16_tflops", 1900.0)
    # digit products per real multiply-add of the tensor-core kernels (orders <= 6 of 7 digits
    # for FP64 data, <= 4 of 4 digits for FP32 data) and real multiply-adds per complex one
    products = 13 if mixed else 28
    cfac = 4 if cplx else 1
    # algorithmic work per stage: bytes that must move (apply), useful digit products (Gram,
    # rotation)
    work_units = {
        # H psi and S psi: psi read twice (stencil, copy), H psi and S psi written once
        "apply_HS": ("hbm", 4.0 * esize * nb * K, hbm * 1e9, "B/s"),
        # the two Hermitian Gram matrices (upper triangles), digit products on the tensor cores
        "gram_HS": ("tensor", 2 * 2.0 * products * cfac * nb * (nb + 1) / 2 * K, bf16 * 1e12, "BF16 FLOP/s"),
        "rotate": ("tensor", 2.0 * products * cfac * nb * nb * K, bf16 * 1e12, "BF16 FLOP/s"),
    }
    dom = max((k for k in stages if k in work_units), key=lambda k: stages[k])
    bound, amount, peak, unit = work_units[dom]
    achieved = amount / (stages[dom] * 1e-3)
    kernel_of = {"apply_HS": "stencil + project_kernel + nonlocal_add_kernel (x2) + copy",
                 "gram_HS": "slice_kernel (x2) + sliced_gram_kernel (x2) + overlap correction",
                 "rotate": "slice_t_kernel + sliced_gram_kernel (digit-product rotation)"}
    scale = 1e12 if unit.endswith("FLOP/s") or unit == "FP64 instr/s" else 1e9
    roof_unit = {"BF16 FLOP/s": "TFLOP/s", "FP64 instr/s": "Tinstr/s", "B/s": "GB/s"}[unit]
    # the dominant kernel: the Gram MMA kernel (two launches per pawfd_gram_hs call), timed by
    # CUDA events around each launch on the context's stream; algorithmic work per launch = the
    # digit products of one Hermitian Gram's upper triangle
    mma_avg_ms = mma_ms / mma_launches if mma_launches and mma_launches > 0 else None
    gram_launch_flops = 2.0 * products * cfac * nb * (nb + 1) / 2 * K
    kernel_roof = None
    if mma_avg_ms:
        # two Hermitian Grams per step, over however many K-block launches they took
        ach = 2 * args.steps * gram_launch_flops / (mma_ms * 1e-3)
        kernel_roof = {"kernel": "sliced_gram_kernel (Gram mode; %d launches timed)" % mma_launches,
                       "bound": "tensor", "achieved": ach / 1e12, "peak": bf16, "unit": "TFLOP/s",
                       "frac": ach / (bf16 * 1e12), "avg_launch_ms": mma_avg_ms,
                       "traffic": kernel_traffic("gram_mma", args.precision, cplx, K, nb),
                       "traffic_unit": "DRAM bytes per launch (ncu at 64^3 x 256 bands, mean of the pair's two "
                                       "launches, scaled by grid points)",
                       "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst)",
                       "work": "useful (Hermitian upper-triangle) BF16 digit products of the step's two Grams "
                               "over the summed launch times" + (
                                   "" if cplx else "; the kernel executes %.2fx that in 128 x 96 tiles"
                                   % (sg_tiles_area(nb) / (nb * (nb + 1) / 2)))}

    result = {
        "metric": METRIC, "value_definition": VALUE_DEF,
        "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {8: "f64", 16: "c128", 4: "f32"}[esize] if not (mixed and cplx) else "c64",
        "data": "synthetic (seeded; bands: %s)" % psi_src,
        "config": {"workload": w.name, "grid": list(system.n), "bands": nb, "atoms": system.natoms,
                   "projectors_per_atom": int(system.nproj[0]) if system.natoms else 0,
                   "precision": args.precision, "parallelism": "replicas" if world > 1 else "single-gpu",
                   "tc_scratch_mb": args.tc_scratch_mb,
                   "l2": "inputs larger than L2 (%.2f GB of bands per step)" % (2 * nb * K * esize / 1e9)},
        "rr_steps_per_s": args.steps * world / elapsed,
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
        "stages_ms": stages,
        "stages_note": "per-stage times from a second run of the same number of steps with one library call per "
                       "stage (the timed value calls pawfd_rr_step, which also overlaps the rotation's slicing "
                       "of psi with the subspace solve)",
        "apply_HS_gptband_s": nb * K / (stages["apply_HS"] * 1e-3) / 1e9,
        "eig_drift_ha": drift,
        "job": job,
        "roofline": kernel_roof,
        "stage_roofline": {"stage": dom, "kernel": kernel_of[dom], "bound": bound, "achieved": achieved / scale,
                           "peak": peak / scale, "unit": roof_unit, "frac": achieved / peak,
                           "traffic": stage_traffic(dom, args.precision, cplx, K, nb, system.natoms),
                           "traffic_unit": "DRAM bytes per stage call (ncu at 64^3 x 256 bands, scaled by grid "
                                           "points)",
                           "peak_source": {"tensor": "MEASURED_PEAKS.json bf16_tflops (burst)",
                                           "hbm": "MEASURED_PEAKS.json hbm_gbs",
                                           "alu": "nominal GB300 FP64 rate 1.25 TFLOP/s / 2 (FMA)"}[bound]},
        "gpu_launches": int(launches),
        "clocks": clk,
    }

    if not args.no_e2e:
        result["e2e"] = e2e_gpu(ctx, psi_host, work, args, dev)
    if mixed and not args.no_refine:
        # the last step's input bands and its eigenvector matrix (the refinement rotates the
        # former by the latter in FP64); its rotated output is not needed
        last_in = psi[1 - latest_idx]
        C_last = C_latest
        eps_mixed = eps_latest
        for key in ("Hpsi", "Spsi"):
            work[key] = None
        psi[latest_idx] = None
        torch.cuda.empty_cache()
        result["refine"] = refine_gpu(system, nb, last_in, C_last, eps_mixed, dev, args.tc_scratch_mb)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(system, w, args.precision)
    if world > 1:
        dist.barrier()
    ctx.close()
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        dist.destroy_process_group()


def refine_gpu(system, nb, psi_in, C_lo, eps_mixed, dev, tc_scratch_mb=0):
    """The final FP64 refinement (pawfd_refine) of the last mixed step: its input bands psi_in
    rotated by its eigenvector matrix C_lo in FP64, then an FP64 Rayleigh-Ritz step; timed.
    The refined eigenvalues are compared with the plain FP64 path of the same library on the
    same input (apply_HS, Gram H and S, subspace solve of the promoted FP32 values), the path
    the full-size FP64 parity test checks against the oracle."""
    import torch
    from paper_2310_14776_gb300 import api
    fp = api.Context(system, max_bands=nb, device=dev, precision="fp64")
    if tc_scratch_mb:
        fp.set_option("tc_scratch_mb", tc_scratch_mb)
    fp.refine(psi_in, C_lo)        # untimed first call
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    out = fp.refine(psi_in, C_lo, check=False)
    e1.record()
    torch.cuda.synchronize(dev)
    fp.sync()
    ms = e0.elapsed_time(e1)
    eps = out["eps"].clone()
    theta = out["theta"].clone()
    resid = out["resid"].clone()
    # the plain FP64 step on the same input, in the refinement's work arrays
    x = out["psi"]
    x.copy_(psi_in)                # exact promotion of the FP32 values
    P = torch.empty((max(fp.Ip, 1), nb), dtype=fp.dtype, device=dev)
    fp.apply_hs(x, Hpsi=out["Hpsi"], Spsi=out["Spsi"], P=P)
    fp.gram_hs(x, out["Hpsi"], P, Hnm=out["Hnm"], Snm=out["Snm"])
    eps64, _ = fp.subspace_diag(out["Hnm"], out["Snm"], C=out["C"], overwrite=True)
    torch.cuda.synchronize(dev)
    res = {"ms": ms,
           "max_abs_eps_refined_minus_fp64_ha": float((eps - eps64).abs().max()),
           "max_abs_eps_mixed_minus_fp64_ha": float((eps_mixed - eps64).abs().max()),
           "max_abs_theta_minus_eps_ha": float((theta - eps).abs().max()),
           "max_residual_norm": float(resid.max()), "median_residual_norm": float(resid.median()),
           "tolerance_ha": 1e-8,
           "what": "psi' = psi_in C_lo rotated in FP64 (psi_in, C_lo: the last mixed step's input bands and "
                   "eigenvector matrix), FP64 H psi' and S psi', Hermitian Grams, Rayleigh quotients, second "
                   "subspace solve, residual norms ||H psi'_n - eps_n S psi'_n||; errors against the FP64 "
                   "Rayleigh-Ritz step of the same library on the same input"}
    fp.close()
    del out, P, x
    torch.cuda.empty_cache()
    return res


def device_bands(ctx, nb, seed):
    """uniform(-1, 1) bands generated on the device by a seeded torch generator."""
    import torch
    g = torch.Generator(device=ctx.device)
    g.manual_seed(int(seed))
    shape = (nb,) + tuple(ctx.n[::-1])
    rdt = torch.float32 if ctx.precision == "mixed" else torch.float64
    re = torch.rand(shape, generator=g, device=ctx.device, dtype=rdt) * 2 - 1
    if not ctx.complex:
        return re
    im = torch.rand(shape, generator=g, device=ctx.device, dtype=rdt) * 2 - 1
    return torch.complex(re, im)


def e2e_gpu(ctx, psi_host, work, args, dev):
    """The same iterated step through the public API with host buffers: every step copies its
    input bands from pinned host memory to the device, makes one pawfd_rr_step call and copies
    the eigenvalues and the rotated bands back; the next step's input is that host copy (the
    bands stay on the host between steps, as in a host-driven loop)."""
    import torch
    nb = psi_host.shape[0]
    h_bufs = [torch.from_numpy(psi_host).pin_memory(), torch.empty_like(torch.from_numpy(psi_host)).pin_memory()]
    h_eps = torch.empty(nb, dtype=torch.float64).pin_memory()
    d_in = torch.empty_like(h_bufs[0], device=dev)
    d_out = torch.empty_like(h_bufs[0], device=dev)
    stream = torch.cuda.current_stream(dev)
    it = [0]

    def one():
        h_in, h_out = h_bufs[it[0] % 2], h_bufs[(it[0] + 1) % 2]
        d_in.copy_(h_in, non_blocking=True)
        ctx.rr_step(d_in, out=d_out, work=work)      # the single public call of one step
        h_eps.copy_(work["eps"], non_blocking=True)
        h_out.copy_(d_out, non_blocking=True)
        it[0] += 1

    # untimed: the first steps from the random start (the Cholesky path and dense Jacobi sweeps)
    for _ in range(2):
        one()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.e2e_steps):
        one()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ctx.sync()
    el = e0.elapsed_time(e1) * 1e-3
    K = psi_host[0].size
    per_step_bytes = h_bufs[0].numel() * h_bufs[0].element_size()
    return {"value": nb * K * args.e2e_steps / el / 1e9, "unit": UNIT, "steps": args.e2e_steps,
            "api": "Context.rr_step (pawfd_rr_step) with pinned host buffers; each step's input is the previous "
                   "step's rotated bands read back to the host",
            "h2d_bytes_per_step": per_step_bytes, "d2h_bytes_per_step": per_step_bytes + nb * 8}


# ------------------------------------------------------------------------------------------
# Batched and served forms
# ------------------------------------------------------------------------------------------
def contraction_bf16_flops(inst, precision):
    """BF16 digit-product FLOP of one instance step's Hermitian Gram pair and rotation."""
    products = 13 if precision == "mixed" else 28
    cfac = 4 if inst.complex_wf else 1
    nb, K = inst.nbands, inst.npoints
    return 2.0 * products * cfac * (2 * nb * (nb + 1) / 2 + nb * nb) * K


def fp64_step_seconds(inst, dev, system=None, reps=1):
    """One plain FP64 single-instance step (pawfd_rr_step, eager), timed after one warm-up step."""
    import torch
    from paper_2310_14776_gb300 import api
    s = system if system is not None else inst.system()
    ctx = api.Context(s, max_bands=inst.nbands, device=dev, precision="fp64")
    psi = device_bands(ctx, inst.nbands, inst.seed)
    out = torch.empty_like(psi)
    work = ctx.alloc_work(inst.nbands)
    ctx.rr_step(psi, out=out, work=work)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        ctx.rr_step(psi, out=out, work=work)
    e1.record()
    torch.cuda.synchronize(dev)
    ctx.sync()
    t = e0.elapsed_time(e1) * 1e-3 / reps
    ctx.close()
    del psi, out, work
    torch.cuda.empty_cache()
    return t


def run_batch(args):
    """64 independent instances (seeded sizes), one RR step of all of them per graph launch."""
    import torch
    import torch.distributed as dist
    from paper_2310_14776_gb300 import api, autotune

    world, rank, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    insts = synth.batch_instances(64, complex_wf=not args.real)
    ent_a, ent_b, tuned = [], [], {}
    for inst in insts:
        ctx = api.Context(inst.system(), max_bands=inst.nbands, device=dev, precision=args.precision)
        if args.tc_scratch_mb:
            # the whole grid in one K block (every instance's planes fit in 8 GB)
            ctx.set_option("tc_scratch_mb", args.tc_scratch_mb)
        psi_a = device_bands(ctx, inst.nbands, inst.seed)
        psi_b = torch.empty_like(psi_a)
        work = ctx.alloc_work(inst.nbands)
        work["C"].copy_(torch.eye(inst.nbands, dtype=work["C"].dtype, device=dev))
        opts = autotune.tune(ctx, psi_a, work)
        tuned[str(autotune.shape_key(ctx, inst.nbands))] = opts
        ent_a.append((ctx, psi_a, psi_b, work))
        ent_b.append((ctx, psi_b, psi_a, work))
    batches = [api.Batch(ent_a, use_graph=True), api.Batch(ent_b, use_graph=True)]
    for i in range(args.warmup):
        batches[i % 2].launch()
    for b in batches:
        b.sync()
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    evs[0].record()
    for i in range(args.steps):
        batches[(args.warmup + i) % 2].launch()
        evs[i + 1].record()
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    for b in batches:
        b.sync()
    elapsed = evs[0].elapsed_time(evs[-1]) * 1e-3
    elapsed = max_over_ranks(elapsed, world, dev)
    per_launch = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]
    units = sum(inst.npoints * inst.nbands for inst in insts)
    value = job_throughput(units * args.steps, world, elapsed)
    rr = len(insts) * args.steps * world / elapsed
    flops = sum(contraction_bf16_flops(inst, args.precision) for inst in insts)
    peaks = load_peaks()
    bf16 = peaks.get("bf16_tflops", 1900.0)
    achieved = flops * args.steps / elapsed
    graph = all(b.is_graph for b in batches)
    kernels = batches[0].kernel_count
    for b in batches:
        b.close()
    for ctx, *_ in ent_a:
        ctx.close()
    del ent_a, ent_b, batches
    torch.cuda.empty_cache()
    # the plain FP64 single-instance path on the same instances, one after another
    fp64_total = 0.0
    if rank == 0:
        fp64_total = sum(fp64_step_seconds(inst, dev) for inst in insts)
    result = {
        "metric": METRIC, "value_definition": VALUE_DEF + " (summed over the batch's instances)",
        "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": ("c64" if not args.real else "f32") if args.precision == "mixed"
        else ("c128" if not args.real else "f64"),
        "data": "synthetic (seeded sizes; bands from a seeded torch generator on the device)",
        "config": {"workload": "batch64: 64 instances, grids 32-80 per axis, 32-256 bands, 2-24 atoms x 18 "
                               "projectors, %s" % ("Bloch k" if not args.real else "Gamma"),
                   "instances": len(insts), "points_x_bands": units, "precision": args.precision,
                   "launch": "one CUDA graph launch per batch step" if graph else "eager streams",
                   "parallelism": "replicas" if world > 1 else "single-gpu", "tc_scratch_mb": args.tc_scratch_mb,
                   "l2": "inputs larger than L2 (%.1f GB of bands per step)" % (
                       2 * units * (8 if not args.real else 4) * (2 if args.precision == "fp64" else 1) / 1e9)},
        "rr_steps_per_s": rr,
        "latency_ms": {"p50": float(np.percentile(per_launch, 50)), "p99": float(np.percentile(per_launch, 99))},
        "fp64_sequential": {"rr_steps_per_s": len(insts) / fp64_total if fp64_total else None,
                            "seconds_per_batch_step": fp64_total,
                            "how": "each instance alone, plain FP64 pawfd_rr_step, one after another"},
        "speedup_vs_fp64_sequential": (rr / world) / (len(insts) / fp64_total) if fp64_total else None,
        "autotuned": tuned,
        "roofline": {"stage": "whole batch step", "kernel": "sliced_gram_kernel (Gram pair + rotation of all "
                     "instances)", "bound": "tensor", "achieved": achieved / 1e12, "peak": bf16, "unit": "TFLOP/s",
                     "frac": achieved / (bf16 * 1e12), "traffic": None,
                     "note": "BF16 digit-product work of all contractions / whole batch step time (a lower bound "
                             "on the contraction kernels' own rate)"},
        "gpu_launches": int(kernels * args.steps), "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_served(args):
    """Poisson stream of eigensolver jobs through the continuous-batching server."""
    import torch
    from paper_2310_14776_gb300 import serve

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    systems = serve.catalogue(complex_wf=not args.real)
    jobs = serve.job_stream(args.rate, args.serve_seconds, 64, 8, seed=4 + rank)
    srv = serve.Server(systems, dev, precision=args.precision, iterations=5)
    srv.prepare(sorted({j.system for j in jobs}))
    clocks = ClockSampler(local)
    clocks.start()
    out = srv.run(jobs, duration=args.serve_seconds * 1.25 + 5.0)
    clk = clocks.stop()
    srv.close()
    recs = out["records"]
    steps_done = 5 * len(recs)
    lat = serve.latency_stats(recs, warmup=args.serve_warmup)
    lat_note = "jobs arriving after the warm-up window"
    if not lat.get("jobs"):
        # saturated stream served in arrival order: no job after the warm-up window finished
        lat = serve.latency_stats(recs, warmup=0.0)
        lat_note = "all completed jobs (none arriving after the warm-up window finished: the queue only grew)"
    arrived = [j for j in jobs if j.arrival <= out["elapsed"]]
    saturated = out["unfinished"] > 0
    # plain FP64 sequential on a sample of the same mix: 8 small systems and 1 large one
    small = [systems[i] for i in sorted({j.system for j in jobs if j.system < 64})[:8]]
    large = [systems[i] for i in sorted({j.system for j in jobs if j.system >= 64})[:1]]
    t_small = [fp64_step_seconds(inst, dev, srv.system(systems.index(inst))) for inst in small]
    t_large = [fp64_step_seconds(inst, dev, srv.system(systems.index(inst))) for inst in large]
    frac_large = sum(j.system >= 64 for j in jobs) / max(1, len(jobs))
    t_job = 5 * ((1 - frac_large) * float(np.mean(t_small)) + (frac_large * float(np.mean(t_large)) if t_large else 0))
    result = {
        "metric": METRIC, "value_definition": "grid points x bands of completed Rayleigh-Ritz steps per second / 1e9",
        "value": sum(5 * systems[r.job.system].npoints * systems[r.job.system].nbands for r in recs) / out["elapsed"] / 1e9,
        "unit": UNIT, "n_gpus": 1, "steps": steps_done, "warmup": 0, "ms_per_step": out["elapsed"] / max(1, steps_done) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64" if (args.precision == "mixed" and not args.real) else "mixed",
        "data": "synthetic (seeded catalogue of 72 systems; bands seeded per job on the device)",
        "config": {"workload": "served: Poisson %.0f jobs/s for %.0f s, 5 RR iterations per job, 90%% batched-size "
                               "systems and 10%% 128^3 x 512-band systems" % (args.rate, args.serve_seconds),
                   "precision": args.precision, "hbm_budget_gb": out["budget"] / 1e9, "max_active": srv.sched.max_active,
                   "parallelism": "single-gpu"},
        "rr_steps_per_s": steps_done / out["elapsed"],
        "latency_ms": {"p50": lat.get("p50_ms"), "p99": lat.get("p99_ms"), "jobs": lat.get("jobs"),
                       "over": lat_note, "warmup_s": args.serve_warmup},
        "jobs": {"arrived": len(arrived), "completed": len(recs), "unfinished_at_stop": out["unfinished"],
                 "max_queue": out["max_queue"], "peak_hbm_gb": out["peak_used"] / 1e9,
                 "device_peak_hbm_gb": out["device_peak_used"] / 1e9, "arena_gb": out["arena_bytes"] / 1e9,
                 "arena_peak_gb": out["arena_peak"] / 1e9, "contexts_gb": out["context_bytes"] / 1e9,
                 "budget_overruns": out["overruns"],
                 "device_peak_note": "free device memory at the server's start less the smallest free memory "
                                     "sampled during the run (every loop pass)"},
        "saturated": saturated,
        "max_sustainable_jobs_per_s": len(recs) / out["elapsed"] if saturated else ">= %.0f" % args.rate,
        "fp64_sequential": {"rr_steps_per_s": 5.0 / t_job if t_job else None, "seconds_per_job": t_job,
                            "how": "plain FP64 pawfd_rr_step, one job at a time, on 8 small and %d large systems "
                                   "of the stream, weighted by its large fraction %.3f" % (len(large), frac_large)},
        "speedup_vs_fp64_sequential": (steps_done / out["elapsed"]) / (5.0 / t_job) if t_job else None,
        "roofline": None, "gpu_launches": int(out["kernel_launches"]), "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(result), flush=True)


# ------------------------------------------------------------------------------------------
# Block-Davidson steps (the iterative eigensolver after the Rayleigh-Ritz step)
# ------------------------------------------------------------------------------------------
def run_davidson(args):
    """Block-Davidson steps (pawfd_davidson_step: residuals, corrections by the kinetic
    preconditioner -(T + 0.5 Ha)^-1, Rayleigh-Ritz over the 2n columns) on the 96^3 x 256-band
    FP64 system, started from Ritz vectors of three Rayleigh-Ritz steps of seeded random bands.
    An untimed run of ten steps from that start records the largest residual norm before each
    step and after the tenth."""
    import torch

    from paper_2310_14776_gb300 import api

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = synth.WORKLOADS["gamma-96c-256b"]
    system = w.system()
    nb, K = (args.bands or w.nbands), system.npoints
    ctx = api.Context(system, max_bands=2 * nb, device=dev, precision=args.precision)
    if args.tc_scratch_mb:
        ctx.set_option("tc_scratch_mb", 2 * args.tc_scratch_mb)
    psi = device_bands(ctx, nb, w.seed)
    work = ctx.alloc_work(nb)
    for _ in range(3):
        res = ctx.rr_step(psi, work=work)
        psi = res["psi_rot"].clone()
    W = ctx.alloc_davidson(nb)
    eps0 = work["eps"].clone()
    # convergence from the start: max residual norm of the input of steps 1 .. 11
    W["X"][:nb].copy_(psi)
    eps = eps0.clone()
    history = []
    for _ in range(11):
        ctx.davidson_step(W, nb, eps)
        history.append(float(W["rnorm"].max()))
        eps = W["eps"][:nb].clone()
        W["X"][:nb].copy_(W["psi_out"])
    lowest_after_10 = float(W["eps"][0])
    W["X"][:nb].copy_(psi)
    eps = eps0.clone()
    del psi, work
    for _ in range(args.warmup):
        ctx.davidson_step(W, nb, eps)
        eps = W["eps"][:nb].clone()
        W["X"][:nb].copy_(W["psi_out"])
    ctx.sync()
    r_start = W["rnorm"].clone()
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize(dev)
    l0 = ctx.launch_count()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    evs[0].record()
    for i in range(args.steps):
        ctx.davidson_step(W, nb, eps)
        eps = W["eps"][:nb].clone()
        W["X"][:nb].copy_(W["psi_out"])
        evs[i + 1].record()
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ctx.sync()
    launches = (ctx.launch_count() - l0) // max(1, args.steps)
    elapsed = evs[0].elapsed_time(evs[-1]) * 1e-3
    step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]
    r_end = W["rnorm"]
    cb = None
    if not args.no_cpu_baseline:
        from oracle import oracle as O
        O.build()
        nb_s = 16
        psi_s = w.psi(system, nb=nb_s)
        rr = O.rayleigh_ritz(system, psi_s)
        t = time.perf_counter()
        O.davidson_step(system, rr["psi_rot"], rr["eps"])
        ts = time.perf_counter() - t
        cb = {"value": K * nb_s / ts / 1e9, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle", "seconds": ts,
              "sample": "one oracle block-Davidson step (FP64) of the gamma-96c-256b system on %d bands" % nb_s}
    esize = 4 if args.precision == "mixed" else 8
    result = {
        "metric": METRIC, "value_definition": "grid points x bands of whole block-Davidson steps per second / 1e9",
        "value": K * nb * args.steps / elapsed / 1e9, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if esize == 8 else "f32",
        "data": "synthetic (seeded; bands from a seeded torch generator on the device)",
        "config": {"workload": "davidson: block-Davidson steps on gamma-96c-256b (2n = %d subspace)" % (2 * nb),
                   "grid": list(system.n), "bands": nb, "precision": args.precision,
                   "tc_scratch_mb": 2 * args.tc_scratch_mb, "parallelism": "single-gpu",
                   "l2": "inputs larger than L2 (%.2f GB of bands per step)" % (4 * nb * K * esize / 1e9)},
        "davidson_steps_per_s": args.steps / elapsed,
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
        "residual_norm": {"max_before": float(r_start.max()), "max_after": float(r_end.max()),
                          "median_before": float(r_start.median()), "median_after": float(r_end.median())},
        "lowest_ritz_value": float(eps[0]),
        "convergence": {"max_residual_per_step": history, "reduction_over_10_steps": history[0] / history[10],
                        "lowest_ritz_value_after_10": lowest_after_10,
                        "preconditioner": "kinetic -(T + 0.5 Ha)^-1 (FP32 FFT)"},
        "roofline": None, "gpu_launches": launches * args.steps, "clocks": clk, "cpu_baseline": cb,
    }
    print(json.dumps(result), flush=True)


# ------------------------------------------------------------------------------------------
# Density reductions after the eigensolver
# ------------------------------------------------------------------------------------------
def run_density(args):
    """The pseudo density (pawfd_density) and the atomic density matrices
    (pawfd_atomic_density) of the 96^3 x 256-band system's bands, occupations 2."""
    import torch

    from paper_2310_14776_gb300 import api

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = synth.WORKLOADS["gamma-96c-256b"]
    system = w.system()
    nb, K = (args.bands or w.nbands), system.npoints
    ctx = api.Context(system, max_bands=nb, device=dev, precision=args.precision)
    psi = device_bands(ctx, nb, w.seed)
    f = torch.full((nb,), 2.0, dtype=torch.float64, device=dev)
    rho = torch.empty(K, dtype=torch.float64, device=dev)
    P = ctx.project(psi)
    D = ctx.atomic_density(P, f)
    esize = psi.element_size()
    for _ in range(args.warmup):
        ctx.density(psi, f, rho=rho)
        ctx.atomic_density(P, f, D=D)
    ctx.sync()
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize(dev)
    l0 = ctx.launch_count()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps + 1)]
    evs[0].record()
    for i in range(args.steps):
        ctx.density(psi, f, rho=rho)
        evs[2 * i + 1].record()
        ctx.atomic_density(P, f, D=D)
        evs[2 * i + 2].record()
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ctx.sync()
    launches = ctx.launch_count() - l0
    elapsed = evs[0].elapsed_time(evs[-1]) * 1e-3
    dens_ms = [evs[2 * i].elapsed_time(evs[2 * i + 1]) for i in range(args.steps)]
    peaks = load_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    bytes_per_launch = nb * K * esize + K * 8
    achieved = bytes_per_launch / (np.mean(dens_ms) * 1e-3) / 1e9
    cb = None
    if not args.no_cpu_baseline:
        from oracle import oracle as O
        nb_s = 64
        psi_s = w.psi(system, nb=nb_s)
        t = time.perf_counter()
        O.density(system, psi_s, np.full(nb_s, 2.0))
        ts = time.perf_counter() - t
        cb = {"value": K * nb_s / ts / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle", "seconds": ts,
              "sample": "the oracle pseudo density of %d bands of the gamma-96c-256b system (numpy, one core)" % nb_s}
    result = {
        "metric": METRIC, "value_definition": "grid points x bands reduced into the pseudo density (plus the atomic "
                                              "density matrices) per second / 1e9",
        "value": K * nb * args.steps / elapsed / 1e9, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {8: "f64", 4: "f32"}[esize],
        "data": "synthetic (seeded; bands from a seeded torch generator on the device)",
        "config": {"workload": "density: pseudo density + atomic density matrices of gamma-96c-256b", "grid":
                   list(system.n), "bands": nb, "precision": args.precision, "parallelism": "single-gpu",
                   "l2": "inputs larger than L2 (%.2f GB of bands per step)" % (nb * K * esize / 1e9)},
        "latency_ms": {"p50": float(np.percentile(dens_ms, 50)), "p99": float(np.percentile(dens_ms, 99))},
        "roofline": {"stage": "pawfd_density", "kernel": "density_kernel", "bound": "hbm", "achieved": achieved,
                     "peak": hbm, "unit": "GB/s", "frac": achieved / hbm, "traffic": None,
                     "bytes_per_launch": bytes_per_launch, "peak_source": "MEASURED_PEAKS.json hbm_gbs"},
        "gpu_launches": launches, "clocks": clk, "cpu_baseline": cb,
    }
    print(json.dumps(result), flush=True)


# ------------------------------------------------------------------------------------------
# The Poisson solve (Hartree potential of the bands' density)
# ------------------------------------------------------------------------------------------
def run_poisson(args):
    """The Hartree potential of the pseudo density of the 96^3 x 256-band system's seeded bands
    (occupations 2): the direct Fourier route (pawfd_poisson_fft) timed with CUDA events, and
    the CG route (pawfd_poisson to 1e-11) host-timed beside it."""
    import torch

    from paper_2310_14776_gb300 import api

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = synth.WORKLOADS["gamma-96c-256b"]
    system = w.system()
    nb, K = (args.bands or w.nbands), system.npoints
    ctx = api.Context(system, max_bands=nb, device=dev, precision="fp64")
    psi = device_bands(ctx, nb, w.seed)
    rho = ctx.density(psi, torch.full((nb,), 2.0, dtype=torch.float64, device=dev))
    ctx.sync()
    del psi
    pctx = api.poisson_context(system, device=dev)
    v = torch.empty(K, dtype=torch.float64, device=dev)
    vcg = torch.empty(K, dtype=torch.float64, device=dev)
    work = torch.empty(K, dtype=torch.complex128, device=dev)
    # a buffer larger than L2, written between timed solves: rho, v and work (28 MB) would
    # otherwise stay in L2 from one solve to the next
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device=dev)
    tol, maxiter = 1e-11, 5000
    for _ in range(max(3, args.warmup)):
        pctx.poisson_fft(rho, v=v, work=work)
        pctx.poisson(rho, v=vcg, tol=tol, maxiter=maxiter)
    pctx.sync()
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize(dev)
    l0 = pctx.launch_count()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for e0, e1 in evs:
        flush.fill_(1)
        e0.record()
        pctx.poisson_fft(rho, v=v, work=work)
        e1.record()
    torch.cuda.synchronize(dev)
    launches = pctx.launch_count() - l0
    fft_ms = [e0.elapsed_time(e1) for e0, e1 in evs]
    times, iters = [], []
    for _ in range(args.steps):
        t = time.perf_counter()
        _, it, res = pctx.poisson(rho, v=vcg, tol=tol, maxiter=maxiter)
        torch.cuda.synchronize(dev)
        times.append(time.perf_counter() - t)
        iters.append(it)
    clk = clocks.stop()
    pctx.sync()
    # e2e: the density copied in from pinned host memory, the potential copied back
    rho_h = rho.cpu().pin_memory()
    v_h = torch.empty(K, dtype=torch.float64).pin_memory()
    rho_d = torch.empty_like(rho)
    torch.cuda.synchronize(dev)
    t = time.perf_counter()
    for _ in range(args.steps):
        rho_d.copy_(rho_h, non_blocking=True)
        pctx.poisson_fft(rho_d, v=v, work=work)
        v_h.copy_(v, non_blocking=True)
        torch.cuda.synchronize(dev)
    e2e_s = (time.perf_counter() - t) / args.steps
    vf = v.cpu().numpy()
    diff_cg = float(np.max(np.abs(vcg.cpu().numpy() - vf)) / np.max(np.abs(vf)))
    cb = None
    if not args.no_cpu_baseline:
        from oracle import oracle as O
        t = time.perf_counter()
        ref = O.poisson(synth.free_grid(system), rho.cpu().numpy()).reshape(-1)
        ts = time.perf_counter() - t
        cb = {"value": 1.0 / ts, "unit": "solves/s", "cores": 1, "kind": "oracle", "seconds": ts,
              "sample": "the oracle's direct Fourier solve of the same FD equation on the full 96^3 grid "
                        "(numpy FFT, one thread)",
              "max_rel_diff_gpu_fft": float(np.max(np.abs(vf - ref)) / np.max(np.abs(ref)))}
        # context: the same solve with a multithreaded FFT on every host core (scipy.fft
        # workers), the strongest CPU form of the direct route on this machine (not the oracle)
        try:
            import scipy.fft as sf
            rr = rho.cpu().numpy().reshape(system.n[2], system.n[1], system.n[0])
            fac = np.zeros(rr.shape)
            Lsym = O.laplacian_symbol(synth.free_grid(system))
            nz = Lsym != 0
            fac[nz] = -4.0 * np.pi / Lsym[nz]
            fac[0, 0, 0] = 0.0
            ncpu = os.cpu_count() or 1
            best = None
            for _ in range(3):
                t = time.perf_counter()
                sf.ifftn(sf.fftn(rr, workers=ncpu) * fac, workers=ncpu).real
                dt = time.perf_counter() - t
                best = dt if best is None else min(best, dt)
            cb["multithreaded_fft"] = {"seconds": best, "workers": ncpu,
                                       "what": "scipy.fft fftn / ifftn with all host cores, same FD symbol"}
        except ImportError:
            pass
    ms = float(np.mean(fft_ms))
    peaks = load_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    # algorithmic bytes: rho read once, v written once (8 B each per point)
    alg = 16 * K
    ach = alg / (ms * 1e-3) / 1e9
    result = {
        "metric": METRIC, "value_definition": "Poisson solves per second (the direct Fourier route on the order-6 "
                                              "FD Laplacian's symbol, 96^3 grid)",
        "value": 1e3 / ms, "unit": "solves/s", "n_gpus": 1, "steps": args.steps, "warmup": max(3, args.warmup),
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic (the pseudo density of seeded bands, occupations 2)",
        "config": {"workload": "poisson: Hartree potential of the gamma-96c-256b density", "grid": list(system.n),
                   "parallelism": "single-gpu",
                   "l2": "a 256 MB buffer written before each timed solve (rho, v, work: 28 MB)"},
        "latency_ms": {"p50": float(np.percentile(fft_ms, 50)), "p99": float(np.percentile(fft_ms, 99))},
        "cg": {"solves_per_s": args.steps / sum(times), "ms": sum(times) / args.steps * 1e3, "iterations": iters,
               "ms_per_iteration": sum(times) / max(1, sum(iters)) * 1e3, "tolerance": tol,
               "final_relative_residual": res, "max_rel_diff_to_fft": diff_cg,
               "note": "host-timed including the residual reads every 25 iterations"},
        "roofline": {"stage": "pawfd_poisson_fft", "kernel": "fft_pass_kernel (6 passes)", "bound": "hbm",
                     "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm, "traffic": None,
                     "bytes_per_solve": alg,
                     "note": "algorithmic bytes = rho in + v out; the 16 B/point work array of the six passes "
                             "stays in L2 (14 MB at 96^3)"},
        "gpu_launches": launches, "clocks": clk, "cpu_baseline": cb,
        "e2e": {"value": 1.0 / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": 8 * K, "d2h_bytes_per_step": 8 * K},
    }
    print(json.dumps(result), flush=True)


# ------------------------------------------------------------------------------------------
# H and S in the plane-wave representation
# ------------------------------------------------------------------------------------------
def run_pw(args):
    """pawfd_pw_apply_H + pawfd_pw_apply_S on the 96^3 grid (0.2 Angstrom spacing, 32 atoms x
    18 projectors) with 256 bands of complex coefficients at a Bloch vector, all G of the FFT
    grid (complex128, or complex64 with --precision mixed)."""
    import torch

    from paper_2310_14776_gb300 import api

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = synth.WORKLOADS["gamma-96c-256b"]
    base = w.system()
    L = base.cell
    kvec = (2 * np.pi * 0.25 / L[0], 2 * np.pi * 0.125 / L[1], 2 * np.pi * 0.375 / L[2])
    system = synth.build_system(base.n, base.cell, base.pos, base.wells, base.pset,
                                [base.dH[int(base.dmat_off[a]):int(base.dmat_off[a + 1])].reshape(18, 18)
                                 for a in range(base.natoms)],
                                [base.dS[int(base.dmat_off[a]):int(base.dmat_off[a + 1])].reshape(18, 18)
                                 for a in range(base.natoms)], k=kvec, complex_wf=True)
    nb, K = (args.bands or w.nbands), system.npoints
    ctx = api.Context(system, max_bands=nb, device=dev, precision=args.precision)
    C = device_bands(ctx, nb, w.seed)
    HC, SC = ctx.empty_bands(nb), ctx.empty_bands(nb)
    work = ctx.empty_bands(2 * nb)
    for _ in range(args.warmup):
        ctx.pw_apply(C, "H", out=HC, work=work)
        ctx.pw_apply(C, "S", out=SC, work=work)
    ctx.sync()
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize(dev)
    l0 = ctx.launch_count()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps + 1)]
    evs[0].record()
    for i in range(args.steps):
        ctx.pw_apply(C, "H", out=HC, work=work)
        evs[2 * i + 1].record()
        ctx.pw_apply(C, "S", out=SC, work=work)
        evs[2 * i + 2].record()
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ctx.sync()
    launches = ctx.launch_count() - l0
    elapsed = evs[0].elapsed_time(evs[-1]) * 1e-3
    h_ms = [evs[2 * i].elapsed_time(evs[2 * i + 1]) for i in range(args.steps)]
    s_ms = [evs[2 * i + 1].elapsed_time(evs[2 * i + 2]) for i in range(args.steps)]
    esize = C.element_size()
    peaks = load_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    # FFT passes per apply, each reading and writing every value once: three each way, or two
    # each way when x and y run as one pass per xy plane (FP32, both plane buffers within 200 KB
    # of shared memory)
    n1, n2 = int(system.n[0]), int(system.n[1])
    xy = esize == 8 and 8 * (n1 + n2 + 2 * n2 * (n1 + 1)) + 16 * n2 <= 200 * 1024
    passes = 4 if xy else 6
    fft_bytes = passes * 2 * esize * nb * K
    ach = fft_bytes / (np.mean(h_ms) * 1e-3) / 1e9
    result = {
        "metric": METRIC, "value_definition": "grid points x bands of plane-wave H C and S C per second / 1e9 "
                                              "(one H application and one S application per step)",
        "value": K * nb * args.steps / elapsed / 1e9, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64" if esize == 8 else "c128",
        "data": "synthetic (coefficients from a seeded torch generator on the device)",
        "config": {"workload": "pw: plane-wave H and S, 96^3 grid, 256 bands, Bloch k, all G",
                   "grid": list(system.n), "bands": nb, "precision": args.precision, "parallelism": "single-gpu",
                   "l2": "inputs larger than L2 (%.2f GB of coefficients)" % (nb * K * esize / 1e9)},
        "apply_H_ms": float(np.mean(h_ms)), "apply_S_ms": float(np.mean(s_ms)),
        "roofline": {"stage": "pawfd_pw_apply_H", "kernel": "fft_pass_kernel (%d passes) + project + back-add" % passes,
                     "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                     "traffic": None, "bytes_per_apply": fft_bytes,
                     "note": "bytes of the %d FFT passes (each reads and writes every value once) over the whole "
                             "H application time; FP64 butterflies run on the FP64 pipe" % passes},
        "gpu_launches": launches, "clocks": clk,
    }
    print(json.dumps(result), flush=True)


# ------------------------------------------------------------------------------------------
# CPU oracle baseline / reference arm
# ------------------------------------------------------------------------------------------
def oracle_step_time(system, psi, stages=None):
    """Seconds of one full oracle Rayleigh-Ritz step.  The step is made of the oracle's own
    calls in the order of its Rayleigh-Ritz step (H psi, S psi, the two Gram matrices, the
    subspace diagonalization, the rotation), each timed; `stages` (a dict) collects them."""
    from oracle import oracle as O
    t = {} if stages is None else stages

    def timed(name, f, *a):
        t0 = time.perf_counter()
        r = f(*a)
        t[name] = t.get(name, 0.0) + time.perf_counter() - t0
        return r
    nb = psi.shape[0]
    Hpsi, _ = timed("apply_H", O.apply_H, system, psi)
    Spsi, _ = timed("apply_S", O.apply_S, system, psi)
    Hnm = timed("gram_HS", O.gram, psi, Hpsi, system.dV, nb)
    Snm = timed("gram_HS", O.gram, psi, Spsi, system.dV, nb)
    _, C, _ = timed("subspace_diag", O.subspace_diag, Hnm, Snm)
    timed("rotate", O.rotate, psi, C)
    return sum(t[k] for k in ("apply_H", "apply_S", "gram_HS", "subspace_diag", "rotate"))


def oracle_small_one_thread():
    """Seconds of one oracle Rayleigh-Ritz step of the 24^3 x 16 workload on one host thread
    (OMP_NUM_THREADS=1 in a child process), or None if that run fails."""
    code = ("import sys, time; sys.path.insert(0, %r); import bench; from paper_2310_14776_gb300 import synth; "
            "w = synth.WORKLOADS['gamma-24c-16b']; s = w.system(); p = w.psi(s); bench.oracle_step_time(s, p); "
            "print(min(bench.oracle_step_time(s, p) for _ in range(3)))" % ROOT)
    try:
        r = subprocess.run([sys.executable, "-c", code], env=dict(os.environ, OMP_NUM_THREADS="1"),
                           capture_output=True, text=True, timeout=120)
        return float(r.stdout.strip().splitlines()[-1]) if r.returncode == 0 else None
    except (subprocess.TimeoutExpired, ValueError, IndexError):
        return None


def oracle_sample(system, w, precision, budget=2.3e8):
    """The bounded CPU sample of a workload: one full oracle Rayleigh-Ritz step on the first
    nb_s bands, nb_s = all bands when K * nb <= budget (2.3e8 is the 96^3 x 256 workload,
    about 20 s on 16 cores), else the most bands within the budget (at least 8)."""
    nb_s = w.nbands if system.npoints * w.nbands <= budget else max(8, int(budget // system.npoints))
    psi = w.psi(system, nb=nb_s)
    if precision == "mixed":
        psi = psi.astype(np.complex64 if system.complex_wf else np.float32)
    psi = psi.astype(np.complex128 if system.complex_wf else np.float64)
    return nb_s, psi


def cpu_baseline(system, w, precision):
    from oracle import oracle as O
    O.build()
    nb_s, psi = oracle_sample(system, w, precision)
    stages = {}
    t = oracle_step_time(system, psi, stages)
    t1 = oracle_small_one_thread()
    return {"value": system.npoints * nb_s / t / 1e9, "unit": UNIT, "cores": O.num_threads(),
            "kind": "oracle", "seconds": t, "stages_s": stages,
            "one_thread_24c_16b": {"seconds": t1, "value": 24 ** 3 * 16 / t1 / 1e9 if t1 else None,
                                   "how": "best of 3 oracle RR steps of the 24^3 x 16 workload, OMP_NUM_THREADS=1"},
            "sample": "one full FP64 Rayleigh-Ritz step (apply_H, apply_S, two Gram matrices, subspace diag, "
                      "rotation) of the %s workload on %d of its %d bands, on the host cores"
                      % (w.name, nb_s, w.nbands)}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    if args.workload not in synth.WORKLOADS:
        print(json.dumps({"impl": "reference", "unavailable": "the oracle arm covers the single-system workloads; "
                          "%s is timed against sequential plain FP64 on the GPU inside its own line"
                          % args.workload}), flush=True)
        return
    w = synth.WORKLOADS[args.workload]
    system = w.system()
    # each reference step is a bounded sample (about 4 s on 16 cores at 96^3) so that the
    # driver's warm-up + timed steps end within a few minutes
    nb_s, psi = oracle_sample(system, w, args.precision, budget=5e7)
    for _ in range(args.warmup):
        oracle_step_time(system, psi)
    times = [oracle_step_time(system, psi) for _ in range(args.steps)]
    el = sum(times)
    value = system.npoints * nb_s * args.steps / el / 1e9
    sample = ("one full FP64 Rayleigh-Ritz step of the %s workload on %d of its %d bands per step"
              % (w.name, nb_s, w.nbands))
    cb = {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle", "sample": sample}
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value_definition": VALUE_DEF,
        "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c128" if system.complex_wf else "f64", "data": "synthetic (seeded)",
        "config": {"workload": w.name, "grid": list(system.n), "bands": w.nbands, "atoms": system.natoms,
                   "projectors_per_atom": int(system.nproj[0]) if system.natoms else 0,
                   "precision": args.precision, "parallelism": "single-gpu"},
        "cpu_baseline": cb, "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                                    "d2h_bytes_per_step": 0}}), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch64":
        run_batch(args)
    elif args.workload in ("served", "davidson", "density", "poisson", "pw"):
        if single_gpu_arm(args.workload):
            {"served": run_served, "davidson": run_davidson, "density": run_density,
             "poisson": run_poisson, "pw": run_pw}[args.workload](args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
