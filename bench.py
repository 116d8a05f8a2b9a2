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

FP64_NOMINAL_TFLOPS = 1.25   # GB300 FP64 (vector and tensor), nominal
FP32_PROBE_TFLOPS = 70.1     # GB300 FP32 FMA rate measured by a DFMA/FFMA probe kernel on this machine


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="pawfd", choices=["pawfd", "reference"])
    p.add_argument("--workload", default="gamma-96c-256b", choices=sorted(synth.WORKLOADS))
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    return p.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


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
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.out,
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
    nb, K = w.nbands, system.npoints
    psi_host = w.psi(system)
    cplx = system.complex_wf
    if args.precision == "mixed":
        psi_host = psi_host.astype(np.complex64 if cplx else np.float32)
    ctx = api.Context(system, max_bands=nb, device=dev, precision=args.precision)
    psi = [torch.from_numpy(psi_host).to(dev), torch.empty_like(torch.from_numpy(psi_host), device=dev)]
    work = {"Hpsi": ctx.empty_bands(nb), "Spsi": ctx.empty_bands(nb),
            "Hnm": torch.empty((nb, nb), dtype=ctx.mat_dtype, device=dev),
            "Snm": torch.empty((nb, nb), dtype=ctx.mat_dtype, device=dev),
            "eps": torch.empty(nb, dtype=torch.float64, device=dev),
            "C": torch.empty((nb, nb), dtype=ctx.mat_dtype, device=dev)}
    stream = torch.cuda.current_stream(dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def step(cur, nxt, marks=None):
        # marks: events between the stages apply_H | apply_S | Gram H | Gram S | subspace | rotate
        def mark(i):
            if marks is not None:
                marks[i].record(stream)
        mark(0)
        ctx.apply_H(cur, out=work["Hpsi"])
        mark(1)
        ctx.apply_S(cur, out=work["Spsi"])
        mark(2)
        ctx.gram(cur, work["Hpsi"], M=work["Hnm"], hermitian=True)
        mark(3)
        ctx.gram(cur, work["Spsi"], M=work["Snm"], hermitian=True)
        mark(4)
        ctx.subspace_diag(work["Hnm"], work["Snm"], eps=work["eps"], C=work["C"], overwrite=True, check=False)
        mark(5)
        ctx.rotate(cur, work["C"], out=nxt)
        mark(6)

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
    marks = [[ev() for _ in range(7)] for _ in range(args.steps)]
    t0, t1 = ev(), ev()
    t0.record(stream)
    for i in range(args.steps):
        step(psi[(args.warmup + i) % 2], psi[(args.warmup + i + 1) % 2], marks[i])
    t1.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ctx.sync()
    launches = ctx.launch_count() - launches0
    elapsed = t0.elapsed_time(t1) * 1e-3
    if world > 1:
        tt = torch.tensor([elapsed], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        elapsed = tt.item()
    step_ms = [m[0].elapsed_time(m[6]) for m in marks]
    names = ["apply_H", "apply_S", "gram_H", "gram_S", "subspace_diag", "rotate"]
    stages = {nm: statistics.mean(m[i].elapsed_time(m[i + 1]) for m in marks) for i, nm in enumerate(names)}
    drift = float(torch.max(torch.abs(work["eps"] - eps_first)).item())

    units = float(nb) * K * args.steps * world
    value = units / elapsed / 1e9
    esize = psi_host.itemsize
    mixed = args.precision == "mixed"
    peaks = load_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    bf16 = peaks.get("bf16_tflops", 1900.0)
    # digit products per real multiply-add of the tensor-core kernels (orders <= 6 of 7 digits
    # for FP64 data, <= 4 of 4 digits for FP32 data) and real multiply-adds per complex one
    products = 13 if mixed else 28
    cfac = 4 if cplx else 1
    # algorithmic work per stage (see the roofline table of the design notes)
    work_units = {
        # FP64: 19 FP64 instructions per point-band (9 add, 9 FMA, 1 mul), vs the FP64 issue rate
        "apply_H": ("alu", 19.0 * nb * K * (2 if cplx else 1), FP64_NOMINAL_TFLOPS / 2 * 1e12, "FP64 instr/s")
        if not mixed else ("hbm", 2.0 * esize * nb * K, hbm * 1e9, "B/s"),
        "gram_H": ("tensor", 2.0 * products * cfac * nb * (nb + 1) / 2 * K, bf16 * 1e12, "BF16 FLOP/s"),
        "gram_S": ("tensor", 2.0 * products * cfac * nb * (nb + 1) / 2 * K, bf16 * 1e12, "BF16 FLOP/s"),
        "rotate": ("tensor", 2.0 * products * cfac * nb * nb * K, bf16 * 1e12, "BF16 FLOP/s"),
    }
    dom = max((k for k in stages if k in work_units), key=lambda k: stages[k])
    bound, amount, peak, unit = work_units[dom]
    achieved = amount / (stages[dom] * 1e-3)
    kernel_of = {"apply_H": "kinetic_local_kernel + project_kernel + nonlocal_add_kernel",
                 "gram_H": "slice_kernel + sliced_gram_kernel (digit-product Gram)",
                 "gram_S": "slice_kernel + sliced_gram_kernel (digit-product Gram)",
                 "rotate": "slice_t_kernel + sliced_gram_kernel (digit-product rotation)"}
    scale = 1e12 if unit.endswith("FLOP/s") or unit == "FP64 instr/s" else 1e9
    roof_unit = {"BF16 FLOP/s": "TFLOP/s", "FP64 instr/s": "Tinstr/s", "B/s": "GB/s"}[unit]

    result = {
        "metric": "H|psi> Gpt.band/s over whole Rayleigh-Ritz steps (apply_H + apply_S + Gram + subspace diag + rotate)",
        "value": value, "unit": "Gpt.band/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {8: "f64", 16: "c128", 4: "f32"}[esize] if not (mixed and cplx) else "c64",
        "data": "synthetic (seeded)",
        "config": {"workload": w.name, "grid": list(system.n), "bands": nb, "atoms": system.natoms,
                   "projectors_per_atom": int(system.nproj[0]) if system.natoms else 0,
                   "precision": args.precision, "parallelism": "replicas" if world > 1 else "single-gpu",
                   "l2": "inputs larger than L2 (%.2f GB of bands per step)" % (2 * nb * K * esize / 1e9)},
        "rr_steps_per_s": args.steps * world / elapsed,
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
        "stages_ms": stages,
        "apply_H_gptband_s": nb * K / (stages["apply_H"] * 1e-3) / 1e9,
        "eig_drift_ha": drift,
        "roofline": {"stage": dom, "kernel": kernel_of[dom], "bound": bound, "achieved": achieved / scale,
                     "peak": peak / scale, "unit": roof_unit, "frac": achieved / peak, "traffic": None,
                     "peak_source": {"tensor": "MEASURED_PEAKS.json bf16_tflops (burst)",
                                     "hbm": "MEASURED_PEAKS.json hbm_gbs",
                                     "alu": "nominal GB300 FP64 rate 1.25 TFLOP/s / 2 (FMA)"}[bound]},
        "gpu_launches": int(launches),
        "clocks": clk,
    }

    if not args.no_e2e:
        result["e2e"] = e2e_gpu(ctx, psi_host, work, args, dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(system, psi_host, w)
    if world > 1:
        dist.barrier()
    ctx.close()
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        dist.destroy_process_group()


def e2e_gpu(ctx, psi_host, work, args, dev):
    """Same step through the public API with host buffers: H2D of psi and D2H of eps + rotated bands."""
    import torch
    nb = psi_host.shape[0]
    h_in = torch.from_numpy(psi_host).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    h_eps = torch.empty(nb, dtype=torch.float64).pin_memory()
    d_in = torch.empty_like(h_in, device=dev)
    d_out = torch.empty_like(h_in, device=dev)
    stream = torch.cuda.current_stream(dev)

    def one():
        d_in.copy_(h_in, non_blocking=True)
        ctx.apply_H(d_in, out=work["Hpsi"])
        ctx.apply_S(d_in, out=work["Spsi"])
        ctx.gram(d_in, work["Hpsi"], M=work["Hnm"], hermitian=True)
        ctx.gram(d_in, work["Spsi"], M=work["Snm"], hermitian=True)
        ctx.subspace_diag(work["Hnm"], work["Snm"], eps=work["eps"], C=work["C"], overwrite=True, check=False)
        ctx.rotate(d_in, work["C"], out=d_out)
        h_eps.copy_(work["eps"], non_blocking=True)
        h_out.copy_(d_out, non_blocking=True)

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
    per_step_bytes = h_in.numel() * h_in.element_size()
    return {"value": nb * K * args.e2e_steps / el / 1e9, "unit": "Gpt.band/s", "steps": args.e2e_steps,
            "h2d_bytes_per_step": per_step_bytes, "d2h_bytes_per_step": per_step_bytes + nb * 8}


# ------------------------------------------------------------------------------------------
# CPU oracle baseline / reference arm
# ------------------------------------------------------------------------------------------
def oracle_step_time(system, psi):
    from oracle import oracle as O
    t = time.perf_counter()
    O.rayleigh_ritz(system, psi)
    return time.perf_counter() - t


def cpu_baseline(system, psi, w):
    from oracle import oracle as O
    O.build()
    t = oracle_step_time(system, psi)
    return {"value": system.npoints * w.nbands / t / 1e9, "unit": "Gpt.band/s", "cores": O.num_threads(),
            "kind": "oracle", "seconds": t,
            "sample": "one full Rayleigh-Ritz step of the %s workload (apply_H, apply_S, two Gram matrices, "
                      "subspace diag, rotation) on the host cores" % w.name}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    w = synth.WORKLOADS[args.workload]
    system = w.system()
    psi = w.psi(system)
    for _ in range(args.warmup):
        oracle_step_time(system, psi)
    times = [oracle_step_time(system, psi) for _ in range(args.steps)]
    el = sum(times)
    value = system.npoints * w.nbands * args.steps / el / 1e9
    cb = {"value": value, "unit": "Gpt.band/s", "cores": O.num_threads(), "kind": "oracle",
          "sample": "one full Rayleigh-Ritz step of the %s workload per step" % w.name}
    print(json.dumps({
        "impl": "reference", "metric": "H|psi> Gpt.band/s over whole Rayleigh-Ritz steps (apply_H + apply_S + "
                                       "Gram + subspace diag + rotate)",
        "value": value, "unit": "Gpt.band/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c128" if system.complex_wf else "f64", "data": "synthetic (seeded)",
        "config": {"workload": w.name, "grid": list(system.n), "bands": w.nbands, "atoms": system.natoms,
                   "precision": "fp64"},
        "cpu_baseline": cb, "e2e": {"value": value, "unit": "Gpt.band/s", "h2d_bytes_per_step": 0,
                                    "d2h_bytes_per_step": 0}}), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
