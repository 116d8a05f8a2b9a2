"""Served form: a continuous-batching request loop for eigensolver jobs on one GPU.

Jobs arrive as a seeded Poisson stream.  Each names a system (grid, bands, atoms, Bloch
vector) from a seeded catalogue and runs a fixed number of Rayleigh-Ritz iterations.  Its
bands, projections and subspace matrices stay resident on the device for its whole life.
The loop admits a waiting job as soon as a slot and enough of the HBM budget are free
(first fit over the head of the queue).  Every admitted job runs on a CUDA stream of its own,
so its kernels overlap with those of all other jobs on the GPU.  A finished job's arrays
return to the budget at once, and its context goes back to a pool for the next job of the
same system; idle contexts are evicted when memory is short.

``Scheduler`` is the host-side bookkeeping (queue, budget, admission, retirement) and needs
no GPU.  ``Server`` drives it with the library's contexts.
"""
from __future__ import annotations

import collections
import dataclasses
import time
from typing import Callable, Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import synth


# ------------------------------------------------------------------------------------------
# jobs and the catalogue of systems
# ------------------------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class Job:
    job_id: int
    arrival: float          # seconds after the start of the stream
    system: int             # index into the catalogue
    psi_seed: int


def catalogue(n_small: int = 64, n_large: int = 8, complex_wf: bool = True, seed0: int = 4,
              large=((128, 128, 128), 512, 24)) -> List[synth.Instance]:
    """The systems jobs draw from: n_small sized as batched instances, then n_large large ones."""
    small = [synth.batch_instance(seed0 + i, complex_wf) for i in range(n_small)]
    out = list(small)
    for i in range(n_large):
        seed = seed0 + 100000 + i
        k = (0.0, 0.0, 0.0)
        if complex_wf:
            uk = synth.uniform01(seed, synth.STREAM_KPT, 0, 3)
            k = tuple(float(uk[c] * np.pi / (large[0][c] * synth.H_02A)) for c in range(3))
        out.append(synth.Instance(tuple(large[0]), large[1], large[2], seed, complex_wf, k))
    return out


def job_stream(rate: float, duration: float, n_small: int, n_large: int, large_fraction: float = 0.1,
               seed: int = 4) -> List[Job]:
    """Poisson arrivals at `rate` per second for `duration` seconds.  With probability
    `large_fraction` a job draws one of the large systems, otherwise one of the small ones
    (uniformly); its bands are seeded by its id."""
    count = max(1, int(rate * duration * 1.5) + 16)
    t = synth.poisson_arrivals(rate, count, seed)
    t = t[t <= duration]
    u = synth.uniform01(seed, synth.STREAM_SIZES, 1 << 24, 2 * len(t)).reshape(-1, 2)
    jobs = []
    for j, (ta, (ul, us)) in enumerate(zip(t, u)):
        if n_large and ul < large_fraction:
            sysid = n_small + min(n_large - 1, int(us * n_large))
        else:
            sysid = min(n_small - 1, int(us * n_small))
        jobs.append(Job(j, float(ta), sysid, seed * 1000003 + j))
    return jobs


def array_bytes(inst: synth.Instance, precision: str) -> int:
    """Device bytes of one job's own arrays: two band blocks (ping-pong), H psi, S psi, and
    the six nb x nb / nb-sized matrices and vectors of a step."""
    esize = {("mixed", False): 4, ("mixed", True): 8, ("fp64", False): 8, ("fp64", True): 16}[
        (precision, inst.complex_wf)]
    msize = 16 if inst.complex_wf else 8
    nb = inst.nbands
    return 4 * inst.npoints * nb * esize + 3 * nb * nb * msize + nb * 8


# ------------------------------------------------------------------------------------------
# host-side scheduling (no GPU)
# ------------------------------------------------------------------------------------------

class Scheduler:
    """Queue + HBM budget + first-fit admission.  `need(job)` gives the bytes a job would
    take if admitted now (its arrays, plus a context unless an idle one is pooled)."""

    def __init__(self, budget: int, max_active: int, lookahead: int = 16):
        self.budget = int(budget)
        self.used = 0
        self.max_active = max_active
        self.lookahead = lookahead
        self.queue: collections.deque = collections.deque()
        self.active: Dict[int, int] = {}      # job id -> bytes held
        self.peak_used = 0
        self.max_queue = 0
        self.overruns = 0

    def arrive(self, job: Job):
        self.queue.append(job)
        self.max_queue = max(self.max_queue, len(self.queue))

    def free_bytes(self) -> int:
        return self.budget - self.used

    def pick(self, need: Callable[[Job], int], reclaim: Callable[[int], int]) -> Optional[Job]:
        """The first of the first `lookahead` waiting jobs that fits (after reclaiming idle
        memory through `reclaim(bytes_short)`, which returns the bytes it freed), or None."""
        if len(self.active) >= self.max_active:
            return None
        for i, job in enumerate(list(self.queue)[: self.lookahead]):
            b = need(job)
            if b > self.budget:
                continue                   # can never run under this budget
            if b > self.free_bytes():
                self.used -= reclaim(b - self.free_bytes())
            if b <= self.free_bytes():
                del self.queue[i]
                return job
        return None

    def admit(self, job: Job, nbytes: int):
        self.active[job.job_id] = nbytes
        self.used += nbytes
        self.peak_used = max(self.peak_used, self.used)
        if self.used > self.budget:
            # a context measured larger than its estimate: counted, and the estimate is
            # corrected for the next job of that system
            self.overruns += 1

    def retire(self, job: Job, keep: int = 0):
        """Release a finished job; `keep` bytes stay charged (its pooled context)."""
        self.used -= self.active.pop(job.job_id) - keep

    def release(self, nbytes: int):
        self.used -= nbytes


# ------------------------------------------------------------------------------------------
# GPU executor
# ------------------------------------------------------------------------------------------

@dataclasses.dataclass
class JobRecord:
    job: Job
    admitted: float = 0.0
    finished: float = 0.0
    eps: Optional[np.ndarray] = None


class Server:
    """Runs a job stream on one GPU with the library's contexts (see the module docstring)."""

    def __init__(self, systems: Sequence[synth.Instance], device, precision: str = "mixed",
                 iterations: int = 5, budget_fraction: float = 0.8, budget_bytes: Optional[int] = None,
                 max_active: int = 48, tune: bool = True):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.systems = list(systems)
        self.precision = precision
        self.iterations = iterations
        self.tune = tune
        free, _ = torch.cuda.mem_get_info(self.device)
        budget = int(budget_fraction * free) if budget_bytes is None else int(budget_bytes)
        self.sched = Scheduler(budget, max_active)
        self._sys_cache: Dict[int, object] = {}
        self.pool: Dict[int, List[Tuple[object, int]]] = collections.defaultdict(list)   # idle (ctx, bytes)
        self.ctx_bytes: Dict[int, int] = {}                     # measured per system
        self.idle_lru: collections.OrderedDict = collections.OrderedDict()

    # -- systems and contexts ----------------------------------------------------------
    def system(self, sysid: int):
        if sysid not in self._sys_cache:
            self._sys_cache[sysid] = self.systems[sysid].system()
        return self._sys_cache[sysid]

    def prepare(self, sysids: Sequence[int], contexts: bool = True):
        """Ahead of the stream (not part of any job's latency): build the host-side systems
        and, with `contexts`, one pooled context per system, tuned for its shape, while the
        budget allows (smallest first)."""
        torch = self.torch
        for s in sysids:
            self.system(s)
        if not contexts:
            return
        for s in sorted(sysids, key=lambda i: array_bytes(self.systems[i], self.precision)):
            inst = self.systems[s]
            if self._ctx_estimate(s) + array_bytes(inst, self.precision) > self.sched.free_bytes():
                continue
            ctx, cbytes, _ = self._get_ctx(s)
            if self.tune:
                from . import autotune
                psi = self._bands(inst, inst.seed, torch.cuda.current_stream(self.device))
                work = ctx.alloc_work(inst.nbands)
                work["C"].copy_(torch.eye(inst.nbands, dtype=work["C"].dtype, device=self.device))
                autotune.tune(ctx, psi, work)
                del psi, work
            self.pool[s].append((ctx, cbytes))
            self.idle_lru[(s, id(ctx))] = True
            self.sched.used += cbytes
        torch.cuda.synchronize(self.device)
        torch.cuda.empty_cache()

    def _ctx_estimate(self, sysid: int) -> int:
        if sysid in self.ctx_bytes:
            return self.ctx_bytes[sysid]
        inst = self.systems[sysid]
        nb = inst.nbands
        return (320 << 20) + 24 * nb * nb * 16 + 2 * inst.npoints * 8

    def need(self, job: Job) -> int:
        inst = self.systems[job.system]
        b = array_bytes(inst, self.precision)
        if not self.pool[job.system]:
            b += self._ctx_estimate(job.system)
        return b

    def reclaim(self, short: int) -> int:
        freed = 0
        while freed < short and self.idle_lru:
            key, _ = self.idle_lru.popitem(last=False)
            sysid, idx = key
            lst = self.pool[sysid]
            for i, (ctx, nbytes) in enumerate(lst):
                if id(ctx) == idx:
                    ctx.close()
                    del lst[i]
                    freed += nbytes
                    break
        return freed

    def _get_ctx(self, sysid: int):
        from . import api
        torch = self.torch
        if self.pool[sysid]:
            ctx, nbytes = self.pool[sysid].pop()
            self.idle_lru.pop((sysid, id(ctx)), None)
            return ctx, nbytes, False
        inst = self.systems[sysid]
        f0, _ = torch.cuda.mem_get_info(self.device)
        try:
            ctx = api.Context(self.system(sysid), max_bands=inst.nbands, device=self.device, precision=self.precision)
        except api.PawFDError:
            # the library allocates with cudaMalloc: give back what torch's cache holds, once
            torch.cuda.empty_cache()
            f0, _ = torch.cuda.mem_get_info(self.device)
            ctx = api.Context(self.system(sysid), max_bands=inst.nbands, device=self.device, precision=self.precision)
        f1, _ = torch.cuda.mem_get_info(self.device)
        nbytes = max(0, f0 - f1)
        self.ctx_bytes[sysid] = max(nbytes, self.ctx_bytes.get(sysid, 0))
        return ctx, nbytes, True

    # -- one job ------------------------------------------------------------------------
    def _bands(self, inst, seed, gen_stream):
        torch = self.torch
        g = torch.Generator(device=self.device)
        g.manual_seed(int(seed))
        shape = (inst.nbands,) + tuple(inst.n[::-1])
        rdt = torch.float32 if self.precision == "mixed" else torch.float64
        with torch.cuda.stream(gen_stream):
            re = torch.rand(shape, generator=g, device=self.device, dtype=rdt) * 2 - 1
            if inst.complex_wf:
                im = torch.rand(shape, generator=g, device=self.device, dtype=rdt) * 2 - 1
                return torch.complex(re, im)
            return re

    def start(self, job: Job, now: float):
        torch = self.torch
        inst = self.systems[job.system]
        ctx, cbytes, fresh = self._get_ctx(job.system)
        stream = torch.cuda.Stream(self.device)
        with torch.cuda.stream(stream):
            psi = self._bands(inst, job.psi_seed, stream)
            out = torch.empty_like(psi)
            work = ctx.alloc_work(inst.nbands)
            if self.tune:
                from . import autotune
                if autotune.shape_key(ctx, inst.nbands) not in autotune._CACHE:
                    work["C"].copy_(torch.eye(inst.nbands, dtype=work["C"].dtype, device=self.device))
                autotune.tune(ctx, psi, work)
            bufs = [psi, out]
            for it in range(self.iterations):
                ctx.rr_step(bufs[it % 2], out=bufs[(it + 1) % 2], work=work)
            done = torch.cuda.Event()
            done.record(stream)
        nbytes = array_bytes(inst, self.precision) + (cbytes if fresh else 0)
        state = dict(job=job, ctx=ctx, cbytes=cbytes, fresh=fresh, stream=stream, done=done, bufs=bufs, work=work,
                     rec=JobRecord(job, admitted=now), nbytes=nbytes)
        return state, nbytes

    def finish(self, state, now: float) -> JobRecord:
        rec = state["rec"]
        with self.torch.cuda.stream(state["stream"]):
            rec.eps = state["work"]["eps"].cpu().numpy()
        state["ctx"].sync()
        rec.finished = now
        sysid = state["job"].system
        self.pool[sysid].append((state["ctx"], state["cbytes"]))
        self.idle_lru[(sysid, id(state["ctx"]))] = True
        return rec

    # -- the loop -------------------------------------------------------------------------
    def run(self, jobs: Sequence[Job], duration: Optional[float] = None, poll_s: float = 2e-4,
            clock: Callable[[], float] = time.perf_counter) -> Dict:
        """Serve `jobs` (sorted by arrival) in real time.  Stops when every job has finished,
        or at `duration` seconds (unfinished jobs are counted, not waited for)."""
        pending = collections.deque(sorted(jobs, key=lambda j: j.arrival))
        active: Dict[int, dict] = {}
        done: List[JobRecord] = []
        t0 = clock()
        while pending or self.sched.queue or active:
            now = clock() - t0
            if duration is not None and now >= duration:
                break
            progressed = False
            while pending and pending[0].arrival <= now:
                self.sched.arrive(pending.popleft())
            for jid in list(active):
                st = active[jid]
                if st["done"].query():
                    rec = self.finish(st, clock() - t0)
                    done.append(rec)
                    # the job's arrays are released; a context it created stays charged while pooled
                    self.sched.retire(st["job"], keep=st["cbytes"] if st["fresh"] else 0)
                    del active[jid]
                    progressed = True
            while True:
                job = self.sched.pick(self.need, self.reclaim)
                if job is None:
                    break
                st, nbytes = self.start(job, clock() - t0)
                self.sched.admit(job, nbytes)
                active[job.job_id] = st
                progressed = True
            if not progressed:
                nxt = pending[0].arrival - (clock() - t0) if pending else poll_s
                time.sleep(max(0.0, min(poll_s, nxt)))
        elapsed = clock() - t0
        return {"records": done, "elapsed": elapsed, "unfinished": len(active) + len(self.sched.queue) + len(pending),
                "active_at_end": len(active), "queued_at_end": len(self.sched.queue), "peak_used": self.sched.peak_used,
                "budget": self.sched.budget, "max_queue": self.sched.max_queue, "overruns": self.sched.overruns}

    def close(self):
        for lst in self.pool.values():
            for ctx, _ in lst:
                ctx.close()
        self.pool.clear()
        self.idle_lru.clear()


def latency_stats(records: Sequence[JobRecord], warmup: float = 0.0) -> Dict:
    """p50 / p99 latency (arrival to finish) over jobs that arrived after `warmup` seconds."""
    lat = [r.finished - r.job.arrival for r in records if r.job.arrival >= warmup]
    if not lat:
        return {"jobs": 0}
    return {"jobs": len(lat), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(np.mean(lat) * 1e3)}
