"""Served form: a continuous-batching request loop for eigensolver jobs on one GPU.

Jobs arrive as a seeded Poisson stream.  Each names a system (grid, bands, atoms, Bloch
vector) from a seeded catalogue and runs a fixed number of Rayleigh-Ritz iterations.  Its
bands, projections and subspace matrices stay resident on the device for its whole life.
The loop admits a waiting job as soon as a slot and enough of the HBM budget are free
(first fit over the head of the queue).  Every admitted job runs on a CUDA stream of its own,
so its kernels overlap with those of all other jobs on the GPU.  A finished job's arrays
return to the budget at once, and its context goes back to a pool for the next job of the
same system; idle contexts are evicted when memory is short.

Memory is held to the budget by construction.  The budget is split in two:
  * an arena: one device allocation made once, from which every job's arrays are carved by
    a host-side first-fit allocator (``Arena``) and returned when the job ends, so the loop
    makes no device allocation per job and the caching allocator's blocks do not pile up;
  * the contexts (the library allocates their tables and scratch itself): each is charged at
    its measured size (the drop in free device memory when it was created, known for every
    system after its first context) before a job that needs a new one is admitted, and idle
    pooled contexts are evicted, least recently used first, to make room.

``Scheduler`` is the host-side bookkeeping (queue, budget, admission, retirement) and needs
no GPU, nor does ``Arena``.  ``Server`` drives them with the library's contexts.
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

    def pick_with(self, try_start: Callable[[Job], object]) -> Optional[Tuple[Job, object]]:
        """First fit with a caller-side test: the first of the first `lookahead` waiting jobs
        for which `try_start(job)` returns something other than None (it reserves whatever
        the job needs), removed from the queue; None if no slot is free or nothing fits."""
        if len(self.active) >= self.max_active:
            return None
        for i, job in enumerate(list(self.queue)[: self.lookahead]):
            r = try_start(job)
            if r is not None:
                del self.queue[i]
                return job, r
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


class Arena:
    """First-fit allocation of byte ranges of [0, size), each starting at a multiple of
    `align`; a freed range merges with free neighbours.  Host bookkeeping only: the device
    memory is one buffer that the server allocates once."""

    def __init__(self, size: int, align: int = 256):
        self.align = int(align)
        self.size = int(size) // self.align * self.align
        self.free_ranges: List[Tuple[int, int]] = [(0, self.size)] if self.size > 0 else []   # sorted (offset, length)
        self.used = 0
        self.peak = 0

    def _round(self, nbytes: int) -> int:
        return max(self.align, (int(nbytes) + self.align - 1) // self.align * self.align)

    def alloc(self, nbytes: int) -> Optional[int]:
        n = self._round(nbytes)
        for i, (off, ln) in enumerate(self.free_ranges):
            if ln >= n:
                if ln == n:
                    del self.free_ranges[i]
                else:
                    self.free_ranges[i] = (off + n, ln - n)
                self.used += n
                self.peak = max(self.peak, self.used)
                return off
        return None

    def free(self, off: int, nbytes: int):
        n = self._round(nbytes)
        i = 0
        while i < len(self.free_ranges) and self.free_ranges[i][0] < off:
            i += 1
        self.free_ranges.insert(i, (off, n))
        # merge with the following range, then with the preceding one
        if i + 1 < len(self.free_ranges) and off + n == self.free_ranges[i + 1][0]:
            self.free_ranges[i] = (off, n + self.free_ranges[i + 1][1])
            del self.free_ranges[i + 1]
        if i > 0 and self.free_ranges[i - 1][0] + self.free_ranges[i - 1][1] == off:
            self.free_ranges[i - 1] = (self.free_ranges[i - 1][0], self.free_ranges[i - 1][1] + self.free_ranges[i][1])
            del self.free_ranges[i]
        self.used -= n

    def alloc_all(self, sizes: Sequence[int]) -> Optional[List[int]]:
        """Offsets for every size, or None (and nothing held) if one does not fit."""
        offs: List[int] = []
        for nb in sizes:
            off = self.alloc(nb)
            if off is None:
                for o, n in zip(offs, sizes):
                    self.free(o, n)
                return None
            offs.append(off)
        return offs


# ------------------------------------------------------------------------------------------
# GPU executor
# ------------------------------------------------------------------------------------------

@dataclasses.dataclass
class JobRecord:
    job: Job
    admitted: float = 0.0
    finished: float = 0.0
    eps: Optional[np.ndarray] = None


def job_array_sizes(inst: synth.Instance, precision: str) -> List[int]:
    """Byte sizes of one job's arrays, in the order the server carves them: the two band
    blocks (ping-pong), H psi, S psi, then Hnm, Snm, C and eps (their sum is array_bytes)."""
    esize = {("mixed", False): 4, ("mixed", True): 8, ("fp64", False): 8, ("fp64", True): 16}[
        (precision, inst.complex_wf)]
    msize = 16 if inst.complex_wf else 8
    nb = inst.nbands
    band = inst.npoints * nb * esize
    return [band] * 4 + [nb * nb * msize] * 3 + [nb * 8]


class Server:
    """Runs a job stream on one GPU with the library's contexts (see the module docstring).

    budget: `budget_bytes`, or `budget_fraction` of the free device memory at construction.
    After ``prepare`` (contexts of the stream's systems made ahead) the arena takes what the
    contexts leave, less `ctx_reserve_fraction` of the budget kept for contexts made during
    the run; without it, the arena takes `arena_fraction` of the budget at the first run."""

    def __init__(self, systems: Sequence[synth.Instance], device, precision: str = "mixed",
                 iterations: int = 5, budget_fraction: float = 0.8, budget_bytes: Optional[int] = None,
                 max_active: int = 48, tune: bool = True, arena_fraction: float = 0.5,
                 ctx_reserve_fraction: float = 0.1):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.systems = list(systems)
        self.precision = precision
        self.iterations = iterations
        self.kernel_launches = 0
        self.tune = tune
        free, _ = torch.cuda.mem_get_info(self.device)
        self.free_at_start = free
        self.min_free = free
        budget = int(budget_fraction * free) if budget_bytes is None else int(budget_bytes)
        self.sched = Scheduler(budget, max_active)
        self.arena_fraction = arena_fraction
        self.ctx_reserve_fraction = ctx_reserve_fraction
        self.arena: Optional[Arena] = None
        self.mem = None                                          # the arena's device buffer
        self.ctx_used = 0                                        # measured bytes of live contexts
        self._sys_cache: Dict[int, object] = {}
        self.pool: Dict[int, List[Tuple[object, int]]] = collections.defaultdict(list)   # idle (ctx, bytes)
        self.ctx_bytes: Dict[int, int] = {}                     # measured per system
        self.idle_lru: collections.OrderedDict = collections.OrderedDict()
        # one CUDA stream per slot, made once (a stream per job would leave device resources
        # behind for every job served)
        self.streams = [torch.cuda.Stream(self.device) for _ in range(max_active)]
        self.free_streams = list(range(max_active))

    # -- budget ---------------------------------------------------------------------------
    def margin(self) -> int:
        """Device bytes of the budget left out of the arena and the contexts' share: what the
        library and the runtime allocate outside them (the contexts' auxiliary streams and
        events, allocations a context makes on first use, torch's small buffers)."""
        return int(0.02 * self.sched.budget)

    def ctx_cap(self) -> int:
        """Bytes the contexts may hold: the budget less the arena and the margin."""
        return self.sched.budget - (self.arena.size if self.arena is not None else 0) - self.margin()

    def _account(self):
        used = self.ctx_used + (self.arena.used if self.arena is not None else 0)
        self.sched.used = used
        self.sched.peak_used = max(self.sched.peak_used, used)

    def _sample_device(self):
        f, _ = self.torch.cuda.mem_get_info(self.device)
        self.min_free = min(self.min_free, f)

    def _make_arena(self, size: int):
        torch = self.torch
        torch.cuda.synchronize(self.device)
        torch.cuda.empty_cache()
        self.arena = Arena(max(0, int(size)))
        self.mem = torch.empty(max(self.arena.size, 256), dtype=torch.uint8, device=self.device)
        self._sample_device()

    def _view(self, off: int, nbytes: int, dtype, shape):
        return self.mem[off:off + nbytes].view(dtype).view(shape)

    # -- systems and contexts ----------------------------------------------------------
    def system(self, sysid: int):
        if sysid not in self._sys_cache:
            self._sys_cache[sysid] = self.systems[sysid].system()
        return self._sys_cache[sysid]

    def prepare(self, sysids: Sequence[int], contexts: bool = True):
        """Ahead of the stream (not part of any job's latency): build the host-side systems,
        and with `contexts` one pooled context per system, tuned for its shape, smallest first
        while they leave half the budget; then the arena from what remains."""
        torch = self.torch
        for s in sysids:
            self.system(s)
        if contexts:
            limit = int((1.0 - max(self.arena_fraction, 0.0)) * self.sched.budget)
            for s in sorted(sysids, key=lambda i: array_bytes(self.systems[i], self.precision)):
                inst = self.systems[s]
                if self.ctx_used + self._ctx_estimate(s) > limit:
                    continue
                ctx, cbytes = self._new_ctx(s)
                self.ctx_used += cbytes
                if self.tune:
                    from . import autotune
                    psi = self._bands_alloc(inst, inst.seed)
                    work = ctx.alloc_work(inst.nbands)
                    work["C"].zero_()
                    work["C"].diagonal().fill_(1.0)
                    autotune.tune(ctx, psi, work)
                    del psi, work
                self.pool[s].append((ctx, cbytes))
                self.idle_lru[(s, id(ctx))] = True
        reserve = int(self.ctx_reserve_fraction * self.sched.budget)
        self._make_arena(self.sched.budget - self.ctx_used - reserve - self.margin())
        self._account()

    def _ctx_estimate(self, sysid: int) -> int:
        """Bytes of a new context of the system: measured if one was made before, else an
        upper estimate of its scratch (projections, Gram partials, subspace workspace, digit
        planes of the tensor-core Gram and rotation, potential tables)."""
        if sysid in self.ctx_bytes:
            return self.ctx_bytes[sysid]
        inst = self.systems[sysid]
        nb = inst.nbands
        return (1536 << 20) + 24 * nb * nb * 16 + 4 * inst.npoints * 8

    def reclaim(self, short: int) -> int:
        """Evict idle pooled contexts, least recently used first, until `short` bytes are
        freed (or none is left); returns the bytes freed."""
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

    def _new_ctx(self, sysid: int):
        """A new context of the system and its measured device bytes."""
        from . import api
        torch = self.torch
        inst = self.systems[sysid]
        torch.cuda.synchronize(self.device)
        f0, _ = torch.cuda.mem_get_info(self.device)
        ctx = api.Context(self.system(sysid), max_bands=inst.nbands, device=self.device, precision=self.precision)
        f1, _ = torch.cuda.mem_get_info(self.device)
        nbytes = max(0, f0 - f1)
        self.ctx_bytes[sysid] = max(nbytes, self.ctx_bytes.get(sysid, 0))
        self.min_free = min(self.min_free, f1)
        return ctx, nbytes

    # -- one job ------------------------------------------------------------------------
    def _bands_alloc(self, inst, seed):
        """uniform(-1, 1) bands of the instance from a seeded generator (newly allocated)."""
        torch = self.torch
        g = torch.Generator(device=self.device)
        g.manual_seed(int(seed))
        shape = (inst.nbands,) + tuple(inst.n[::-1])
        rdt = torch.float32 if self.precision == "mixed" else torch.float64
        re = torch.rand(shape, generator=g, device=self.device, dtype=rdt) * 2 - 1
        if inst.complex_wf:
            im = torch.rand(shape, generator=g, device=self.device, dtype=rdt) * 2 - 1
            return torch.complex(re, im)
        return re

    def _bands_into(self, inst, seed, psi, scratch):
        """The same values as _bands_alloc, written into psi; `scratch` (a band array of the
        same size) holds the real and imaginary parts of complex bands on the way."""
        torch = self.torch
        g = torch.Generator(device=self.device)
        g.manual_seed(int(seed))
        shape = (inst.nbands,) + tuple(inst.n[::-1])
        if not inst.complex_wf:
            torch.rand(shape, generator=g, out=psi)
            psi.mul_(2).sub_(1)
            return
        parts = scratch.view(psi.real.dtype).view((2,) + shape)
        re, im = parts[0], parts[1]
        torch.rand(shape, generator=g, out=re)
        re.mul_(2).sub_(1)
        torch.rand(shape, generator=g, out=im)
        im.mul_(2).sub_(1)
        torch.complex(re, im, out=psi)

    def try_start(self, job: Job):
        """Reserve what the job needs now, or None: its arrays in the arena, and a context
        (an idle pooled one of its system, or a new one charged at its measured size, made
        only when its measured or estimated size fits the contexts' share of the budget after
        evicting idle contexts)."""
        inst = self.systems[job.system]
        sizes = job_array_sizes(inst, self.precision)
        offs = self.arena.alloc_all(sizes)
        if offs is None:
            return None
        if self.pool[job.system]:
            ctx, cbytes = self.pool[job.system].pop()
            self.idle_lru.pop((job.system, id(ctx)), None)
            return offs, ctx, cbytes
        cap = self.ctx_cap()
        est = self._ctx_estimate(job.system)
        if self.ctx_used + est > cap:
            self.ctx_used -= self.reclaim(self.ctx_used + est - cap)
        if self.ctx_used + est > cap:
            for o, n in zip(offs, sizes):
                self.arena.free(o, n)
            return None
        ctx, cbytes = self._new_ctx(job.system)
        self.ctx_used += cbytes
        if self.ctx_used > cap:
            self.ctx_used -= self.reclaim(self.ctx_used - cap)
            if self.ctx_used > cap:
                self.sched.overruns += 1
        return offs, ctx, cbytes

    def start(self, job: Job, reservation, now: float):
        torch = self.torch
        offs, ctx, cbytes = reservation
        inst = self.systems[job.system]
        sizes = job_array_sizes(inst, self.precision)
        nb, shape = inst.nbands, (inst.nbands,) + tuple(inst.n[::-1])
        bufs = [self._view(offs[i], sizes[i], ctx.dtype, shape) for i in range(4)]
        work = {"Hpsi": bufs[2], "Spsi": bufs[3],
                "Hnm": self._view(offs[4], sizes[4], ctx.mat_dtype, (nb, nb)),
                "Snm": self._view(offs[5], sizes[5], ctx.mat_dtype, (nb, nb)),
                "C": self._view(offs[6], sizes[6], ctx.mat_dtype, (nb, nb)),
                "eps": self._view(offs[7], sizes[7], torch.float64, (nb,))}
        sidx = self.free_streams.pop()
        stream = self.streams[sidx]
        # the arena's ranges were last used on other streams: order after the work enqueued so far
        stream.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(stream):
            psi, out = bufs[0], bufs[1]
            self._bands_into(inst, job.psi_seed, psi, out)
            launches0 = ctx.launch_count()
            if self.tune:
                from . import autotune
                if autotune.shape_key(ctx, nb) not in autotune._CACHE:
                    work["C"].zero_()
                    work["C"].diagonal().fill_(1.0)
                autotune.tune(ctx, psi, work)
                self._bands_into(inst, job.psi_seed, psi, out)   # tuning may have written into the work arrays
            pair = [psi, out]
            for it in range(self.iterations):
                ctx.rr_step(pair[it % 2], out=pair[(it + 1) % 2], work=work)
            self.kernel_launches += ctx.launch_count() - launches0
            done = torch.cuda.Event()
            done.record(stream)
        return dict(job=job, ctx=ctx, cbytes=cbytes, stream=stream, sidx=sidx, done=done, offs=offs, sizes=sizes,
                    work=work, rec=JobRecord(job, admitted=now))

    def finish(self, state, now: float) -> JobRecord:
        rec = state["rec"]
        with self.torch.cuda.stream(state["stream"]):
            rec.eps = state["work"]["eps"].cpu().numpy()
        state["ctx"].sync()
        rec.finished = now
        for o, n in zip(state["offs"], state["sizes"]):
            self.arena.free(o, n)
        self.free_streams.append(state["sidx"])
        sysid = state["job"].system
        self.pool[sysid].append((state["ctx"], state["cbytes"]))
        self.idle_lru[(sysid, id(state["ctx"]))] = True
        return rec

    # -- the loop -------------------------------------------------------------------------
    def run(self, jobs: Sequence[Job], duration: Optional[float] = None, poll_s: float = 2e-4,
            clock: Callable[[], float] = time.perf_counter) -> Dict:
        """Serve `jobs` (sorted by arrival) in real time.  Stops when every job has finished,
        or at `duration` seconds (unfinished jobs are counted, not waited for)."""
        if self.arena is None:
            self._make_arena(int(self.arena_fraction * self.sched.budget) - self.ctx_used - self.margin())
        pending = collections.deque(sorted(jobs, key=lambda j: j.arrival))
        active: Dict[int, dict] = {}
        done: List[JobRecord] = []
        self.kernel_launches = 0   # library kernels the jobs launched (tuning included)
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
                    self.sched.retire(st["job"])
                    del active[jid]
                    progressed = True
            while True:
                got = self.sched.pick_with(self.try_start)
                if got is None:
                    break
                job, reservation = got
                st = self.start(job, reservation, clock() - t0)
                self.sched.active[job.job_id] = 0          # a slot; bytes are accounted below
                active[job.job_id] = st
                progressed = True
            self._account()
            self._sample_device()
            if not progressed:
                nxt = pending[0].arrival - (clock() - t0) if pending else poll_s
                time.sleep(max(0.0, min(poll_s, nxt)))
        elapsed = clock() - t0
        self._sample_device()
        return {"records": done, "elapsed": elapsed, "kernel_launches": self.kernel_launches,
                "unfinished": len(active) + len(self.sched.queue) + len(pending),
                "active_at_end": len(active), "queued_at_end": len(self.sched.queue), "peak_used": self.sched.peak_used,
                "budget": self.sched.budget, "max_queue": self.sched.max_queue, "overruns": self.sched.overruns,
                "device_peak_used": self.free_at_start - self.min_free, "arena_bytes": self.arena.size,
                "arena_peak": self.arena.peak, "context_bytes": self.ctx_used}

    def close(self):
        for lst in self.pool.values():
            for ctx, _ in lst:
                ctx.close()
        self.pool.clear()
        self.idle_lru.clear()
        self.mem = None
        self.arena = None


def latency_stats(records: Sequence[JobRecord], warmup: float = 0.0) -> Dict:
    """p50 / p99 latency (arrival to finish) over jobs that arrived after `warmup` seconds."""
    lat = [r.finished - r.job.arrival for r in records if r.job.arrival >= warmup]
    if not lat:
        return {"jobs": 0}
    return {"jobs": len(lat), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(np.mean(lat) * 1e3)}
