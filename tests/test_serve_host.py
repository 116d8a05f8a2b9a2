"""Host-side logic (no GPU): the batched and served forms (seeded instance sizes, the Poisson
job stream, the scheduler's HBM budget and admission rules, latency statistics), the bench's
helpers (tile count, oracle stage timing), and the seeded input generator (SplitMix64,
projector normalisation, real harmonics, the free grid of the Poisson solve)."""
import numpy as np

from paper_2310_14776_gb300 import serve, synth


def test_batch_instances_are_seeded_and_in_range():
    a = synth.batch_instances(64)
    b = synth.batch_instances(64)
    assert a == b
    for inst in a:
        assert all(32 <= v <= 80 for v in inst.n)
        assert 32 <= inst.nbands <= 256 and 2 <= inst.natoms <= 24
        assert all(0.0 <= inst.k[c] < np.pi / inst.cell[c] for c in range(3))
        assert abs(inst.cell[0] / inst.n[0] - 0.2 * synth.BOHR_PER_ANGSTROM) < 1e-12
    # the sizes actually vary (non-cubic grids allowed)
    assert len({inst.n for inst in a}) > 50
    assert any(len(set(inst.n)) > 1 for inst in a)


def test_poisson_stream_rate_and_mix():
    jobs = serve.job_stream(200.0, 30.0, 64, 8)
    assert jobs == serve.job_stream(200.0, 30.0, 64, 8)
    n = len(jobs)
    # Poisson count: mean 6000, sd ~77
    assert abs(n - 6000) < 5 * np.sqrt(6000)
    gaps = np.diff([0.0] + [j.arrival for j in jobs])
    assert np.all(gaps >= 0) and abs(gaps.mean() - 1 / 200.0) < 5 * (1 / 200.0) / np.sqrt(n)
    large = sum(j.system >= 64 for j in jobs) / n
    assert abs(large - 0.1) < 5 * np.sqrt(0.09 / n)
    assert all(0 <= j.system < 72 for j in jobs)


def test_scheduler_never_exceeds_budget_and_admits_first_fit():
    rng = np.random.default_rng(1)
    sizes = {j: int(rng.integers(1, 40)) for j in range(300)}
    sch = serve.Scheduler(budget=100, max_active=6)
    jobs = [serve.Job(j, float(j), 0, j) for j in range(300)]
    need = lambda job: sizes[job.job_id]  # noqa: E731
    no_reclaim = lambda short: 0  # noqa: E731
    running, finished = [], []
    for job in jobs:
        sch.arrive(job)
        while True:
            window, free, full = list(sch.queue)[: sch.lookahead], sch.free_bytes(), len(sch.active) >= 6
            pick = sch.pick(need, no_reclaim)
            if pick is None:
                # nothing in the window fits (or every slot is taken)
                assert full or all(need(j) > free for j in window)
                break
            # first fit: no earlier waiting job within the lookahead would have fit
            pos = window.index(pick)
            assert need(pick) <= free and all(need(j) > free for j in window[:pos])
            assert pick not in sch.queue
            sch.admit(pick, need(pick))
            running.append(pick)
            assert sch.used <= sch.budget and len(sch.active) <= 6
        if running and rng.random() < 0.6:
            done = running.pop(int(rng.integers(len(running))))
            sch.retire(done)
            finished.append(done)
    while running:
        sch.retire(running.pop())
    assert sch.used == 0 and sch.overruns == 0
    assert sch.peak_used <= 100


def test_scheduler_reclaims_idle_memory_and_skips_impossible_jobs():
    sch = serve.Scheduler(budget=100, max_active=4)
    sch.used = 90                       # idle pooled contexts hold 90
    pool = [50, 40]

    def reclaim(short):
        freed = 0
        while pool and freed < short:
            freed += pool.pop(0)
        return freed

    sch.arrive(serve.Job(0, 0.0, 0, 0))   # needs 200: never fits this budget
    sch.arrive(serve.Job(1, 0.0, 0, 1))   # needs 30: fits after reclaiming one context
    need = {0: 200, 1: 30}
    pick = sch.pick(lambda j: need[j.job_id], reclaim)
    assert pick.job_id == 1 and sch.used == 40 and pool == [40]
    assert [j.job_id for j in sch.queue] == [0]


def test_arena_first_fit_alignment_and_coalescing():
    a = serve.Arena(10000, align=256)
    assert a.size == 9984
    offs = [a.alloc(n) for n in (100, 300, 256, 1000)]
    assert offs == [0, 256, 768, 1024]                      # first fit, 256-byte aligned
    assert a.used == 256 + 512 + 256 + 1024
    a.free(256, 300)                                        # a hole of 512 bytes
    assert a.alloc(600) == 2048                             # does not fit the hole
    assert a.alloc(500) == 256                              # the first range that fits
    a.free(0, 100)
    a.free(256, 500)
    a.free(768, 256)
    # the three freed neighbours merged into one range at 0
    assert a.free_ranges[0] == (0, 1024)
    a.free(1024, 1000)
    a.free(2048, 600)
    assert a.free_ranges == [(0, 9984)] and a.used == 0
    assert a.peak == 256 + 512 + 256 + 1024 + 768


def test_arena_alloc_all_is_all_or_nothing():
    a = serve.Arena(4096, align=256)
    held = a.alloc(2048)
    assert a.alloc_all([1024, 1024, 256]) is None
    assert a.used == 2048 and a.free_ranges == [(2048, 2048)]
    offs = a.alloc_all([1024, 1024])
    assert offs == [2048, 3072] and a.used == 4096
    for o in offs:
        a.free(o, 1024)
    a.free(held, 2048)
    assert a.free_ranges == [(0, 4096)]


def test_arena_random_alloc_free_never_overlaps():
    rng = np.random.default_rng(3)
    a = serve.Arena(1 << 20, align=256)
    live = {}
    for step in range(3000):
        if live and (rng.random() < 0.45 or len(live) > 60):
            off = list(live)[int(rng.integers(len(live)))]
            a.free(off, live.pop(off))
        else:
            n = int(rng.integers(1, 40000))
            off = a.alloc(n)
            if off is not None:
                assert off % 256 == 0 and off + n <= a.size
                live[off] = n
        spans = sorted((o, o + ((n + 255) // 256) * 256) for o, n in live.items())
        assert all(spans[i][1] <= spans[i + 1][0] for i in range(len(spans) - 1))
        assert a.used == sum(e - o for o, e in spans)
        free = sum(ln for _, ln in a.free_ranges)
        assert free + a.used == a.size
        assert all(a.free_ranges[i][0] + a.free_ranges[i][1] < a.free_ranges[i + 1][0]
                   for i in range(len(a.free_ranges) - 1))    # no two free ranges left unmerged


def test_scheduler_pick_with_first_fit_and_slots():
    sch = serve.Scheduler(budget=100, max_active=2)
    for j in range(5):
        sch.arrive(serve.Job(j, 0.0, 0, j))
    fits = {0: None, 1: None, 2: "r2", 3: "r3", 4: "r4"}
    job, r = sch.pick_with(lambda job: fits[job.job_id])
    assert job.job_id == 2 and r == "r2" and [j.job_id for j in sch.queue] == [0, 1, 3, 4]
    sch.active[2] = 0
    sch.active[9] = 0
    assert sch.pick_with(lambda job: "any") is None         # no free slot


def test_array_bytes():
    inst = synth.Instance((10, 11, 12), 7, 2, 0, True, (0.0, 0.0, 0.0))
    assert serve.array_bytes(inst, "mixed") == 4 * 1320 * 7 * 8 + 3 * 49 * 16 + 56
    assert serve.array_bytes(inst, "fp64") == 4 * 1320 * 7 * 16 + 3 * 49 * 16 + 56


def test_bench_tile_area_counts_upper_triangle_tiles():
    # the bench's count of the entries the real Hermitian Gram kernel computes (128 x 96 tiles
    # that hold an element with row <= column; for 192 < nb <= 256 the four tiles of the
    # symmetric cover) against a brute-force enumeration
    import bench
    for nb in (1, 17, 96, 128, 150, 192, 193, 256, 257, 300, 1024):
        tiles = 0
        for r0 in range(0, nb, 128):
            for c0 in range(0, nb, 96):
                if any(r <= c for r in range(r0, min(nb, r0 + 128)) for c in range(c0, min(nb, c0 + 96))):
                    tiles += 1
        if 192 < nb <= 256:
            tiles = 4
        assert bench.sg_tiles_area(nb) == tiles * 128 * 96, nb


def test_symmetric_cover_table_holds_every_block_pair():
    # the cover table of the tensor-core Gram (csrc/tc_gram.cu): four tiles of 128 rows (from a
    # 32-row block) x three 32-row B blocks whose entries and mirrors hold every pair of the
    # eight blocks of a 256-band Hermitian matrix; the kernel's write rule (first tile that
    # holds a pair owns it, direct orientation when it has one) then writes every upper entry
    # exactly once
    import pathlib
    import re
    root = pathlib.Path(__file__).resolve().parents[1]
    src = (root / "paper_2310_14776_gb300" / "csrc" / "tc_gram.cu").read_text()
    rows = [int(v) for v in re.search(r"kCoverRowBlk\[sg::COVER_TILES\] = \{([^}]*)\}", src).group(1).split(",")]
    segs = [[int(v) for v in t.split(",")] for t in re.findall(r"\{(\d+, \d+, \d+)\}",
                                                             src[src.find("kCoverSegBlk"):src.find("bool use_cover")])]
    assert len(rows) == 4 and len(segs) == 4
    nb = 256
    cnt = np.zeros((nb, nb), int)
    owned = set()
    for t in range(4):
        mine = {}
        for lo in range(8):
            for hi in range(lo, 8):
                if (lo, hi) in owned:
                    continue
                direct = rows[t] <= lo < rows[t] + 4 and hi in segs[t]
                mirrored = rows[t] <= hi < rows[t] + 4 and lo in segs[t]
                if direct or mirrored:
                    owned.add((lo, hi))
                    mine[(lo, hi)] = direct
        for n in range(32 * rows[t], 32 * rows[t] + 128):
            for c in range(96):
                m = 32 * segs[t][c // 32] + c % 32
                bi, bj = n // 32, m // 32
                key = (min(bi, bj), max(bi, bj))
                if key not in mine:
                    continue
                if bi == bj:
                    write = n <= m
                else:
                    write = bi == key[0] if mine[key] else bi == key[1]
                if write:
                    cnt[min(n, m), max(n, m)] += 1
    assert len(owned) == 36
    assert np.array_equal(cnt, np.triu(np.ones((nb, nb), int)))


def test_free_grid_is_the_bare_operator():
    s = synth.make_system((12, 10, 8), (6.0, 5.0, 4.0), 3, synth.PSET_SP, seed=5, k=(0.1, 0.0, 0.2), complex_wf=True)
    f = synth.free_grid(s)
    assert f.natoms == 0 and f.nproj_total == 0 and not f.complex_wf and tuple(f.k) == (0.0, 0.0, 0.0)
    assert np.all(f.vloc == 0) and f.vloc.shape == s.vloc.shape and tuple(f.n) == tuple(s.n)
    assert tuple(f.cell) == tuple(s.cell)


def test_latency_stats_over_the_jobs_after_the_warmup():
    finished = [1.5, 2.0, 4.0, 3.5, 9.0]
    recs = [serve.JobRecord(serve.Job(i, float(i), 0, i), admitted=float(i), finished=f) for i, f in enumerate(finished)]
    st = serve.latency_stats(recs, warmup=1.0)
    lat = np.array(finished[1:]) - np.arange(1, 5)      # finished - arrival of jobs 1..4
    assert st["jobs"] == 4
    assert abs(st["p50_ms"] - 1e3 * np.median(lat)) < 1e-9
    assert abs(st["mean_ms"] - 1e3 * lat.mean()) < 1e-9
    assert serve.latency_stats(recs, warmup=10.0) == {"jobs": 0}


def test_bench_oracle_stage_timing():
    # the CPU baseline's step is the oracle's own calls, each timed; the total is their sum
    import bench
    w = synth.WORKLOADS["gamma-24c-16b"]
    s = w.system()
    stages = {}
    total = bench.oracle_step_time(s, w.psi(s, nb=4), stages)
    assert set(stages) == {"apply_H", "apply_S", "gram_HS", "subspace_diag", "rotate"}
    assert all(v > 0 for v in stages.values())
    assert abs(total - sum(stages.values())) < 1e-12


def test_splitmix64_matches_the_published_sequence():
    # the generator's mixing function is SplitMix64's output function: with the state advanced
    # by the golden-ratio increment from seed 0, the first outputs of the published generator
    # (Steele, Lea & Flood, OOPSLA 2014; the widely used splitmix64.c) are these
    g = np.uint64(0x9E3779B97F4A7C15)
    with np.errstate(over="ignore"):
        z = synth._mix64(np.array([g * np.uint64(i) for i in (1, 2, 3)], dtype=np.uint64))
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    # element i of a stream does not depend on where the draw starts
    a = synth.uniform01(7, synth.STREAM_PSI_RE, 0, 100)
    b = synth.uniform01(7, synth.STREAM_PSI_RE, 40, 60)
    assert np.array_equal(a[40:], b) and np.all((a >= 0) & (a < 1))


def test_projector_radial_normalisation_by_quadrature():
    # N^2 int_0^inf r^(2l+2) exp(-r^2 / sigma^2) dr = 1 (the untruncated projector has unit norm)
    from scipy.integrate import quad
    for l in (0, 1, 2):
        for sigma in (0.5, 0.8):
            N = synth.radial_norm(l, sigma)
            val, err = quad(lambda r: N * N * r ** (2 * l + 2) * np.exp(-r * r / sigma ** 2), 0, np.inf)
            assert abs(val - 1.0) < 1e-10, (l, sigma, val)


def test_real_harmonics_are_orthonormal_on_the_sphere():
    # Gauss-Legendre in cos(theta) x uniform phi integrates these polynomials exactly
    mu, wmu = np.polynomial.legendre.leggauss(12)
    phi = np.arange(24) * (2 * np.pi / 24)
    M, P = np.meshgrid(mu, phi, indexing="ij")
    W = np.outer(wmu, np.full(24, 2 * np.pi / 24))
    st = np.sqrt(1 - M * M)
    x, y, z = st * np.cos(P), st * np.sin(P), M
    Y = [f for l in (0, 1, 2) for f in synth.solid_harmonics(l, x, y, z)]
    G = np.array([[np.sum(W * a * b) for b in Y] for a in Y])
    assert np.allclose(G, np.eye(9), rtol=0, atol=1e-13)
