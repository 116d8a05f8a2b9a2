"""Per-shape autotuner for the kernel choices of a context.

Each candidate is a setting of ``pawfd_set_option`` that computes the same result to the
context's tolerance: a different stencil tiling (bitwise the same output), or, for FP64
data, the tensor-core digit-product Gram and rotation against the FP64 FMA kernels.
Candidates are timed with CUDA events on the instance's own arrays, on the current stream,
after one untimed call; the fastest setting is applied to the context and remembered per
shape key (precision, kind, grid, bands, projector rows), so that instances of one shape are
tuned once.
"""
from __future__ import annotations

from typing import Dict, List, Optional, Tuple

import torch

from ._lib import PawFDError

_CACHE: Dict[tuple, Dict[str, int]] = {}


def shape_key(ctx, nb: int) -> tuple:
    return (ctx.precision, ctx.complex, tuple(ctx.n), int(nb), int(ctx.Ip))


def stencil_candidates(ctx) -> List[Dict[str, int]]:
    """Tilings of the stencil kernel that applies to the context's dtype and grid."""
    if ctx.precision == "mixed" and not ctx.complex and ctx.n[0] % 4 == 0 and ctx.n[0] >= 8:
        cands = [{"stencil_variant": 1}]
        for yb in (1, 2, 3):
            for per in (2, 4, 6):
                cands.append({"stencil_variant": 0, "stencil_yblock": yb, "stencil_rows": yb * per})
        return cands
    if (ctx.precision == "mixed" and ctx.complex and ctx.n[0] % 2 == 0 and ctx.n[0] >= 8 and ctx.n[1] >= 3
            and ctx.n[2] >= 3):
        # the complex bulk-copy ring kernel (its tilings are bitwise equal) or the general one
        cands = [{"stencil_variant": 1}]
        for depth in (6, 8):
            for yb in (1, 2, 3):
                for per in (2, 4):
                    cands.append({"stencil_variant": 0, "stencil_ring": depth, "stencil_yblock": yb,
                                  "stencil_rows": yb * per})
        return cands
    return [{"stencil_zsplit": z} for z in (1, 2, 4, 8, 16)]


def contraction_candidates(ctx) -> List[Dict[str, int]]:
    """Gram / rotation variants of equal accuracy.  For FP64 data both the digit-product
    tensor-core kernels and the FP64 FMA kernels meet the FP64 tolerance.  For FP32 data the FMA
    kernels form FP32 products (about 1e-7 relative), far less accurate than the exact digit
    products, so the mixed form keeps the tensor-core path.  The tensor-core Gram's K block (its
    tiling of the grid: whole-scratch blocks, or blocks of 4, 16 or 64 exactness chunks of 512
    values whose digit planes stay in L2 between the slicing and the MMA kernels) is a candidate
    as well: the chunks' exact digit sums are the same for every K block, only the order in which
    the FP64 partial sums of the blocks are added changes (results agree to FP64 rounding)."""
    tc = [{"tensor_cores": 1, "tc_kblk": k} for k in (0, 4, 16, 64)]
    if ctx.precision == "fp64":
        return tc + [{"tensor_cores": 0}]
    return tc


def _time(fn, reps: int) -> float:
    fn()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def _best(ctx, cands, fn, reps) -> Tuple[Optional[Dict[str, int]], List[Tuple[Dict[str, int], float]]]:
    table = []
    for cand in cands:
        try:
            for k, v in cand.items():
                ctx.set_option(k, v)
            table.append((cand, _time(fn, reps)))
        except PawFDError:
            continue   # a variant that does not apply to this context
    if not table:
        return None, table
    return min(table, key=lambda t: t[1])[0], table


def tune(ctx, psi: torch.Tensor, work: dict, reps: int = 2, use_cache: bool = True) -> Dict[str, int]:
    """Pick and apply the fastest stencil tiling and contraction variant for this context's
    shape.  ``psi`` and ``work`` (Hpsi, C) are the instance's own device arrays; their
    contents are overwritten (Hpsi) or read (C, which must hold finite values)."""
    nb = psi.numel() // ctx.K
    key = shape_key(ctx, nb)
    if use_cache and key in _CACHE:
        best = _CACHE[key]
    else:
        best = {}
        s, _ = _best(ctx, stencil_candidates(ctx), lambda: ctx.kinetic_local(psi, out=work["Hpsi"]), reps)
        if s:
            best.update(s)
            for k, v in s.items():
                ctx.set_option(k, v)
        tmp = work["Spsi"]

        def contraction():
            ctx.gram(psi, work["Hpsi"], M=work["Hnm"], hermitian=True)
            ctx.rotate(psi, work["C"], out=tmp)

        cands = contraction_candidates(ctx)
        if cands:
            g, _ = _best(ctx, cands, contraction, reps)
            if g:
                best.update(g)
        _CACHE[key] = best
    for k, v in best.items():
        ctx.set_option(k, v)
    return dict(best)


def clear_cache():
    _CACHE.clear()
