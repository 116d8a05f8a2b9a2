"""The allocation-free Gram entry point (pawfd_gram_noalloc) against pawfd_gram and the oracle.

pawfd_gram_noalloc serves callers that may not allocate device memory (their memory is
owned by another pool allocator, or their serving loop cannot afford cudaMalloc), so it
takes no context and keeps its split-K partials in a fixed device array inside the
library.  This file is collected last so that, should it fail, a run stopping at the first
failure has already run every other test; it passes alone in a fresh process too.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2310_14776_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda:0")


def _noalloc(lib, A, B, nb, dtype_code, dV, M):
    stream = ctypes.c_void_p(torch.cuda.current_stream(A.device).cuda_stream)
    return lib.pawfd_gram_noalloc(ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                                  A.numel() // nb, nb, dtype_code, dV, ctypes.c_void_p(M.data_ptr()), stream)


def _check_two_calls(lib, A, B, nb, cplx, dV, ref, want):
    """Two calls in a row (they share and reuse the static scratch), each against the context
    Gram ``ref`` (1e-12 of its largest entry) and the oracle's Gram ``want`` (the same bar)."""
    from paper_2310_14776_gb300 import _lib
    code = _lib.PAWFD_C128 if cplx else _lib.PAWFD_R64
    scale = float(np.max(np.abs(want)))
    for _ in range(2):
        M = torch.full((nb, nb), float("nan"), dtype=ref.dtype, device=A.device)
        assert _noalloc(lib, A, B, nb, code, dV, M) == 0
        torch.cuda.synchronize(A.device)
        got = M.cpu().numpy()
        assert np.max(np.abs(got - ref.cpu().numpy())) <= 1e-12 * scale
        assert np.max(np.abs(got - want)) <= 1e-12 * scale


@pytest.mark.parametrize("cplx", [False, True])
def test_noalloc_gram_matches_context_gram(dev, cplx):
    from paper_2310_14776_gb300 import _lib, api
    k = (0.3, -0.2, 0.1) if cplx else (0.0, 0.0, 0.0)
    s = synth.make_system((40, 36, 30), (9.0, 8.0, 7.0), 5, synth.PSET_SPD2, seed=401, k=k, complex_wf=cplx)
    nb = 70                      # two 64-wide tiles with a ragged tail
    ctx = api.Context(s, max_bands=nb, device=dev)
    psi_h = synth.make_psi(s, nb, 402)
    psi = torch.from_numpy(psi_h).to(dev)
    hpsi = ctx.apply_H(psi)
    ref = ctx.gram(psi, hpsi)
    torch.cuda.synchronize(dev)
    want = O.gram(psi_h, hpsi.cpu().numpy(), s.dV, nb)
    _check_two_calls(_lib.load(), psi, hpsi, nb, cplx, s.dV, ref, want)
    ctx.close()


@pytest.mark.parametrize("cplx,nb", [(False, 1024), (True, 724)])
def test_noalloc_gram_at_the_array_limit(dev, cplx, nb):
    # the largest band counts whose one nb x nb partial fits the 8 MiB array: the split over K
    # is capped at one partial there (a single K chunk per tile)
    from paper_2310_14776_gb300 import _lib, api
    k = (0.2, 0.1, -0.3) if cplx else (0.0, 0.0, 0.0)
    s = synth.make_system((12, 10, 8), (5.0, 4.4, 3.9), 2, synth.PSET_SP, seed=403, k=k, complex_wf=cplx)
    ctx = api.Context(s, max_bands=nb, device=dev)
    a_h = synth.make_psi(s, nb, 404)
    b_h = synth.make_psi(s, nb, 405)
    A = torch.from_numpy(a_h).to(dev)
    B = torch.from_numpy(b_h).to(dev)
    ref = ctx.gram(A, B)
    torch.cuda.synchronize(dev)
    want = O.gram(a_h, b_h, s.dV, nb)
    _check_two_calls(_lib.load(), A, B, nb, cplx, s.dV, ref, want)
    ctx.close()


def test_noalloc_gram_rejects_sizes_beyond_its_array(dev):
    from paper_2310_14776_gb300 import _lib
    lib = _lib.load()
    x = torch.zeros(16, dtype=torch.float64, device=dev)
    # one 1025 x 1025 real partial (8.4 MB) exceeds the 8 MiB array; checked before any launch
    assert _noalloc(lib, x, x, 1025, _lib.PAWFD_R64, 1.0, x) == -1
    assert _noalloc(lib, x, x, 725, _lib.PAWFD_C128, 1.0, x) == -1
    assert _noalloc(lib, x, x, 1, 7, 1.0, x) == -1
    torch.cuda.synchronize(dev)
    assert np.isfinite(x.cpu().numpy()).all()
