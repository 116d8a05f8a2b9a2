"""GPU parity of the density reductions (pawfd_density, pawfd_atomic_density) against the FP64
oracle through the C ABI: pseudo density and atomic density matrices for real / complex FP64
and FP32 bands, on grids with an odd number of points (a ragged tail for the two points per
thread)."""
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


@pytest.mark.parametrize("precision,cplx", [("fp64", False), ("fp64", True), ("mixed", False), ("mixed", True)])
def test_density_and_atomic_density_match_oracle(dev, precision, cplx):
    from paper_2310_14776_gb300 import api
    k = (0.2, 0.1, -0.3) if cplx else (0.0, 0.0, 0.0)
    s = synth.make_system((31, 27, 25), (7.0, 6.5, 6.0), 4, synth.PSET_SPD2, seed=631, k=k, complex_wf=cplx)
    assert s.npoints % 2 == 1
    nb = 37
    ctx = api.Context(s, max_bands=nb, device=dev, precision=precision)
    psi_np = synth.make_psi(s, nb, 632)
    psi = torch.from_numpy(psi_np).to(dev).to(ctx.dtype)
    f_np = np.linspace(2.0, 0.0, nb)
    f = torch.from_numpy(f_np).to(dev)
    rho = ctx.density(psi, f).cpu().numpy()
    P = ctx.project(psi)
    D = ctx.atomic_density(P, f).cpu().numpy()
    ctx.sync()
    # the oracle on the bands the GPU holds (FP32-rounded for the mixed form) and on the
    # GPU's projections (the projections themselves are checked by the parity tests)
    psi_ref = psi.cpu().numpy().astype(np.complex128 if cplx else np.float64)
    ref_rho = O.density(s, psi_ref, f_np).reshape(-1)
    ref_D = O.atomic_density(s, P.cpu().numpy().astype(np.complex128 if cplx else np.float64), f_np)
    rel = 1e-12 if precision == "fp64" else 2e-6
    assert np.max(np.abs(rho - ref_rho)) <= rel * np.max(ref_rho), np.max(np.abs(rho - ref_rho)) / np.max(ref_rho)
    assert np.max(np.abs(D - ref_D)) <= rel * np.max(np.abs(ref_D))
    ctx.close()


@pytest.mark.parametrize("n", [(30, 28, 26), (48, 40, 36)])
def test_poisson_matches_oracle(dev, n):
    """pawfd_poisson (conjugate gradients with the stencil kernel: the general FP64 kernel on
    the smaller grid, the double-float kernel on the larger) against the oracle's Fourier
    solve of the same FD equation."""
    from paper_2310_14776_gb300 import api
    s = synth.make_system(n, (7.0, 6.5, 6.0), 3, synth.PSET_SP, seed=651)
    f = synth.free_grid(s)
    rho_np = np.abs(synth.make_psi(s, 1, 652)).reshape(-1) ** 2
    ctx = api.poisson_context(s, device=dev)
    v, iters, res = ctx.poisson(torch.from_numpy(rho_np).to(dev), tol=1e-12, maxiter=4000)
    ctx.sync()
    ref = O.poisson(f, rho_np).reshape(-1)
    assert res <= 1e-12 and 0 < iters < 4000
    assert np.max(np.abs(v.cpu().numpy() - ref)) <= 1e-9 * np.max(np.abs(ref))
    ctx.close()


@pytest.mark.parametrize("n", [(30, 24, 20), (48, 40, 36), (60, 45, 32), (96, 96, 96)])
def test_poisson_fft_matches_oracle(dev, n):
    """pawfd_poisson_fft (the direct Fourier route on the library's FFT kernels: radices 4, 2, 3
    and 5, ragged line tiles) against the oracle's numpy solve of the same FD equation, and
    against the CG route (pawfd_poisson) on the same density."""
    from paper_2310_14776_gb300 import api
    s = synth.make_system(n, (7.0, 6.5, 6.0), 3, synth.PSET_SP, seed=653)
    f = synth.free_grid(s)
    rho_np = np.abs(synth.make_psi(s, 1, 654)).reshape(-1) ** 2
    ctx = api.poisson_context(s, device=dev)
    rho = torch.from_numpy(rho_np).to(dev)
    v = ctx.poisson_fft(rho).cpu().numpy()
    ref = O.poisson(f, rho_np).reshape(-1)
    assert np.max(np.abs(v - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert abs(v.mean()) <= 1e-13 * np.max(np.abs(ref))
    if n[0] <= 48:
        vcg, _, _ = ctx.poisson(rho, tol=1e-12, maxiter=4000)
        assert np.max(np.abs(vcg.cpu().numpy() - v)) <= 1e-9 * np.max(np.abs(ref))
    ctx.close()


def test_poisson_fft_closed_form(dev):
    """A single cosine density: v = -4 pi rho / L(G) at its one wavevector, the Laplacian's
    symbol written out from the order-6 weights."""
    from paper_2310_14776_gb300 import api
    n, cell = (24, 20, 18), (9.0, 7.5, 6.75)
    s = synth.make_system(n, cell, 1, synth.PSET_SP, seed=655)
    j = (3, -2, 1)
    x = [np.arange(n[c]) * cell[c] / n[c] for c in range(3)]
    Z, Y, X = np.meshgrid(x[2], x[1], x[0], indexing="ij")
    g = [2 * np.pi * j[c] / cell[c] for c in range(3)]
    rho = np.cos(g[0] * X + g[1] * Y + g[2] * Z)
    w = (-49 / 18, 3 / 2, -3 / 20, 1 / 90)
    L = sum((w[0] + 2 * sum(w[m] * np.cos(m * g[c] * cell[c] / n[c]) for m in (1, 2, 3))) / (cell[c] / n[c]) ** 2
            for c in range(3))
    ctx = api.poisson_context(s, device=dev)
    v = ctx.poisson_fft(torch.from_numpy(rho.reshape(-1)).to(dev)).cpu().numpy()
    ctx.close()
    assert np.max(np.abs(v - (-4 * np.pi / L) * rho.reshape(-1))) <= 1e-12 * abs(4 * np.pi / L)


def test_poisson_fft_rejects_other_contexts(dev):
    from paper_2310_14776_gb300 import api, _lib
    s = synth.make_system((12, 10, 8), (5.0, 4.0, 3.5), 1, synth.PSET_SP, seed=656)
    ctx = api.Context(s, max_bands=1, device=dev)   # has atoms and a potential
    rho = torch.zeros(s.npoints, dtype=torch.float64, device=dev)
    with pytest.raises(_lib.PawFDError):
        ctx.poisson_fft(rho)
    ctx.close()
    s7 = synth.make_system((14, 10, 8), (5.0, 4.0, 3.5), 1, synth.PSET_SP, seed=657)
    ctx = api.poisson_context(s7, device=dev)
    with pytest.raises(_lib.PawFDError):
        ctx.poisson_fft(torch.zeros(s7.npoints, dtype=torch.float64, device=dev))
    ctx.close()
