"""GPU parity of the block-Davidson step (the iterative eigensolver of the Kohn-Sham section,
in the reading of ``oracle.davidson_step``) through the C ABI: residual norms, corrections,
the 2n Ritz values and the n output vectors against the FP64 oracle, and a run of steps
against the exact spectrum of the dense operators on a tiny grid."""
import numpy as np
import pytest
import scipy.linalg
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


def to_dev(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def gpu_step(ctx, psi, eps, nb, dev):
    w = ctx.alloc_davidson(nb)
    w["X"][:nb].copy_(to_dev(psi, dev).reshape(w["X"][:nb].shape))
    ctx.davidson_step(w, nb, to_dev(np.asarray(eps[:nb], np.float64), dev))
    ctx.sync()
    return w


U32 = 2.0 ** -24


def fft32_bound(s):
    """Per-band relative bound of an FP32 Fourier-space solve (pawfd_kinetic_precond): the
    input rounded to FP32, three passes each way (a few roundings per radix stage), the table
    entry: 8 u log2 K."""
    return 8 * U32 * np.log2(s.npoints)


@pytest.mark.parametrize("precond", ["kinetic", "jacobi"])
@pytest.mark.parametrize("cplx", [False, True])
def test_davidson_step_matches_oracle(dev, cplx, precond):
    from paper_2310_14776_gb300 import api
    k = (0.2, 0.1, -0.3) if cplx else (0.0, 0.0, 0.0)
    s = synth.make_system((30, 24, 20), (7.0, 6.5, 6.0), 4, synth.PSET_SPD2, seed=611, k=k, complex_wf=cplx)
    nb = 24
    rr = O.rayleigh_ritz(s, synth.make_psi(s, nb, 612))
    ref = O.davidson_step(s, rr["psi_rot"], rr["eps"], precond=precond)
    ctx = api.Context(s, max_bands=2 * nb, device=dev)
    ctx.set_option("davidson_precond", 1 if precond == "kinetic" else 0)
    w = gpu_step(ctx, rr["psi_rot"], rr["eps"], nb, dev)
    K = s.npoints
    assert np.allclose(w["rnorm"].cpu().numpy(), ref["rnorm"], rtol=1e-11, atol=0)
    corr = w["X"][nb:].cpu().numpy().reshape(nb, K)
    rcorr = ref["X"].reshape(2 * nb, K)[nb:]
    eps = w["eps"].cpu().numpy()
    if precond == "jacobi":
        # FP32 weights: d - eps in FP32 cancels at most tenfold (the floor is a tenth of d0), so
        # each weight is within 16 u of the FP64 one
        assert np.all(np.abs(corr - rcorr) <= 16 * U32 * np.abs(rcorr) + 1e-300)
    else:
        # FP32 transforms: the corrections to the FP32 bound
        err = np.linalg.norm(corr - rcorr, axis=1) / np.linalg.norm(rcorr, axis=1)
        assert err.max() <= fft32_bound(s), err.max()
    # the Ritz values exactly those of the GPU's own subspace X (the oracle's Rayleigh-Ritz on
    # it), and within the effect of the FP32 corrections of the oracle's FP64 step
    X = w["X"].cpu().numpy()
    HX, _ = O.apply_H(s, X)
    SX, _ = O.apply_S(s, X)
    own, _, _ = O.subspace_diag(O.gram(X, HX, s.dV, 2 * nb), O.gram(X, SX, s.dV, 2 * nb))
    assert np.max(np.abs(eps - own)) <= 1e-10, np.max(np.abs(eps - own))
    assert np.max(np.abs(eps[:nb] - ref["eps"][:nb])) <= 1e-5 * max(1.0, np.max(np.abs(ref["eps"])))
    # the output vectors: S-orthonormal Ritz vectors with the n lowest Ritz values
    out = w["psi_out"].cpu().numpy()
    check = O.rayleigh_ritz(s, out)
    assert np.max(np.abs(check["Snm"] - np.eye(nb))) <= 1e-10
    assert np.max(np.abs(check["Hnm"] - np.diag(eps[:nb]))) <= 1e-10 * max(1.0, np.max(np.abs(ref["eps"])))
    ctx.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_rotate_n_is_the_first_columns_of_rotate(dev, precision):
    from paper_2310_14776_gb300 import api
    s = synth.make_system((30, 28, 26), (7.0, 6.5, 6.0), 4, synth.PSET_SPD2, seed=621)
    nb = 150
    ctx = api.Context(s, max_bands=nb, device=dev, precision=precision)
    psi = to_dev(synth.make_psi(s, nb, 622), dev).to(ctx.dtype)
    C = to_dev(np.linalg.qr(np.random.default_rng(623).standard_normal((nb, nb)))[0], dev)
    full = ctx.rotate(psi, C)
    for nout in (1, 37, 128, 149):
        part = ctx.rotate_n(psi, C, nout)
        assert torch.equal(part, full[:nout])
    ctx.close()


@pytest.mark.parametrize("case", ["bloch", "selfwrap"])
def test_davidson_iteration_against_dense_spectrum(dev, case):
    # GPU steps from the same start: Ritz values stay above the exact eigenvalues, never rise,
    # and approach them (tiny grids: the general stencil kernel and the FMA Gram path)
    import test_oracle_pins as T
    from paper_2310_14776_gb300 import api
    s = T.small_system(**T.TINY[case])
    H, S = T.dense_operators(s)
    exact = scipy.linalg.eigh(H, S, eigvals_only=True)
    nb = 4
    rr = O.rayleigh_ritz(s, T.rand_psi(s, nb, 5))
    ctx = api.Context(s, max_bands=2 * nb, device=dev)
    w = ctx.alloc_davidson(nb)
    w["X"][:nb].copy_(to_dev(rr["psi_rot"], dev).reshape(w["X"][:nb].shape))
    eps = to_dev(rr["eps"], dev)
    first = None
    for it in range(40):
        ctx.davidson_step(w, nb, eps)
        new = w["eps"][:nb].clone()
        e = new.cpu().numpy()
        assert np.all(e >= exact[:nb] - 1e-10)
        assert np.all(e <= eps.cpu().numpy() + 1e-10)
        if first is None:
            first = np.sum(e - exact[:nb])
        w["X"][:nb].copy_(w["psi_out"])
        eps = new
    ctx.sync()
    assert np.sum(eps.cpu().numpy() - exact[:nb]) < first / 50
    ctx.close()


def test_davidson_step_mixed_form(dev):
    """The step on FP32 bands (mixed context): residual norms, the 2n Ritz values and the
    S-orthonormal output against the FP64 oracle step on the same FP32-rounded input, to the
    FP32 level (the corrections are formed from FP32 H psi and S psi)."""
    from paper_2310_14776_gb300 import api
    s = synth.make_system((30, 28, 26), (7.0, 6.5, 6.0), 4, synth.PSET_SPD2, seed=671)
    nb = 24
    rr = O.rayleigh_ritz(s, synth.make_psi(s, nb, 672))
    psi32 = rr["psi_rot"].astype(np.float32)
    # 28 = 4 x 7 and 26 = 2 x 13: no FFT of these sizes, so the step takes the Jacobi
    # preconditioner (the documented rule of pawfd_davidson_step)
    ref = O.davidson_step(s, psi32.astype(np.float64), rr["eps"], precond="jacobi")
    ctx = api.Context(s, max_bands=2 * nb, device=dev, precision="mixed")
    w = gpu_step(ctx, psi32, rr["eps"], nb, dev)
    assert np.allclose(w["rnorm"].cpu().numpy(), ref["rnorm"], rtol=1e-5, atol=0)
    eps = w["eps"].cpu().numpy()
    scale = max(1.0, np.max(np.abs(ref["eps"])))
    assert np.max(np.abs(eps - ref["eps"])) <= 1e-5 * scale, np.max(np.abs(eps - ref["eps"]))
    out = w["psi_out"].cpu().numpy().astype(np.float64)
    check = O.rayleigh_ritz(s, out)
    assert np.max(np.abs(check["Snm"] - np.eye(nb))) <= 1e-5
    ctx.close()


@pytest.mark.parametrize("precision,cplx,nb,n", [("fp64", False, 6, (30, 24, 20)), ("fp64", True, 5, (30, 24, 20)),
                                                 ("mixed", False, 7, (30, 24, 20)), ("mixed", True, 4, (30, 24, 20)),
                                                 ("fp64", False, 1, (30, 24, 20)), ("mixed", False, 3, (128, 100, 6)),
                                                 ("fp64", True, 2, (128, 100, 6))])
def test_kinetic_precond_against_oracle(dev, precision, cplx, nb, n):
    """pawfd_kinetic_precond against the oracle's -(T + sigma)^-1 on grids of radices 4, 2, 3
    and 5, real (band pairs per transform, an odd count leaving one band alone) and Bloch, FP64
    and FP32 bands, out aliasing R.  On 30 x 24 x 20 the x and y transforms run as one pass per
    xy plane (both plane buffers in shared memory); the 128 x 100 plane does not fit, so there
    they run as separate passes."""
    from paper_2310_14776_gb300 import api
    k = (0.31, -0.22, 0.17) if cplx else (0.0, 0.0, 0.0)
    cell = tuple(0.3 * v for v in n)
    s = synth.make_system(n, cell, 3, synth.PSET_SP, seed=681, k=k, complex_wf=cplx)
    R = synth.make_psi(s, nb, 682)
    ctx = api.Context(s, max_bands=nb, device=dev, precision=precision)
    Rd = to_dev(R, dev).to(ctx.dtype)
    out = ctx.kinetic_precond(Rd).cpu().numpy()
    same = Rd.clone()
    ctx.kinetic_precond(same, out=same)
    ctx.close()
    Rin = Rd.cpu().numpy().astype(np.complex128 if cplx else np.float64)
    ref = O.kinetic_precondition(s, Rin)
    err = np.linalg.norm((out.astype(ref.dtype) - ref).reshape(nb, -1), axis=1) / \
        np.linalg.norm(ref.reshape(nb, -1), axis=1)
    assert err.max() <= fft32_bound(s), err.max()
    assert np.array_equal(same.cpu().numpy(), out)


def test_kinetic_precond_rejects_other_grid_factors(dev):
    from paper_2310_14776_gb300 import api, _lib
    s = synth.make_system((14, 10, 8), (5.0, 4.0, 3.5), 1, synth.PSET_SP, seed=683)
    ctx = api.Context(s, max_bands=2, device=dev)
    with pytest.raises(_lib.PawFDError):
        ctx.kinetic_precond(torch.zeros((2,) + tuple(s.n[::-1]), dtype=torch.float64, device=dev))
    ctx.close()
