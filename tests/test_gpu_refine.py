"""GPU parity of the final refinement of the mixed form against the FP64 oracle.

The refinement takes the FP32 input bands of a mixed Rayleigh-Ritz step and that step's FP64
eigenvector matrix C_lo, rotates the promoted input by C_lo in FP64 (which keeps its span),
and runs an FP64 Rayleigh-Ritz step on the result.  Its stages are held to the FP64 bars:
the rotated bands and H psi', S psi' per band 1e-12 relative, refined eigenvalues and
Rayleigh quotients 1e-10 Ha, residual norms 1e-9 relative.  The end-to-end bar of the mixed
form is asserted as stated: refined eigenvalues within 1e-8 Ha of the oracle's plain FP64
Rayleigh-Ritz step on the same (FP32-valued) input.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2310_14776_gb300 import synth

pytestmark = pytest.mark.gpu

REL = 1e-12
EPS_TOL = 1e-10
MIXED_TOL = 1e-8     # refined mixed-form eigenvalues against the FP64 step


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda:0")


CASES = {
    "gamma": dict(n=(24, 24, 24), cell=(10.0, 10.0, 10.0), natoms=2, pset=synth.PSET_SP, nb=16, cplx=False),
    "bloch": dict(n=(30, 28, 26), cell=(11.3, 10.6, 9.8), natoms=5, pset=synth.PSET_SPD2, nb=24, cplx=True),
    "ragged": dict(n=(45, 19, 13), cell=(9.0, 7.6, 5.2), natoms=4, pset=synth.PSET_SPD2, nb=9, cplx=True),
    "f32x4-ragged": dict(n=(132, 37, 10), cell=(26.0, 7.4, 4.0), natoms=5, pset=synth.PSET_SPD2, nb=5, cplx=False),
}


def _per_band(got, want, nb):
    got, want = got.reshape(nb, -1), want.reshape(nb, -1)
    return np.linalg.norm(got - want, axis=1) / np.linalg.norm(want, axis=1)


@pytest.mark.parametrize("case", sorted(CASES))
def test_refine_against_oracle(dev, case):
    from paper_2310_14776_gb300 import api
    cs = CASES[case]
    k = (0.31, -0.22, 0.17) if cs["cplx"] else (0.0, 0.0, 0.0)
    s = synth.make_system(cs["n"], cs["cell"], cs["natoms"], cs["pset"], seed=700, k=k, complex_wf=cs["cplx"])
    nb = cs["nb"]
    psi32 = synth.make_psi(s, nb, 701).astype(np.complex64 if cs["cplx"] else np.float32)
    mixed = api.Context(s, max_bands=nb, device=dev, precision="mixed")
    fp64 = api.Context(s, max_bands=nb, device=dev, precision="fp64")
    psi_in = torch.from_numpy(psi32).to(dev)
    rr = mixed.rayleigh_ritz(psi_in)
    C_lo = rr["C"]
    out = fp64.refine(psi_in, C_lo)
    torch.cuda.synchronize(dev)
    ref = O.refine(s, psi32, C_lo.cpu().numpy())

    # step 1: the promoted input rotated by C_lo in FP64; step 2: H psi', S psi' in FP64
    assert _per_band(out["psi"].cpu().numpy(), ref["psi"], nb).max() <= REL
    assert _per_band(out["Hpsi"].cpu().numpy(), ref["Hpsi"], nb).max() <= REL
    assert _per_band(out["Spsi"].cpu().numpy(), ref["Spsi"], nb).max() <= REL
    # steps 4-6
    assert np.max(np.abs(out["theta"].cpu().numpy() - ref["theta"])) <= EPS_TOL
    eps = out["eps"].cpu().numpy()
    assert np.max(np.abs(eps - ref["eps"])) <= EPS_TOL
    resid = out["resid"].cpu().numpy()
    assert np.all(np.abs(resid - ref["resid"]) <= 1e-9 * ref["resid"] + 1e-13)
    C = out["C"].cpu().numpy()
    Sh, Hh = 0.5 * (ref["Snm"] + ref["Snm"].conj().T), 0.5 * (ref["Hnm"] + ref["Hnm"].conj().T)
    assert np.allclose(C.conj().T @ Sh @ C, np.eye(nb), rtol=0, atol=1e-11)
    assert np.allclose(C.conj().T @ Hh @ C, np.diag(eps), rtol=0, atol=1e-11 * np.max(np.abs(eps)))

    # end to end: refined eigenvalues against the oracle's plain FP64 step on the same input
    first = O.rayleigh_ritz(s, psi32.astype(np.complex128 if cs["cplx"] else np.float64))
    err = np.abs(eps - first["eps"]).max()
    err_mixed = np.abs(rr["eps"].cpu().numpy() - first["eps"]).max()
    print("%s: max|eps_refined - eps_fp64| = %.2e Ha, max|eps_mixed - eps_fp64| = %.2e Ha, max resid %.2e"
          % (case, err, err_mixed, resid.max()))
    assert err <= MIXED_TOL
    mixed.close()
    fp64.close()


def test_refine_of_rotated_bands_against_oracle(dev):
    # without C_lo the given bands (here the FP32-rounded rotated output of a mixed step) are
    # refined as they are: every stage against the oracle's refinement of the same bands
    from paper_2310_14776_gb300 import api
    cs = CASES["bloch"]
    s = synth.make_system(cs["n"], cs["cell"], cs["natoms"], cs["pset"], seed=702, k=(0.31, -0.22, 0.17),
                          complex_wf=True)
    nb = cs["nb"]
    psi32 = synth.make_psi(s, nb, 703).astype(np.complex64)
    mixed = api.Context(s, max_bands=nb, device=dev, precision="mixed")
    fp64 = api.Context(s, max_bands=nb, device=dev, precision="fp64")
    psi_rot = mixed.rayleigh_ritz(torch.from_numpy(psi32).to(dev))["psi_rot"]
    out = fp64.refine(psi_rot)
    torch.cuda.synchronize(dev)
    ref = O.refine(s, psi_rot.cpu().numpy())
    assert np.array_equal(out["psi"].cpu().numpy(), ref["psi"])
    assert _per_band(out["Hpsi"].cpu().numpy(), ref["Hpsi"], nb).max() <= REL
    assert np.max(np.abs(out["eps"].cpu().numpy() - ref["eps"])) <= EPS_TOL
    assert np.max(np.abs(out["theta"].cpu().numpy() - ref["theta"])) <= EPS_TOL
    mixed.close()
    fp64.close()


def test_refine_argument_errors(dev):
    from paper_2310_14776_gb300 import api, _lib
    s = synth.make_system((16, 16, 16), (8.0, 8.0, 8.0), 2, synth.PSET_SP, seed=710)
    mixed = api.Context(s, max_bands=4, device=dev, precision="mixed")
    fp64 = api.Context(s, max_bands=4, device=dev, precision="fp64")
    psi32 = torch.from_numpy(synth.make_psi(s, 4, 711).astype(np.float32)).to(dev)
    with pytest.raises(ValueError):
        mixed.refine(psi32)
    with pytest.raises(ValueError):
        fp64.refine(psi32.double())
    # the C entry point itself rejects a mixed context
    z = None
    rc = mixed.lib.pawfd_refine(mixed._h, psi32.data_ptr(), 4, z, z, z, z, z, z, z, z, z, z)
    assert _lib.ERRORS[rc] == "PAWFD_EINVAL"
    # more bands than the context holds
    with pytest.raises(_lib.PawFDError):
        fp64.refine(torch.cat([psi32, psi32]))
    mixed.close()
    fp64.close()
