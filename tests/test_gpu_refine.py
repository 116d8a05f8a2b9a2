"""GPU parity of the final refinement of the mixed form against the FP64 oracle.

The refinement is FP64 arithmetic on FP32 inputs promoted exactly, so its outputs are held
to the FP64 bars: H psi' per band 1e-12 relative, refined eigenvalues and Rayleigh quotients
1e-10 Ha, residual norms 1e-9 relative.  The end-to-end claim of the mixed form (refined
eigenvalues against the oracle's FP64 step on the original FP32 input) is checked against a
Weyl bound computed from the oracle's own projected pencil, and printed.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2310_14776_gb300 import synth

pytestmark = pytest.mark.gpu

REL = 1e-12
EPS_TOL = 1e-10


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
    rr = mixed.rayleigh_ritz(torch.from_numpy(psi32).to(dev))
    psi_rot = rr["psi_rot"]
    out = fp64.refine(psi_rot)
    torch.cuda.synchronize(dev)
    lo = psi_rot.cpu().numpy()
    ref = O.refine(s, lo)

    # steps 1-2: promotion is exact, H psi' in FP64
    assert np.array_equal(out["psi"].cpu().numpy(), ref["psi"])
    got = out["Hpsi"].cpu().numpy().reshape(nb, -1)
    want = ref["Hpsi"].reshape(nb, -1)
    assert np.all(np.linalg.norm(got - want, axis=1) <= REL * np.linalg.norm(want, axis=1))
    gs = out["Spsi"].cpu().numpy().reshape(nb, -1)
    ws = ref["Spsi"].reshape(nb, -1)
    assert np.all(np.linalg.norm(gs - ws, axis=1) <= REL * np.linalg.norm(ws, axis=1))
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

    # end to end: refined eigenvalues against the oracle's FP64 step on the original input.
    # In the basis psi C of the exact step the pencil is (diag(eps0), I); psi' differs from
    # psi C by the FP32 rounding of the rotation, and Weyl's bound for the pencil turns the
    # measured pencil difference into an eigenvalue bound.
    first = O.rayleigh_ritz(s, psi32.astype(np.complex128 if cs["cplx"] else np.float64))
    eps0 = first["eps"]
    dH = Hh - np.diag(eps0)
    dS = Sh - np.eye(nb)
    bound = 1.5 * (np.linalg.norm(dH, 2) + np.abs(eps0) * np.linalg.norm(dS, 2)) + 1e-12
    dev_e2e = np.abs(eps - eps0)
    assert np.all(dev_e2e <= bound), (dev_e2e / bound).max()
    print("%s: max|eps_refined - eps_fp64| = %.2e Ha (Weyl bound %.2e), max|eps_mixed - eps_fp64| = %.2e Ha,"
          " max resid %.2e" % (case, dev_e2e.max(), bound.max(), np.abs(rr["eps"].cpu().numpy() - eps0).max(),
                               resid.max()))
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
    rc = mixed.lib.pawfd_refine(mixed._h, psi32.data_ptr(), 4, z, z, z, z, z, z, z, z, z)
    assert _lib.ERRORS[rc] == "PAWFD_EINVAL"
    # more bands than the context holds
    with pytest.raises(_lib.PawFDError):
        fp64.refine(torch.cat([psi32, psi32]))
    mixed.close()
    fp64.close()
