"""GPU parity of the plane-wave representation (pawfd_pw_*) against the oracle's PW functions.

FP64 (complex128 coefficients): the grid transforms, H C and S C per band within 1e-12
relative of the oracle's (numpy FFTs, the oracle's nonlocal term), with and without an energy
cutoff, and the eigenvalues of a plane-wave Rayleigh-Ritz step within 1e-10 Ha.  FP32
(complex64): each of the three FFT passes rounds every value a few times (radix-4/3/5
butterflies, twiddle products), so the error is bounded by a small multiple of u log2(K) of
the result's norm (u = 2^-24); the bar below is 8 u log2(K) per band, with the nonlocal FP32 box
sums inside it.  Grids cover radices 4, 2, 3 and 5, ragged tile edges (x not a multiple of the
line tile) and projector boxes larger than the cell.
"""
import math

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
    "bloch-30x24x20": dict(n=(30, 24, 20), cell=(11.3, 9.0, 7.5), natoms=4, pset=synth.PSET_SPD2, nb=7,
                           k=(0.31, -0.22, 0.17)),
    "selfwrap-6x5x4": dict(n=(6, 5, 4), cell=(3.0, 2.6, 2.2), natoms=2, pset=synth.PSET_SP, nb=3,
                           k=(0.5, 0.7, -0.3)),
    "gamma-48c": dict(n=(48, 48, 48), cell=(18.0, 18.0, 18.0), natoms=6, pset=synth.PSET_SPD2, nb=5,
                      k=(0.0, 0.0, 0.0)),
    "radix5-40x25x12": dict(n=(40, 25, 12), cell=(15.0, 9.4, 4.5), natoms=3, pset=synth.PSET_SPD2, nb=4,
                            k=(0.12, 0.05, -0.2)),
}


def system_of(case, seed=950):
    cs = CASES[case]
    return synth.make_system(cs["n"], cs["cell"], cs["natoms"], cs["pset"], seed=seed, k=cs["k"], complex_wf=True)


def per_band(got, ref, nb):
    got, ref = got.reshape(nb, -1), ref.reshape(nb, -1)
    return np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)


@pytest.mark.parametrize("case", sorted(CASES))
def test_pw_grid_transforms(dev, case):
    from paper_2310_14776_gb300 import api
    s = system_of(case)
    nb = CASES[case]["nb"]
    C = synth.make_psi(s, nb, 951)
    ctx = api.Context(s, max_bands=nb, device=dev)
    Cd = torch.from_numpy(C).to(dev)
    psi = ctx.pw_to_grid(Cd)
    back = ctx.pw_from_grid(psi)
    torch.cuda.synchronize(dev)
    assert per_band(psi.cpu().numpy(), O.pw_to_grid(s, C), nb).max() <= REL
    assert per_band(back.cpu().numpy(), C, nb).max() <= REL
    ctx.close()


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("cut", [0.0, 0.35])
def test_pw_apply_against_oracle(dev, case, cut):
    from paper_2310_14776_gb300 import api
    s = system_of(case)
    nb = CASES[case]["nb"]
    C = synth.make_psi(s, nb, 952)
    ecut = cut * float(np.max(O.pw_kinetic(s)))
    if ecut > 0:
        C = C * (O.pw_kinetic(s) <= ecut)[None]
    ctx = api.Context(s, max_bands=nb, device=dev)
    Cd = torch.from_numpy(C).to(dev)
    HC = ctx.pw_apply(Cd, "H", ecut=ecut).cpu().numpy()
    SC = ctx.pw_apply(Cd, "S", ecut=ecut).cpu().numpy()
    ctx.close()
    refH = O.pw_apply(s, C, "H", ecut=ecut)
    refS = O.pw_apply(s, C, "S", ecut=ecut)
    assert per_band(HC, refH, nb).max() <= REL
    assert per_band(SC, refS, nb).max() <= REL
    if ecut > 0:
        outside = O.pw_kinetic(s) > ecut
        assert np.all(HC[:, outside] == 0) and np.all(SC[:, outside] == 0)


@pytest.mark.parametrize("case", ["bloch-30x24x20", "radix5-40x25x12"])
def test_pw_rayleigh_ritz_against_oracle(dev, case):
    # a Rayleigh-Ritz step in the plane-wave basis: pawfd_pw_apply_H / _S, the Hermitian Gram
    # matrices of the coefficient arrays and the subspace solve, against the oracle's
    from paper_2310_14776_gb300 import api
    s = system_of(case, seed=953)
    nb = 6
    ecut = 0.5 * float(np.max(O.pw_kinetic(s)))
    C = synth.make_psi(s, nb, 954) * (O.pw_kinetic(s) <= ecut)[None]
    ctx = api.Context(s, max_bands=nb, device=dev)
    Cd = torch.from_numpy(C).to(dev)
    HC = ctx.pw_apply(Cd, "H", ecut=ecut)
    SC = ctx.pw_apply(Cd, "S", ecut=ecut)
    Hnm = ctx.gram(Cd, HC, hermitian=True)
    Snm = ctx.gram(Cd, SC, hermitian=True)
    eps, Cv = ctx.subspace_diag(Hnm, Snm)
    ctx.close()
    refH = O.gram(C, O.pw_apply(s, C, "H", ecut=ecut), s.dV, nb)
    refS = O.gram(C, O.pw_apply(s, C, "S", ecut=ecut), s.dV, nb)
    ref_eps, _, _ = O.subspace_diag(refH, refS)
    assert np.max(np.abs(eps.cpu().numpy() - ref_eps)) <= EPS_TOL


def test_pw_plane_waves_closed_form_on_the_gpu(dev):
    # free system: unit coefficient vectors are eigenvectors with |k + G|^2 / 2
    from paper_2310_14776_gb300 import api
    k = (0.37, -0.21, 0.55)
    s = synth.build_system((20, 18, 16), (8.0, 7.2, 6.4), np.zeros((0, 3)), np.zeros((0, 3)), synth.PSET_SP, [], [],
                           k=k, complex_wf=True)
    js = [(0, 0, 0), (1, 0, 0), (0, 2, -1), (3, -4, 2), (-5, 4, 3), (9, -8, 7)]
    C = np.zeros((len(js), 16, 18, 20), complex)
    for b, j in enumerate(js):
        C[b, j[2] % 16, j[1] % 18, j[0] % 20] = 1.0
    ctx = api.Context(s, max_bands=len(js), device=dev)
    HC = ctx.pw_apply(torch.from_numpy(C).to(dev), "H").cpu().numpy()
    ctx.close()
    for b, j in enumerate(js):
        q = [k[c] + 2 * math.pi * j[c] / s.cell[c] for c in range(3)]
        lam = 0.5 * sum(v * v for v in q)
        assert np.max(np.abs(HC[b] - lam * C[b])) <= 1e-13 * max(lam, 1.0)


@pytest.mark.parametrize("case", ["bloch-30x24x20", "radix5-40x25x12"])
def test_pw_fp32_against_fp64_oracle(dev, case):
    from paper_2310_14776_gb300 import api
    s = system_of(case, seed=955)
    nb = 5
    C32 = synth.make_psi(s, nb, 956).astype(np.complex64)
    C64 = C32.astype(np.complex128)
    ctx = api.Context(s, max_bands=nb, device=dev, precision="mixed")
    Cd = torch.from_numpy(C32).to(dev)
    HC = ctx.pw_apply(Cd, "H").cpu().numpy()
    SC = ctx.pw_apply(Cd, "S").cpu().numpy()
    ctx.close()
    bar = 8 * 2.0 ** -24 * math.log2(s.npoints)
    assert per_band(HC.astype(np.complex128), O.pw_apply(s, C64, "H"), nb).max() <= bar
    assert per_band(SC.astype(np.complex128), O.pw_apply(s, C64, "S"), nb).max() <= bar


def test_pw_rejects_real_contexts_and_other_grid_factors(dev):
    from paper_2310_14776_gb300 import api, _lib
    s = synth.make_system((12, 10, 8), (5.0, 4.0, 3.5), 1, synth.PSET_SP, seed=957)
    ctx = api.Context(s, max_bands=2, device=dev)
    x = torch.zeros((2,) + tuple(s.n[::-1]), dtype=torch.float64, device=dev)
    rc = ctx.lib.pawfd_pw_to_grid(ctx._h, x.data_ptr(), 2, x.data_ptr() + 8)
    assert _lib.ERRORS[rc] == "PAWFD_EINVAL"
    ctx.close()
    s7 = synth.make_system((14, 10, 8), (5.0, 4.0, 3.5), 1, synth.PSET_SP, seed=958, k=(0.1, 0.0, 0.0),
                           complex_wf=True)
    ctx = api.Context(s7, max_bands=2, device=dev)
    C = torch.zeros((2,) + tuple(s7.n[::-1]), dtype=torch.complex128, device=dev)
    with pytest.raises(_lib.PawFDError):
        ctx.pw_to_grid(C)
    ctx.close()
