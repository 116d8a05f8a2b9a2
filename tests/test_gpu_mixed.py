"""GPU parity of the mixed form (FP32 band arrays) against the FP64 oracle.

The oracle runs in FP64 on exactly the FP32-rounded inputs, so every difference is
arithmetic error of the mixed path.  Tolerances are rounding bounds derived here:

* H psi / S psi, per band 2-norm:  |err| <= 24 u (|| |T| |psi| + |v'| |psi| || + 64 ||N psi||)
  with u = 2^-24, |T| the stencil with absolute weights (each output is a chain of at most
  19 FP32 fused multiply-adds, so gamma_19 < 20 u, with margin), v' the shifted potential,
  and N psi the nonlocal part (box sums of at most a few thousand FP32 terms; the factor 64
  covers gamma_n for the projection and the back-add well above the random-walk size).
* eigenvalues: Weyl's bound for the pencil, |d eps_i| <= ||L^-1 dH L^-H|| + |eps_i| ||L^-1 dS L^-H||
  with dH, dS the measured Gram errors, times 1.5 for second-order terms.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2310_14776_gb300 import synth

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda:0")


def fp32_inputs(system, nb, seed):
    psi = synth.make_psi(system, nb, seed)
    return psi.astype(np.complex64 if system.complex_wf else np.float32)


def abs_local_norms(system, psi):
    """|| |T| |psi| + |v'| |psi| || per band, from the stencil definition with absolute weights."""
    w = O.fd6_coefficients()
    a = np.abs(psi).astype(np.float64)
    out = np.zeros_like(a)
    centre = 0.0
    for c in range(3):
        h2 = system.h[c] ** 2
        centre += 0.5 * abs(w[0]) / h2
        ax = 3 - c
        for m in (1, 2, 3):
            out += 0.5 * abs(w[m]) / h2 * (np.roll(a, m, axis=ax) + np.roll(a, -m, axis=ax))
    out += (np.abs(system.vloc) + centre)[None] * a
    return np.linalg.norm(out.reshape(len(psi), -1), axis=1)


def band_err(got, ref, nb):
    return np.linalg.norm((got.astype(ref.dtype) - ref).reshape(nb, -1), axis=1)


def weyl_bound(H_ref, S_ref, dH, dS, eps):
    L = np.linalg.cholesky(0.5 * (S_ref + S_ref.conj().T))
    Li = np.linalg.inv(L)
    nh = np.linalg.norm(Li @ dH @ Li.conj().T, 2)
    ns = np.linalg.norm(Li @ dS @ Li.conj().T, 2)
    return nh + np.abs(eps) * ns


CASES = {
    "gamma": dict(n=(24, 24, 24), cell=(10.0, 10.0, 10.0), natoms=2, pset=synth.PSET_SP, nb=16, cplx=False),
    "bloch": dict(n=(36, 30, 28), cell=(13.6, 11.3, 10.6), natoms=6, pset=synth.PSET_SPD2, nb=40, cplx=True),
    "ragged": dict(n=(45, 19, 13), cell=(9.0, 7.6, 5.2), natoms=4, pset=synth.PSET_SPD2, nb=9, cplx=True),
    # FP32 real with N1 % 4 == 0 (the float4 stencil): fewer rows than one y tile, odd N3
    "f32x4-small": dict(n=(28, 9, 11), cell=(7.0, 3.5, 4.4), natoms=3, pset=synth.PSET_SP, nb=7, cplx=False),
    # two x tiles (the second ragged) and three y tiles (the last ragged)
    "f32x4-ragged": dict(n=(132, 37, 10), cell=(26.0, 7.4, 4.0), natoms=5, pset=synth.PSET_SPD2, nb=3,
                         cplx=False),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_mixed_step_against_fp64_oracle(dev, case):
    from paper_2310_14776_gb300 import api
    cs = CASES[case]
    k = (0.31, -0.22, 0.17) if cs["cplx"] else (0.0, 0.0, 0.0)
    s = synth.make_system(cs["n"], cs["cell"], cs["natoms"], cs["pset"], seed=600, k=k, complex_wf=cs["cplx"])
    nb = cs["nb"]
    psi32 = fp32_inputs(s, nb, 601)
    psi64 = psi32.astype(np.complex128 if cs["cplx"] else np.float64)
    ctx = api.Context(s, max_bands=nb, device=dev, precision="mixed")
    res = ctx.rayleigh_ritz(torch.from_numpy(psi32).to(dev), keep_matrices=True)
    torch.cuda.synchronize(dev)
    ref = O.rayleigh_ritz(s, psi64)

    local = abs_local_norms(s, psi64)
    nonloc = np.linalg.norm((ref["Hpsi"] - O.kinetic_local(s, psi64)).reshape(nb, -1), axis=1)
    bound_H = 24 * U32 * (local + 64 * nonloc)
    errH = band_err(res["Hpsi"].cpu().numpy(), ref["Hpsi"], nb)
    assert np.all(errH <= bound_H), (errH / bound_H).max()
    snl = np.linalg.norm((ref["Spsi"] - psi64).reshape(nb, -1), axis=1)
    errS = band_err(res["Spsi"].cpu().numpy(), ref["Spsi"], nb)
    assert np.all(errS <= 24 * U32 * 64 * snl + 1e-30), (errS / (24 * U32 * 64 * snl)).max()

    Hnm, Snm = res["Hnm"].cpu().numpy(), res["Snm"].cpu().numpy()
    eps = res["eps"].cpu().numpy()
    bound = 1.5 * weyl_bound(ref["Hnm"], ref["Snm"], Hnm - ref["Hnm"], Snm - ref["Snm"], ref["eps"])
    deps = np.abs(eps - ref["eps"])
    assert np.all(deps <= bound + 1e-12), (deps / (bound + 1e-12)).max()
    # the mixed step still solves its own FP64 subspace problem to FP64 accuracy
    C = res["C"].cpu().numpy()
    Sh, Hh = 0.5 * (Snm + Snm.conj().T), 0.5 * (Hnm + Hnm.conj().T)
    assert np.allclose(C.conj().T @ Sh @ C, np.eye(nb), rtol=0, atol=1e-11)
    assert np.allclose(C.conj().T @ Hh @ C, np.diag(eps), rtol=0, atol=1e-11 * np.max(np.abs(eps)))
    # rotation: FP32 rounding of C and FP32 sums over nb terms
    rot = res["psi_rot"].cpu().numpy()
    ref_rot = O.rotate(psi64, C)
    bound_rot = (nb + 2) * U32 * np.linalg.norm(np.abs(psi64).reshape(nb, -1).T @ np.abs(C), axis=0)
    assert np.all(band_err(rot, ref_rot, nb) <= bound_rot)
    print("%s: max|d eps| = %.3e Ha, max rel |dHpsi| = %.3e" % (case, deps.max(),
          (errH / np.linalg.norm(ref["Hpsi"].reshape(nb, -1), axis=1)).max()))
    ctx.close()


def test_mixed_projections(dev):
    from paper_2310_14776_gb300 import api
    s = synth.make_system((30, 30, 30), (11.0, 11.0, 11.0), 5, synth.PSET_SPD2, seed=610, k=(0.2, 0.3, -0.1),
                          complex_wf=True)
    nb = 20
    psi32 = fp32_inputs(s, nb, 611)
    ctx = api.Context(s, max_bands=nb, device=dev, precision="mixed")
    P = ctx.project(torch.from_numpy(psi32).to(dev)).cpu().numpy()
    ref = O.project(s, psi32.astype(np.complex128))
    # each P entry is dV times a sum of at most npts FP32 products: |err| <= npts u dV sum|p||psi|
    npts = int(np.max(np.prod(s.box_n, axis=1)))
    scale = s.dV * np.max(np.abs(s.proj)) * npts * 1.0
    assert np.max(np.abs(P - ref)) <= 2 * npts * U32 * scale
    ctx.close()
