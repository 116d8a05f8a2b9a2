"""Pins of the FP64 CPU oracle against what the mathematics fixes (no GPU).

Each test checks the oracle against something other than itself: the order of accuracy
of the finite-difference weights, the closed-form discrete spectrum of plane waves,
Hermiticity, the nonlocal Gram identity, the norm-conserving special cases, exact
discrete translations, Bloch periodicity and time reversal, a dense brute-force
construction of H and S on tiny grids diagonalised by LAPACK, and LAPACK itself for the
Cholesky and eigensolver pieces.  The paper prints no worked example for this path, so
nothing here is a printed value except the published finite-difference weights.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg

from oracle import oracle as O
from paper_2310_14776_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden_weights():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "fd6_weights.txt")) if l.strip() and not l.startswith("#")]
    return np.array([int(r[1]) / int(r[2]) for r in rows])


def free_system(n, cell, k=(0.0, 0.0, 0.0), complex_wf=False, vloc=None):
    s = synth.build_system(n, cell, np.zeros((0, 3)), np.zeros((0, 3)), synth.PSET_SP, [], [], k=k,
                           complex_wf=complex_wf)
    if vloc is not None:
        s.vloc = vloc
    return s


def small_system(n=(12, 11, 10), cell=(6.0, 5.5, 5.2), natoms=3, pset=synth.PSET_SP, seed=11, complex_wf=False,
                 k=None):
    if k is None:
        k = (0.31, -0.17, 0.23) if complex_wf else (0.0, 0.0, 0.0)
    return synth.make_system(n, cell, natoms, pset, seed, k=k, complex_wf=complex_wf)


def rand_psi(system, nb, seed):
    return synth.make_psi(system, nb, seed)


def inner(system, a, b):
    """dV sum_r conj(a) b over whole arrays."""
    return system.dV * np.vdot(a.reshape(-1), b.reshape(-1))


# ------------------------------------------------------------------------------------------
# finite-difference weights
# ------------------------------------------------------------------------------------------

def test_weights_match_published_table():
    assert np.allclose(O.fd6_coefficients(), golden_weights(), rtol=0, atol=1e-16)


def test_weights_solve_taylor_conditions():
    # symmetric weights w_0..w_3 with sum_m w_|m| m^(2j) = 2 delta_{j,1} for j = 0..3 (exact f'' of x^2)
    A = np.array([[1.0, 2.0, 2.0, 2.0]] + [[0.0] + [2.0 * m ** (2 * j) for m in (1, 2, 3)] for j in (1, 2, 3)])
    w = np.linalg.solve(A, np.array([0.0, 2.0, 0.0, 0.0]))
    assert np.allclose(O.fd6_coefficients(), w, rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_kinetic_order_of_accuracy(axis):
    # plane wave cos(G x_c): the discrete kinetic eigenvalue approaches G^2/2 with error ~ theta^6
    errs = []
    for N in (16, 32):
        n = [6, 6, 6]
        n[axis] = N
        L = [3.0, 3.0, 3.0]
        L[axis] = 8.0
        s = free_system(n, L)
        x = np.arange(N) * (L[axis] / N)
        G = 2 * math.pi / L[axis]
        f1 = np.cos(G * x)
        shape = [1, 1, 1]
        shape[2 - axis] = N
        psi = np.broadcast_to(f1.reshape(shape), (n[2], n[1], n[0])).copy()[None]
        out = O.kinetic_local(s, psi)
        lam = np.vdot(psi, out).real / np.vdot(psi, psi).real
        errs.append(abs(lam / (G * G / 2) - 1.0))
    assert errs[0] < 1e-4
    assert 40.0 < errs[0] / errs[1] < 80.0      # order 6: halving h divides the error by 2^6


def test_constant_is_annihilated():
    s = free_system((9, 8, 7), (4.0, 4.0, 4.0))
    out = O.kinetic_local(s, np.ones((1, 7, 8, 9)))
    assert np.max(np.abs(out)) < 1e-12


# ------------------------------------------------------------------------------------------
# I1: closed-form spectrum of plane waves
# ------------------------------------------------------------------------------------------

def plane_wave_eigenvalue(system, q):
    """sum_c 1/(2 h_c^2) [-w0 - 2 sum_m w_m cos(m q_c h_c)] for wave vector q = k + G."""
    w = golden_weights()
    lam = 0.0
    for c in range(3):
        h = system.h[c]
        lam += (-w[0] - 2.0 * sum(w[m] * math.cos(m * q[c] * h) for m in (1, 2, 3))) / (2.0 * h * h)
    return lam


def grid_coords(system):
    z, y, x = np.meshgrid(*[np.arange(system.n[c]) * system.h[c] for c in (2, 1, 0)], indexing="ij")
    return x, y, z


@pytest.mark.parametrize("complex_wf", [False, True])
def test_plane_wave_spectrum(complex_wf):
    k = (0.37, -0.21, 0.55) if complex_wf else (0.0, 0.0, 0.0)
    s = free_system((10, 9, 8), (5.0, 4.6, 4.1), k=k, complex_wf=complex_wf)
    x, y, z = grid_coords(s)
    for j in [(0, 0, 0), (1, 0, 0), (0, 2, -1), (3, -4, 2), (5, 4, 4)]:
        q = [k[c] + 2 * math.pi * j[c] / s.cell[c] for c in range(3)]
        phase = q[0] * x + q[1] * y + q[2] * z
        lam = plane_wave_eigenvalue(s, q)
        waves = [np.exp(1j * phase)] if complex_wf else [np.cos(phase), np.sin(phase)]
        for wv in waves:
            if np.max(np.abs(wv)) < 0.5:
                continue
            out = O.kinetic_local(s, wv[None])
            assert np.max(np.abs(out[0] - lam * wv)) <= 1e-13 * max(abs(lam), 1.0) * 10


def test_plane_wave_block_rayleigh_ritz():
    # RR on a block of plane waves returns exactly their closed-form eigenvalues
    k = (0.2, 0.1, -0.3)
    s = free_system((8, 8, 8), (4.0, 4.0, 4.0), k=k, complex_wf=True)
    x, y, z = grid_coords(s)
    js = [(0, 0, 0), (1, 0, 0), (0, -1, 0), (0, 0, 1), (1, 1, 0), (2, -1, 1), (-3, 2, 2), (4, 0, -2)]
    lams, psi = [], []
    for j in js:
        q = [k[c] + 2 * math.pi * j[c] / s.cell[c] for c in range(3)]
        psi.append(np.exp(1j * (q[0] * x + q[1] * y + q[2] * z)))
        lams.append(plane_wave_eigenvalue(s, q))
    psi = np.array(psi)
    mix = np.linalg.qr(synth.uniform(5, 1, 64, -1, 1).reshape(8, 8))[0]
    psi = np.einsum("nm,nzyx->mzyx", mix, psi)          # hide the eigenvectors in a random basis
    res = O.rayleigh_ritz(s, psi)
    assert np.allclose(res["eps"], np.sort(lams), rtol=0, atol=1e-11)


# ------------------------------------------------------------------------------------------
# I2 / I3 / I4: Hermiticity, nonlocal identity, norm-conserving special cases
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("complex_wf", [False, True])
def test_hermiticity_of_H_and_S(complex_wf):
    s = small_system(complex_wf=complex_wf, pset=synth.PSET_SPD2)
    phi = rand_psi(s, 3, 21)
    psi = rand_psi(s, 3, 22)
    Hphi, _ = O.apply_H(s, phi)
    Hpsi, _ = O.apply_H(s, psi)
    Sphi, _ = O.apply_S(s, phi)
    Spsi, _ = O.apply_S(s, psi)
    for b in range(3):
        a1 = inner(s, phi[b], Hpsi[b])
        a2 = np.conj(inner(s, psi[b], Hphi[b]))
        assert abs(a1 - a2) <= 1e-13 * abs(inner(s, phi[b], phi[b])) * 50
        b1 = inner(s, phi[b], Spsi[b])
        b2 = np.conj(inner(s, psi[b], Sphi[b]))
        assert abs(b1 - b2) <= 1e-13 * abs(inner(s, phi[b], phi[b]))
    # S positive definite on this block
    Snm = O.gram(psi, Spsi, s.dV, 3)
    assert np.all(np.linalg.eigvalsh(0.5 * (Snm + Snm.conj().T)) > 0)


def atom_blocks(system, flat):
    I = system.pset.count
    return [flat[a * I * I:(a + 1) * I * I].reshape(I, I) for a in range(system.natoms)]


@pytest.mark.parametrize("complex_wf", [False, True])
def test_nonlocal_gram_identity(complex_wf):
    # dV phi^H (G dH P_psi) = P_phi^H dH P_psi: projection and back-add are adjoint
    s = small_system(complex_wf=complex_wf, natoms=4, pset=synth.PSET_SPD2)
    phi = rand_psi(s, 4, 31)
    psi = rand_psi(s, 5, 32)
    Hpsi, Ppsi = O.apply_H(s, psi)
    nonlocal_part = Hpsi - O.kinetic_local(s, psi)
    Pphi = O.project(s, phi)
    I = s.pset.count
    K = s.npoints
    lhs = s.dV * phi.reshape(4, K).conj() @ nonlocal_part.reshape(5, K).T
    rhs = np.zeros((4, 5), dtype=lhs.dtype)
    for a, dH in enumerate(atom_blocks(s, s.dH)):
        rows = slice(a * I, (a + 1) * I)
        rhs += Pphi[rows].conj().T @ dH @ Ppsi[rows]
    assert np.allclose(lhs, rhs, rtol=0, atol=1e-12 * np.max(np.abs(rhs)))


def test_ncpp_and_zero_corrections():
    s = small_system(complex_wf=True, natoms=3)
    psi = rand_psi(s, 4, 41)
    # dS = 0: S psi = psi, so S_nm = dV psi^H psi
    s0 = synth.with_corrections(s, dS=np.zeros_like(s.dS))
    Spsi, _ = O.apply_S(s0, psi)
    assert np.array_equal(Spsi, psi)
    # dH = dS = 0: H equals the atom-free operator
    s00 = synth.with_corrections(s, dH=np.zeros_like(s.dH), dS=np.zeros_like(s.dS))
    Hpsi, _ = O.apply_H(s00, psi)
    free = O.kinetic_local(synth.without_atoms(s), psi)
    assert np.array_equal(Hpsi, free)
    # H - (T + v) has rank <= Ip
    Hfull, _ = O.apply_H(s, rand_psi(s, 40, 42))
    diff = (Hfull - O.kinetic_local(s, rand_psi(s, 40, 42))).reshape(40, -1)
    sv = np.linalg.svd(diff, compute_uv=False)
    assert np.sum(sv > 1e-10 * sv[0]) <= s.nproj_total


# ------------------------------------------------------------------------------------------
# I5 / I6: exact discrete translation, Bloch periodicity, time reversal
# ------------------------------------------------------------------------------------------

def bloch_roll(system, psi, shift):
    """psi'(r) = psi(r - shift*h) for a Bloch function: wrapped samples pick up exp(-i k_c L_c)."""
    out = psi
    for c, sc in enumerate(shift):
        ax = 3 - c
        N = system.n[c]
        out = np.roll(out, sc, axis=ax)
        if sc and system.complex_wf:
            ph = np.exp(-1j * system.k[c] * system.cell[c])
            idx = [slice(None)] * out.ndim
            idx[ax] = slice(0, sc)
            out[tuple(idx)] *= ph
    return out


@pytest.mark.parametrize("complex_wf", [False, True])
def test_translation_by_grid_vector(complex_wf):
    s = small_system(complex_wf=complex_wf, natoms=3, pset=synth.PSET_SPD2)
    shift = (3, 2, 5)
    d = np.array([shift[c] * s.h[c] for c in range(3)])
    I = s.pset.count
    t = synth.build_system(s.n, s.cell, s.pos + d, s.wells + d, s.pset, atom_blocks(s, s.dH), atom_blocks(s, s.dS),
                           k=s.k, complex_wf=complex_wf)
    psi = rand_psi(s, 3, 51)
    Hpsi, _ = O.apply_H(s, psi)
    Ht, _ = O.apply_H(t, bloch_roll(s, psi, shift))
    assert np.allclose(Ht, bloch_roll(s, Hpsi, shift), rtol=0, atol=1e-12 * np.max(np.abs(Hpsi)))
    r1 = O.rayleigh_ritz(s, psi)
    r2 = O.rayleigh_ritz(t, bloch_roll(s, psi, shift))
    assert np.allclose(r1["eps"], r2["eps"], rtol=0, atol=1e-11)


def test_bloch_vector_periodicity_and_time_reversal():
    s = small_system(complex_wf=True, natoms=3)
    psi = rand_psi(s, 3, 61)
    Hpsi, _ = O.apply_H(s, psi)
    k2 = tuple(s.k[c] + (2 * math.pi / s.cell[c] if c == 1 else 0.0) for c in range(3))
    s2 = synth.build_system(s.n, s.cell, s.pos, s.wells, s.pset, atom_blocks(s, s.dH), atom_blocks(s, s.dS), k=k2,
                            complex_wf=True)
    H2, _ = O.apply_H(s2, psi)
    assert np.allclose(H2, Hpsi, rtol=0, atol=1e-12 * np.max(np.abs(Hpsi)))
    sm = synth.build_system(s.n, s.cell, s.pos, s.wells, s.pset, atom_blocks(s, s.dH), atom_blocks(s, s.dS),
                            k=tuple(-v for v in s.k), complex_wf=True)
    Hm, _ = O.apply_H(sm, psi.conj())
    assert np.allclose(Hm, Hpsi.conj(), rtol=0, atol=1e-12 * np.max(np.abs(Hpsi)))


# ------------------------------------------------------------------------------------------
# I7: dense brute force on tiny grids
# ------------------------------------------------------------------------------------------

def dense_operators(system):
    """H and S as explicit K x K matrices: Kronecker sums of 1-D Bloch-twisted circulants,
    diag(v), and dV G dX G^H with G[r, i] = sum_T p_i(r + T - R_a) exp(-i k.T) over images T."""
    w = golden_weights()
    n, L, k, h = system.n, system.cell, system.k, system.h

    def second_diff(N, hc, kL):
        D = np.zeros((N, N), complex)
        for i in range(N):
            for m in range(-3, 4):
                t, j = divmod(i + m, N)
                D[i, j] += w[abs(m)] / hc ** 2 * np.exp(1j * kL * t)
        return D

    Dx, Dy, Dz = (second_diff(n[c], h[c], k[c] * L[c]) for c in range(3))
    Ix, Iy, Iz = (np.eye(n[c]) for c in range(3))
    T = -0.5 * (np.kron(Dz, np.kron(Iy, Ix)) + np.kron(Iz, np.kron(Dy, Ix)) + np.kron(Iz, np.kron(Iy, Dx)))
    x, y, z = (a.reshape(-1) for a in grid_coords(system))
    K = system.npoints
    I = system.pset.count
    G = np.zeros((K, system.natoms * I), complex)
    rc = system.pset.rcut
    for a in range(system.natoms):
        R = system.pos[a]
        reach = [int(math.ceil((rc + L[c]) / L[c])) + 1 for c in range(3)]
        for t1 in range(-reach[0], reach[0] + 1):
            for t2 in range(-reach[1], reach[1] + 1):
                for t3 in range(-reach[2], reach[2] + 1):
                    T_ = (t1 * L[0], t2 * L[1], t3 * L[2])
                    vals = synth.projector_values(system.pset, x + T_[0] - R[0], y + T_[1] - R[1], z + T_[2] - R[2])
                    G[:, a * I:(a + 1) * I] += vals.T * np.exp(-1j * (k[0] * T_[0] + k[1] * T_[1] + k[2] * T_[2]))
    dH = scipy.linalg.block_diag(*atom_blocks(system, system.dH)) if system.natoms else np.zeros((0, 0))
    dS = scipy.linalg.block_diag(*atom_blocks(system, system.dS)) if system.natoms else np.zeros((0, 0))
    H = T + np.diag(system.vloc.reshape(-1)) + system.dV * G @ dH @ G.conj().T
    S = np.eye(K) + system.dV * G @ dS @ G.conj().T
    if not system.complex_wf:
        assert np.max(np.abs(H.imag)) < 1e-12 and np.max(np.abs(S.imag)) < 1e-12
        H, S = H.real, S.real
    return H, S


TINY = {
    # the 8^3 grid of the dense brute-force check (512 x 512 pencils), s + p + d projectors
    "cube8": dict(n=(8, 8, 8), cell=(4.2, 4.2, 4.2), natoms=2, pset=synth.PSET_SPD2, seed=74, complex_wf=False),
    "cube8-bloch": dict(n=(8, 8, 8), cell=(4.2, 4.2, 4.2), natoms=2, pset=synth.PSET_SPD2, seed=75,
                        complex_wf=True, k=(0.33, -0.41, 0.27)),
    # boxes smaller than the cell, Bloch phases, s + p + d projectors
    "bloch": dict(n=(8, 7, 6), cell=(6.0, 5.6, 5.1), natoms=2, pset=synth.PSET_SPD2, seed=71, complex_wf=True,
                  k=(0.41, -0.29, 0.13)),
    # boxes larger than the cell (each box wraps onto itself), real Gamma point
    "selfwrap": dict(n=(6, 6, 6), cell=(3.0, 3.0, 3.0), natoms=2, pset=synth.PSET_SP, seed=72, complex_wf=False),
    # boxes larger than the cell with a Bloch phase
    "selfwrap-bloch": dict(n=(6, 5, 6), cell=(3.0, 2.6, 3.1), natoms=1, pset=synth.PSET_SPD2, seed=73,
                           complex_wf=True, k=(0.5, 0.7, -0.3)),
}


@pytest.mark.parametrize("case", sorted(TINY))
def test_dense_bruteforce_apply(case):
    s = small_system(**TINY[case])
    H, S = dense_operators(s)
    psi = rand_psi(s, 4, 81)
    K = s.npoints
    Hpsi, _ = O.apply_H(s, psi)
    Spsi, _ = O.apply_S(s, psi)
    ref_H = (H @ psi.reshape(4, K).T).T
    ref_S = (S @ psi.reshape(4, K).T).T
    assert np.allclose(Hpsi.reshape(4, K), ref_H, rtol=0, atol=1e-12 * np.max(np.abs(ref_H)))
    assert np.allclose(Spsi.reshape(4, K), ref_S, rtol=0, atol=1e-12 * np.max(np.abs(ref_S)))


@pytest.mark.parametrize("case", ["selfwrap", "selfwrap-bloch", "cube8", "cube8-bloch"])
def test_dense_bruteforce_full_spectrum(case):
    # RR over the full grid basis (every band a unit vector) is the full generalized eigenproblem
    s = small_system(**TINY[case])
    H, S = dense_operators(s)
    K = s.npoints
    dt = np.complex128 if s.complex_wf else np.float64
    psi = np.eye(K, dtype=dt).reshape(K, s.n[2], s.n[1], s.n[0])
    res = O.rayleigh_ritz(s, psi)
    exact = scipy.linalg.eigh(H, S, eigvals_only=True)
    assert np.max(np.abs(res["eps"] - exact)) < 1e-11 * max(1.0, np.max(np.abs(exact)))


def test_ritz_values_interlace_exact_spectrum():
    s = small_system(**TINY["bloch"])
    H, S = dense_operators(s)
    exact = scipy.linalg.eigh(H, S, eigvals_only=True)
    psi = rand_psi(s, 16, 91)
    res = O.rayleigh_ritz(s, psi)
    assert np.all(res["eps"] >= exact[:16] - 1e-10)
    # and they are the eigenvalues of the projected dense pencil
    K = s.npoints
    Y = psi.reshape(16, K).T
    ritz = scipy.linalg.eigh(s.dV * Y.conj().T @ H @ Y, s.dV * Y.conj().T @ S @ Y, eigvals_only=True)
    assert np.allclose(res["eps"], ritz, rtol=0, atol=1e-10)


# ------------------------------------------------------------------------------------------
# I8: Rayleigh-Ritz invariants
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("complex_wf", [False, True])
def test_rayleigh_ritz_invariants(complex_wf):
    s = small_system(complex_wf=complex_wf, pset=synth.PSET_SPD2, natoms=3)
    nb = 12
    psi = rand_psi(s, nb, 101)
    res = O.rayleigh_ritz(s, psi)
    C, eps = res["C"], res["eps"]
    assert np.all(np.diff(eps) >= 0)
    Sh = 0.5 * (res["Snm"] + res["Snm"].conj().T)
    Hh = 0.5 * (res["Hnm"] + res["Hnm"].conj().T)
    assert np.allclose(C.conj().T @ Sh @ C, np.eye(nb), rtol=0, atol=1e-12)
    assert np.allclose(C.conj().T @ Hh @ C, np.diag(eps), rtol=0, atol=1e-12 * np.max(np.abs(eps)))
    # phase rule: each column's largest-magnitude entry is real and positive
    for m in range(nb):
        i = np.argmax(np.abs(C[:, m]))
        assert abs(np.imag(C[i, m])) < 1e-14 and np.real(C[i, m]) > 0
    # invariance under psi -> psi M
    M = np.eye(nb) + 0.2 * synth.uniform(7, 1, nb * nb, -1, 1).reshape(nb, nb)
    res2 = O.rayleigh_ritz(s, np.einsum("nm,nzyx->mzyx", M, psi))
    assert np.allclose(res2["eps"], eps, rtol=0, atol=1e-10)
    # idempotence: RR of the rotated block gives the same values and a diagonal subspace problem
    res3 = O.rayleigh_ritz(s, res["psi_rot"])
    assert np.allclose(res3["eps"], eps, rtol=0, atol=1e-10)
    assert np.allclose(np.abs(res3["C"]), np.eye(nb), rtol=0, atol=1e-8)


# ------------------------------------------------------------------------------------------
# I9: dense pieces against LAPACK / BLAS
# ------------------------------------------------------------------------------------------

def _rand_herm(n, seed, cplx):
    A = synth.uniform(seed, 1, n * n, -1, 1).reshape(n, n)
    if cplx:
        A = A + 1j * synth.uniform(seed, 2, n * n, -1, 1).reshape(n, n)
    return 0.5 * (A + A.conj().T)


@pytest.mark.parametrize("cplx", [False, True])
def test_cholesky_against_lapack(cplx):
    A = _rand_herm(40, 3, cplx)
    S = A @ A.conj().T + 40 * np.eye(40)
    assert np.allclose(O.cholesky(S), np.linalg.cholesky(S), rtol=0, atol=1e-13)


def test_cholesky_reports_failing_column():
    S = np.eye(6)
    S[3, 3] = -1.0
    with pytest.raises(O.SubspaceError) as e:
        O.cholesky(S)
    assert e.value.code == -4


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("n", [1, 2, 17, 64])
def test_jacobi_against_lapack(cplx, n):
    A = _rand_herm(n, n, cplx)
    w, V, sweeps = O.jacobi_eigh(A)
    assert np.allclose(np.sort(w), np.linalg.eigvalsh(A), rtol=0, atol=1e-13 * max(1, n))
    assert np.allclose(A @ V, V * w, rtol=0, atol=1e-12 * max(1, n))
    assert np.allclose(V.conj().T @ V, np.eye(n), rtol=0, atol=1e-13 * max(1, n))


def test_jacobi_degenerate_spectrum():
    Q = np.linalg.qr(synth.uniform(9, 1, 400, -1, 1).reshape(20, 20))[0]
    d = np.array([1.0] * 7 + [2.0] * 6 + [3.0 + 1e-9 * i for i in range(7)])
    A = Q @ np.diag(d) @ Q.T
    w, V, _ = O.jacobi_eigh(0.5 * (A + A.T))
    assert np.allclose(np.sort(w), np.sort(d), rtol=0, atol=1e-13)


@pytest.mark.parametrize("cplx", [False, True])
def test_gram_and_rotate_against_blas(cplx):
    nb, K = 7, 1000
    A = synth.uniform(1, 1, nb * K, -1, 1).reshape(nb, K)
    B = synth.uniform(1, 2, nb * K, -1, 1).reshape(nb, K)
    C = synth.uniform(1, 3, nb * nb, -1, 1).reshape(nb, nb)
    if cplx:
        A = A + 1j * synth.uniform(2, 1, nb * K, -1, 1).reshape(nb, K)
        B = B + 1j * synth.uniform(2, 2, nb * K, -1, 1).reshape(nb, K)
        C = C + 1j * synth.uniform(2, 3, nb * nb, -1, 1).reshape(nb, nb)
    M = O.gram(A, B, 0.25, nb)
    assert np.allclose(M, 0.25 * A.conj() @ B.T, rtol=0, atol=1e-12)
    R = O.rotate(A, C)
    assert np.allclose(R, C.T @ A, rtol=0, atol=1e-12)


# ------------------------------------------------------------------------------------------
# the generator's setup functions (inputs, not the method)
# ------------------------------------------------------------------------------------------

def test_projector_functions_orthonormal():
    pset = synth.ProjectorSet(channels=((0, 0.5), (1, 0.5), (2, 0.5)), rcut=6.0)
    h = 0.06
    ax = np.arange(-60, 61) * h
    z, y, x = np.meshgrid(ax, ax, ax, indexing="ij")
    p = synth.projector_values(pset, x, y, z).reshape(pset.count, -1)
    ov = h ** 3 * p @ p.T
    assert np.allclose(ov, np.eye(pset.count), rtol=0, atol=2e-3)


# ------------------------------------------------------------------------------------------
# Final refinement of the mixed form (residual norms, Rayleigh quotients, second RR)
# ------------------------------------------------------------------------------------------

def test_refine_exact_eigenvectors_have_zero_residual():
    # real plane waves cos(G.r) of a free system are exact eigenvectors (I1): the refinement
    # returns their closed-form eigenvalues as eps and theta, and residuals at rounding level
    s = free_system((10, 9, 8), (5.0, 4.6, 4.1))
    x, y, z = grid_coords(s)
    V = s.cell[0] * s.cell[1] * s.cell[2]
    js = [(1, 0, 0), (0, 1, 1), (2, -1, 0), (1, 2, 3)]
    psi, lams = [], []
    for j in js:
        q = [2 * math.pi * j[c] / s.cell[c] for c in range(3)]
        psi.append(np.sqrt(2.0 / V) * np.cos(q[0] * x + q[1] * y + q[2] * z))
        lams.append(plane_wave_eigenvalue(s, q))
    order = np.argsort(lams)
    psi = np.array(psi)[order]
    lams = np.array(lams)[order]
    res = O.refine(s, psi)
    assert np.allclose(res["eps"], lams, rtol=0, atol=1e-11)
    assert np.allclose(res["theta"], lams, rtol=0, atol=1e-11)
    assert np.all(res["resid"] <= 1e-11 * lams.max())
    # the Rayleigh quotient does not depend on a band's norm (<psi|H|psi> / <psi|S|psi>)
    scaled = O.refine(s, psi * np.array([0.5, 2.0, 3.0, 0.25]).reshape((-1,) + (1,) * (psi.ndim - 1)))
    assert np.allclose(scaled["theta"], lams, rtol=0, atol=1e-11)


def test_refine_residual_of_mixed_plane_waves():
    # psi_1,2 = (w_a +- w_b)/sqrt(2) for orthonormal eigenvectors w_a, w_b with eigenvalues
    # l_a < l_b: both Rayleigh quotients are (l_a + l_b)/2, the second RR recovers l_a, l_b,
    # and the residuals taken with eps_n are |l_b - l_a|/sqrt(2) for both bands
    s = free_system((12, 10, 9), (6.0, 5.0, 4.5))
    x, y, z = grid_coords(s)
    V = s.cell[0] * s.cell[1] * s.cell[2]
    qa = [2 * math.pi * j / s.cell[c] for c, j in enumerate((1, 0, 0))]
    qb = [2 * math.pi * j / s.cell[c] for c, j in enumerate((1, 2, -1))]
    wa = np.sqrt(2.0 / V) * np.cos(qa[0] * x + qa[1] * y + qa[2] * z)
    wb = np.sqrt(2.0 / V) * np.cos(qb[0] * x + qb[1] * y + qb[2] * z)
    la, lb = plane_wave_eigenvalue(s, qa), plane_wave_eigenvalue(s, qb)
    assert la < lb
    psi = np.array([(wa + wb) / np.sqrt(2.0), (wa - wb) / np.sqrt(2.0)])
    res = O.refine(s, psi)
    assert np.allclose(res["theta"], [(la + lb) / 2] * 2, rtol=0, atol=1e-11)
    assert np.allclose(res["eps"], [la, lb], rtol=0, atol=1e-11)
    assert np.allclose(res["resid"], [(lb - la) / np.sqrt(2.0)] * 2, rtol=1e-11, atol=0)


@pytest.mark.parametrize("complex_wf", [False, True])
def test_refine_of_ritz_vectors_is_a_fixed_point(complex_wf):
    # a second RR on the (FP64) Ritz vectors of a first one reproduces its eigenvalues, and each
    # Rayleigh quotient equals its eigenvalue (the Ritz vectors diagonalize the projected pencil)
    s = small_system(complex_wf=complex_wf)
    first = O.rayleigh_ritz(s, rand_psi(s, 6, 21))
    res = O.refine(s, first["psi_rot"])
    assert np.allclose(res["eps"], first["eps"], rtol=0, atol=1e-11)
    assert np.allclose(res["theta"], first["eps"], rtol=0, atol=1e-11)
    # residual norms are those of the Ritz pairs: check one against the definition via H, S
    n = 3
    r = res["Hpsi"][n] - first["eps"][n] * res["Spsi"][n]
    assert abs(res["resid"][n] - math.sqrt(s.dV) * np.linalg.norm(r)) <= 1e-12 * res["resid"][n]


@pytest.mark.parametrize("case", ["selfwrap", "bloch"])
def test_refine_of_rotated_input_keeps_its_span(case):
    # refinement of a mixed step's INPUT bands with that step's C: psi' = psi C_lo keeps the span
    # of psi for any nonsingular C_lo, so the refined eps are the Ritz values of span(psi) under
    # the dense pencil (H, S), whatever C_lo is; with C_lo the eigenvector matrix of an exact
    # step the rotated bands are its Ritz vectors, so theta = eps and the residuals are those
    # of the Ritz pairs
    s = small_system(**TINY[case])
    H, S = dense_operators(s)
    n = 5
    psi = rand_psi(s, n, 31)
    lo = psi.astype(np.complex64 if s.complex_wf else np.float32)
    exact_in = lo.astype(np.complex128 if s.complex_wf else np.float64)
    ritz = _dense_ritz(s, H, S, exact_in, n)
    rng = np.random.default_rng(32)
    M = rng.standard_normal((n, n)) + 3.0 * np.eye(n)
    if s.complex_wf:
        M = M + 1j * rng.standard_normal((n, n))
    res = O.refine(s, lo, M)
    assert np.allclose(res["eps"], ritz, rtol=0, atol=1e-10 * max(1.0, np.max(np.abs(ritz))))
    assert np.allclose(res["psi"].reshape(n, -1), (exact_in.reshape(n, -1).T @ M).T, rtol=0, atol=1e-13 * n)
    C0 = O.rayleigh_ritz(s, exact_in)["C"]
    res0 = O.refine(s, lo, C0)
    assert np.allclose(res0["eps"], ritz, rtol=0, atol=1e-10 * max(1.0, np.max(np.abs(ritz))))
    assert np.allclose(res0["theta"], ritz, rtol=0, atol=1e-10 * max(1.0, np.max(np.abs(ritz))))
    Z = res0["psi"].reshape(n, -1).T
    R = H @ Z - (S @ Z) * res0["eps"][None, :]
    assert np.allclose(res0["resid"], np.sqrt(s.dV * np.sum(np.abs(R) ** 2, axis=0)), rtol=1e-9, atol=1e-12)
    # without C_lo the bands are refined as given (the FP32 bands' own span)
    plain = O.refine(s, lo)
    assert np.allclose(plain["eps"], ritz, rtol=0, atol=1e-10 * max(1.0, np.max(np.abs(ritz))))


# ------------------------------------------------------------------------------------------
# f-1: the block-Davidson step (the iterative eigensolver of the Kohn-Sham section; reading)
# ------------------------------------------------------------------------------------------

def _dense_ritz(s, H, S, X, nb):
    Y = X.reshape(nb, s.npoints).T
    return scipy.linalg.eigh(s.dV * Y.conj().T @ H @ Y, s.dV * Y.conj().T @ S @ Y, eigvals_only=True)


@pytest.mark.parametrize("precond", ["kinetic", "jacobi"])
@pytest.mark.parametrize("case", ["selfwrap", "bloch"])
def test_davidson_step_against_dense_operators(case, precond):
    # the corrections solve (T + sigma) corr = -R with the dense kinetic operator (kinetic
    # preconditioner) or are the weights times the dense residual (Jacobi), and the step's 2n
    # Ritz values are those of the dense pencil projected on X = [psi, corrections]
    s = small_system(**TINY[case])
    H, S = dense_operators(s)
    n, K = 4, s.npoints
    rr = O.rayleigh_ritz(s, rand_psi(s, n, 7))
    psi, eps = rr["psi_rot"], rr["eps"]
    st = O.davidson_step(s, psi, eps, precond=precond)
    Y = psi.reshape(n, K)
    R = (H @ Y.T).T - eps[:, None] * (S @ Y.T).T
    corr = st["X"].reshape(2 * n, K)[n:]
    if precond == "jacobi":
        w = O.davidson_weights(s, eps)
        assert np.all(w < 0)
        assert np.allclose(corr, w * R, rtol=0, atol=1e-11 * np.max(np.abs(w * R)))
    else:
        T, _ = dense_operators(free_system(s.n, s.cell, k=s.k, complex_wf=s.complex_wf,
                                           vloc=np.zeros_like(s.vloc)))
        lhs = (T @ corr.T).T + O.KINETIC_SHIFT * corr
        assert np.allclose(lhs, -R, rtol=0, atol=1e-11 * np.max(np.abs(R)))
    assert np.allclose(st["rnorm"], np.sqrt(s.dV * np.sum(np.abs(R) ** 2, axis=1)), rtol=1e-10, atol=0)
    ritz = _dense_ritz(s, H, S, st["X"], 2 * n)
    assert np.allclose(st["eps"], ritz, rtol=0, atol=1e-10 * max(1.0, np.max(np.abs(ritz))))
    # the output vectors are the n lowest Ritz vectors: S-orthonormal, with those Ritz values
    Z = st["psi_out"].reshape(n, K).T
    assert np.allclose(s.dV * Z.conj().T @ S @ Z, np.eye(n), rtol=0, atol=1e-10)
    assert np.allclose(s.dV * Z.conj().T @ H @ Z, np.diag(st["eps"][:n]), rtol=0, atol=1e-10 * np.max(np.abs(ritz)))


@pytest.mark.parametrize("case", ["selfwrap", "bloch"])
def test_davidson_iteration_converges_from_above(case):
    # Ritz values never fall below the exact eigenvalues (interlacing), never rise from one
    # step to the next (the new subspace contains the old vectors), and approach the exact
    # lowest eigenvalues while the residuals shrink
    s = small_system(**TINY[case])
    H, S = dense_operators(s)
    exact = scipy.linalg.eigh(H, S, eigvals_only=True)
    n = 4
    rr = O.rayleigh_ritz(s, rand_psi(s, n, 5))
    psi, eps = rr["psi_rot"], rr["eps"]
    err0 = None
    for it in range(40):
        st = O.davidson_step(s, psi, eps)
        new = st["eps"][:n]
        assert np.all(new >= exact[:n] - 1e-10)
        assert np.all(new <= eps + 1e-10)
        if it == 0:
            err0, r0 = np.sum(new - exact[:n]), st["rnorm"].max()
        psi, eps = st["psi_out"], new
    assert np.sum(eps - exact[:n]) < err0 / 50
    assert st["rnorm"].max() < r0 / 15


@pytest.mark.parametrize("complex_wf", [False, True])
def test_kinetic_symbol_and_preconditioner_on_bloch_waves(complex_wf):
    # T (the oracle's real-space stencil, Bloch boundary conditions) acting on a grid Bloch wave
    # e^{i(k+G).r} multiplies it by t(k + G); the preconditioner divides it by -(t + sigma)
    k = (0.37, -0.21, 0.55) if complex_wf else (0.0, 0.0, 0.0)
    s = free_system((10, 9, 8), (5.0, 4.4, 3.9), k=k, complex_wf=complex_wf, vloc=None)
    t = O.kinetic_symbol(s)
    z, y, x = np.meshgrid(*[np.arange(s.n[c]) * s.h[c] for c in (2, 1, 0)], indexing="ij")
    for j in [(0, 0, 0), (1, 0, 0), (3, -2, 1), (-4, 4, 3), (5, 4, -4)]:
        q = [s.k[c] + 2 * math.pi * j[c] / s.cell[c] for c in range(3)]
        wave = np.exp(1j * (q[0] * x + q[1] * y + q[2] * z))
        if not complex_wf:
            wave = wave.real
        tj = t[j[2] % s.n[2], j[1] % s.n[1], j[0] % s.n[0]]
        Tw = O.kinetic_local(s, wave[None])[0]
        assert np.allclose(Tw, tj * wave, rtol=0, atol=1e-10 * max(1.0, tj))
        P = O.kinetic_precondition(s, wave[None])[0]
        assert np.allclose(P, -wave / (tj + O.KINETIC_SHIFT), rtol=0, atol=1e-13)
    assert np.all(t >= -1e-12)


def test_davidson_weights_from_the_dense_diagonal():
    # d(r) is the diagonal of the dense T + v (Kronecker sums of the published weights, no
    # atoms), the floor a tenth of the diagonal of T alone; eps values on both sides of the
    # floor
    s = small_system(**TINY["bloch"])
    Tv, _ = dense_operators(free_system(s.n, s.cell, k=s.k, complex_wf=True, vloc=s.vloc))
    T0, _ = dense_operators(free_system(s.n, s.cell, k=s.k, complex_wf=True, vloc=np.zeros_like(s.vloc)))
    d = np.real(np.diag(Tv))
    t0 = np.real(np.diag(T0))
    assert np.allclose(t0, t0[0], rtol=1e-15, atol=0) and t0[0] > 0
    floor = t0[0] / 10
    eps = np.array([d.min() - 7.0, np.median(d) - floor, d.max() - 0.5 * floor, d.max() + 3.0])
    w = O.davidson_weights(s, eps)
    den = d[None, :] - eps[:, None]
    expect = -1.0 / np.maximum(den, floor)
    assert np.any(den > floor) and np.any(den < floor)
    assert np.allclose(w, expect, rtol=1e-13, atol=0)


def test_davidson_fixed_point_is_exact_eigenvectors():
    s = small_system(**TINY["bloch"])
    H, S = dense_operators(s)
    lam, V = scipy.linalg.eigh(H, S)
    n = 3
    psi = (V[:, :n].T / math.sqrt(s.dV)).reshape((n,) + tuple(s.n[::-1]))
    st = O.davidson_step(s, psi, lam[:n])
    assert np.max(st["rnorm"]) < 1e-10 * max(1.0, np.max(np.abs(lam[:n])))
    assert np.allclose(st["eps"][:n], lam[:n], rtol=0, atol=1e-10)


# ------------------------------------------------------------------------------------------
# f-2: pseudo density and atomic density matrices
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("complex_wf", [False, True])
def test_density_paw_charge_and_energy_identities(complex_wf):
    # for S-orthonormal bands, dV sum_r rho + sum_a Tr(D^a dS^a) = sum_n f_n (the PAW norm of
    # every band is 1), and sum_n f_n <psi_n|H|psi_n> = sum_n f_n dV <psi_n|(T + v) psi_n>
    # + sum_a Tr(D^a dH^a) (the expectation-value formula of the PAW section)
    s = small_system(complex_wf=complex_wf, k=(0.3, -0.2, 0.1) if complex_wf else (0.0, 0.0, 0.0))
    nb = 6
    rr = O.rayleigh_ritz(s, rand_psi(s, nb, 31))
    psi = rr["psi_rot"]
    f = np.linspace(2.0, 0.25, nb)
    rho = O.density(s, psi, f)
    P = O.project(s, psi)
    D = O.atomic_density(s, P, f)
    blocksD = atom_blocks(s, D)
    charge = s.dV * np.sum(rho) + sum(np.trace(Da @ dS) for Da, dS in zip(blocksD, atom_blocks(s, s.dS)))
    assert abs(charge - np.sum(f)) < 1e-12 * np.sum(f)
    T = O.kinetic_local(s, psi).reshape(nb, -1)
    local = sum(f[n] * s.dV * np.vdot(psi.reshape(nb, -1)[n], T[n]) for n in range(nb))
    nonlocal_ = sum(np.trace(Da @ dH) for Da, dH in zip(blocksD, atom_blocks(s, s.dH)))
    band = np.sum(f * rr["eps"])
    assert abs(local + nonlocal_ - band) < 1e-11 * max(1.0, abs(band))
    for Da in blocksD:
        assert np.allclose(Da, Da.conj().T, rtol=0, atol=1e-15 * max(1.0, np.max(np.abs(Da))))
        assert np.min(np.linalg.eigvalsh(Da)) > -1e-13 * max(1.0, np.max(np.abs(Da)))


def test_density_of_plane_waves_is_uniform():
    s = free_system((10, 9, 8), (5.0, 4.6, 4.2), complex_wf=True)
    x, y, z = grid_coords(s)
    V = s.cell[0] * s.cell[1] * s.cell[2]
    qs = [(0, 0, 0), (1, 0, 0), (0, -1, 2), (3, 2, -1)]
    psi = np.array([np.exp(2j * math.pi * (q[0] * x / s.cell[0] + q[1] * y / s.cell[1] + q[2] * z / s.cell[2]))
                    / math.sqrt(V) for q in qs])
    f = np.array([2.0, 2.0, 1.0, 0.5])
    rho = O.density(s, psi, f)
    assert np.allclose(rho, np.sum(f) / V, rtol=1e-14, atol=0)


# ------------------------------------------------------------------------------------------
# f-3: the Poisson solve for the Hartree potential
# ------------------------------------------------------------------------------------------

def test_poisson_solution_satisfies_the_fd_equation():
    # the Fourier-route solution, put through the real-space stencil of the oracle (a route
    # that shares nothing with the FFT), gives back 2 pi (rho - <rho>); its mean is zero
    s = small_system(n=(14, 12, 10), natoms=2)
    f = synth.free_grid(s)
    rho = np.abs(rand_psi(s, 1, 51)).reshape(s.n[::-1]) ** 2
    v = O.poisson(f, rho)
    Tv = O.kinetic_local(f, v.reshape((1,) + v.shape)).reshape(v.shape)
    b = 2 * math.pi * (rho - rho.mean())
    assert np.max(np.abs(Tv - b)) < 1e-12 * np.max(np.abs(b))
    assert abs(v.mean()) < 1e-14 * np.max(np.abs(v))


def test_poisson_plane_wave_closed_form():
    # rho = cos(G.r) has v = -4 pi cos(G.r) / L(G) with the FD symbol written out by hand
    s = free_system((12, 10, 9), (6.0, 5.0, 4.5))
    x, y, z = grid_coords(s)
    q = (2, -1, 1)
    G = [2 * math.pi * q[c] / s.cell[c] for c in range(3)]
    rho = np.cos(G[0] * x + G[1] * y + G[2] * z)
    w = golden_weights()
    L = sum((w[0] + 2 * sum(w[m] * math.cos(m * G[c] * s.h[c]) for m in (1, 2, 3))) / s.h[c] ** 2 for c in range(3))
    v = O.poisson(s, rho)
    assert np.allclose(v, -4 * math.pi * rho / L, rtol=0, atol=1e-13 * np.max(np.abs(4 * math.pi * rho / L)))


# ------------------------------------------------------------------------------------------
# f-4: H and S in the plane-wave representation (wave-function section; reading)
# ------------------------------------------------------------------------------------------

def pw_unit_vectors(system, js):
    """Coefficient arrays [len(js)][N3][N2][N1] with a single 1 at the FFT index of G = 2 pi j / L."""
    C = np.zeros((len(js), system.n[2], system.n[1], system.n[0]), complex)
    for b, j in enumerate(js):
        C[b, j[2] % system.n[2], j[1] % system.n[1], j[0] % system.n[0]] = 1.0
    return C


def test_pw_free_plane_waves_closed_form():
    # no potential, no atoms: every basis vector is an eigenvector of H with |k + G|^2 / 2 (the
    # exact kinetic energy, not the finite-difference symbol) and of S with 1
    k = (0.37, -0.21, 0.55)
    s = free_system((10, 9, 8), (5.0, 4.6, 4.1), k=k, complex_wf=True)
    js = [(0, 0, 0), (1, 0, 0), (0, 2, -1), (3, -4, 2), (-5, 4, 3), (4, -4, -4)]
    C = pw_unit_vectors(s, js)
    HC = O.pw_apply(s, C, "H")
    SC = O.pw_apply(s, C, "S")
    for b, j in enumerate(js):
        q = [k[c] + 2 * math.pi * j[c] / s.cell[c] for c in range(3)]
        lam = 0.5 * sum(v * v for v in q)
        assert np.allclose(HC[b], lam * C[b], rtol=0, atol=1e-13 * max(lam, 1.0))
        assert np.allclose(SC[b], C[b], rtol=0, atol=1e-14)


def test_pw_constant_potential_shifts_the_spectrum():
    k = (0.1, 0.2, -0.3)
    v0 = -0.7
    s = free_system((8, 6, 5), (4.0, 3.0, 2.5), k=k, complex_wf=True, vloc=np.full((5, 6, 8), v0))
    C = rand_psi(s, 4, 90)
    HC = O.pw_apply(s, C, "H")
    assert np.allclose(HC, (O.pw_kinetic(s)[None] + v0) * C, rtol=0, atol=1e-13 * np.max(np.abs(HC)))


def test_pw_grid_transforms_are_inverse_and_keep_the_norm():
    s = small_system(complex_wf=True)
    C = rand_psi(s, 3, 91)
    psi = O.pw_to_grid(s, C)
    assert np.allclose(O.grid_to_pw(s, psi), C, rtol=0, atol=1e-14 * np.max(np.abs(C)))
    # Parseval: dV sum_r |psi|^2 = Omega sum_G |C_G|^2
    omega = s.cell[0] * s.cell[1] * s.cell[2]
    assert np.allclose(s.dV * np.sum(np.abs(psi) ** 2, axis=(1, 2, 3)), omega * np.sum(np.abs(C) ** 2, axis=(1, 2, 3)),
                       rtol=1e-13)
    # a single coefficient is the plane wave e^{i(k+G).r} at the grid points
    j = (2, -1, 1)
    x, y, z = grid_coords(s)
    q = [s.k[c] + 2 * math.pi * j[c] / s.cell[c] for c in range(3)]
    wave = O.pw_to_grid(s, pw_unit_vectors(s, [j]))[0]
    assert np.allclose(wave, np.exp(1j * (q[0] * x + q[1] * y + q[2] * z)), rtol=0, atol=1e-13)


@pytest.mark.parametrize("case", ["bloch", "selfwrap-bloch"])
def test_pw_dense_bruteforce(case):
    # the plane-wave operators as explicit K x K matrices in the coefficient basis:
    # A_H = diag(|k+G|^2 / 2) + U^-1 (H - T) U and A_S = U^-1 S U, with U[r, G] = e^{i(k+G).r},
    # U^-1 = U^H / K, and H, S, T (the finite-difference kinetic) the dense real-space operators;
    # applied to random coefficients and diagonalized over the full basis
    s = small_system(**TINY[case])
    H, S = dense_operators(s)
    T, _ = dense_operators(free_system(s.n, s.cell, k=s.k, complex_wf=True))
    K = s.npoints
    qx, qy, qz = (q.reshape(-1) for q in O.pw_wavevectors(s))
    x, y, z = (a.reshape(-1) for a in grid_coords(s))
    U = np.exp(1j * (np.outer(x, qx) + np.outer(y, qy) + np.outer(z, qz)))
    A_H = np.diag(0.5 * (qx * qx + qy * qy + qz * qz)) + U.conj().T @ (H - T) @ U / K
    A_S = U.conj().T @ S @ U / K
    C = rand_psi(s, 5, 92)
    Cm = C.reshape(5, K).T
    HC = O.pw_apply(s, C, "H").reshape(5, K).T
    SC = O.pw_apply(s, C, "S").reshape(5, K).T
    assert np.allclose(HC, A_H @ Cm, rtol=0, atol=1e-12 * np.max(np.abs(HC)))
    assert np.allclose(SC, A_S @ Cm, rtol=0, atol=1e-12 * np.max(np.abs(SC)))
    # the full basis: Rayleigh-Ritz with the oracle's Gram and subspace solve gives the dense
    # generalized spectrum
    E = np.eye(K, dtype=complex).reshape(K, s.n[2], s.n[1], s.n[0])
    Hnm = O.gram(E, O.pw_apply(s, E, "H"), 1.0, K)
    Snm = O.gram(E, O.pw_apply(s, E, "S"), 1.0, K)
    eps, _, _ = O.subspace_diag(Hnm, Snm)
    exact = scipy.linalg.eigh(A_H, A_S, eigvals_only=True)
    assert np.allclose(eps, exact, rtol=0, atol=1e-10 * max(1.0, np.max(np.abs(exact))))


def test_pw_energy_cutoff_masks_the_output():
    s = small_system(complex_wf=True)
    C = rand_psi(s, 2, 93)
    ecut = 0.4 * np.max(O.pw_kinetic(s))
    mask = O.pw_kinetic(s) <= ecut
    Cm = C * mask[None]
    HC = O.pw_apply(s, Cm, "H", ecut=ecut)
    full = O.pw_apply(s, Cm, "H")
    assert np.all(HC[:, ~mask] == 0)
    assert np.array_equal(HC[:, mask], full[:, mask])
