"""Python front end of the FP64 CPU oracle (``paw_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the test suite, by the smoke check and by the
CPU-baseline leg of the benchmark, never by the library itself.  The C source is compiled
here with gcc (``build()``), IEEE semantics kept (no fast-math, no FMA contraction, so the
oracle gives the same bits on x86-64 and aarch64).

Every function takes numpy arrays in the layouts of ``paw_oracle.c`` and a
``paper_2310_14776_gb300.synth.System`` describing the cell, grid, potential, projector
boxes and PAW correction matrices.  Passages followed: Eq. (dh) and the overlap operator
(PAW section), the projector overlaps entering the atomic density matrix (same section),
SCF step 1 of the Kohn-Sham section (subspace diagonalization), and the dense Cholesky +
diagonalization of the parallelization section.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "paw_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libpaw_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``paw_oracle.c`` into ``_build/libpaw_oracle.so`` (OpenMP if the compiler has it)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", _SRC,
            "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i, l, d = ctypes.c_int, ctypes.c_long, ctypes.c_double
            sig = {
                "oracle_fd6_coefficients": [P],
                "oracle_kinetic_local_real": [P, P, P, P, l, P],
                "oracle_kinetic_local_bloch": [P, P, P, P, P, l, P],
                "oracle_project": [P, P, P, i, i, P, P, P, P, P, P, l, P],
                "oracle_apply": [i, P, P, P, i, P, i, P, P, P, P, P, P, P, P, l, P, P],
                "oracle_gram": [i, P, P, l, l, d, P],
                "oracle_subspace_diag": [i, l, P, P, P, P, P],
                "oracle_cholesky": [i, l, P, P],
                "oracle_jacobi_eigh": [i, l, P, P, P, P],
                "oracle_rotate": [i, P, l, l, P, P],
                "oracle_num_threads": [],
            }
            for name, args in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = ctypes.c_int
            _lib = L
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _c(a, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def fd6_coefficients() -> np.ndarray:
    out = np.zeros(4)
    lib().oracle_fd6_coefficients(_ptr(out))
    return out


class _Geometry:
    """Keeps the marshalled system arrays alive for the duration of a call."""

    def __init__(self, system):
        self.n = _c(system.n, np.int32)
        self.L = _c(system.cell, np.float64)
        self.k = _c(system.k, np.float64)
        self.v = _c(system.vloc, np.float64)
        self.nproj = _c(system.nproj, np.int32)
        self.box_lo = _c(system.box_lo, np.int32)
        self.box_n = _c(system.box_n, np.int32)
        self.proj = _c(system.proj, np.float64)
        self.proj_off = _c(system.proj_off, np.int64)
        self.dH = _c(system.dH, np.float64)
        self.dS = _c(system.dS, np.float64)
        self.dmat_off = _c(system.dmat_off, np.int64)
        self.natoms = int(system.natoms)
        self.cplx = bool(system.complex_wf)
        self.Ip = int(system.nproj_total)


def _psi_in(system, psi) -> Tuple[np.ndarray, int]:
    dt = np.complex128 if system.complex_wf else np.float64
    psi = _c(psi, dt)
    nb = psi.size // system.npoints
    return psi, nb


def kinetic_local(system, psi: np.ndarray) -> np.ndarray:
    """-1/2 Lap_FD psi + v psi (the kinetic and local-potential terms of Eq. (dh))."""
    g = _Geometry(system)
    psi, nb = _psi_in(system, psi)
    out = np.empty_like(psi)
    if g.cplx:
        rc = lib().oracle_kinetic_local_bloch(_ptr(g.n), _ptr(g.L), _ptr(g.k), _ptr(g.v), _ptr(psi), nb, _ptr(out))
    else:
        rc = lib().oracle_kinetic_local_real(_ptr(g.n), _ptr(g.L), _ptr(g.v), _ptr(psi), nb, _ptr(out))
    assert rc == 0
    return out


def project(system, psi: np.ndarray) -> np.ndarray:
    """P [Ip][nb] = <p_i^a | psi_n>."""
    g = _Geometry(system)
    psi, nb = _psi_in(system, psi)
    P = np.zeros((g.Ip, nb), dtype=psi.dtype)
    rc = lib().oracle_project(_ptr(g.n), _ptr(g.L), _ptr(g.k), int(g.cplx), g.natoms, _ptr(g.nproj), _ptr(g.box_lo),
                              _ptr(g.box_n), _ptr(g.proj), _ptr(g.proj_off), _ptr(psi), nb, _ptr(P))
    assert rc == 0
    return P


def _apply(which: int, system, psi: np.ndarray):
    g = _Geometry(system)
    psi, nb = _psi_in(system, psi)
    out = np.empty_like(psi)
    P = np.zeros((g.Ip, nb), dtype=psi.dtype)
    dmat = g.dH if which == 0 else g.dS
    rc = lib().oracle_apply(which, _ptr(g.n), _ptr(g.L), _ptr(g.k), int(g.cplx), _ptr(g.v), g.natoms, _ptr(g.nproj),
                            _ptr(g.box_lo), _ptr(g.box_n), _ptr(g.proj), _ptr(g.proj_off), _ptr(dmat),
                            _ptr(g.dmat_off), _ptr(psi), nb, _ptr(out), _ptr(P))
    assert rc == 0
    return out, P


def apply_H(system, psi: np.ndarray):
    """(H psi, P): Eq. (dh) applied to every band."""
    return _apply(0, system, psi)


def apply_S(system, psi: np.ndarray):
    """(S psi, P): the PAW overlap operator applied to every band."""
    return _apply(1, system, psi)


def nonlocal_term(system, psi: np.ndarray, which: str = "H") -> np.ndarray:
    """sum_a sum_ii' |p_i^a> X^a_ii' <p_i'^a|psi> for X = dH ("H") or dS ("S"): the nonlocal
    term of Eq. (dh) and of the overlap operator, without the kinetic, local and identity
    terms."""
    g = _Geometry(system)
    psi, nb = _psi_in(system, psi)
    out = np.empty_like(psi)
    P = np.zeros((g.Ip, nb), dtype=psi.dtype)
    dmat = g.dH if which == "H" else g.dS
    rc = lib().oracle_apply(2, _ptr(g.n), _ptr(g.L), _ptr(g.k), int(g.cplx), _ptr(g.v), g.natoms, _ptr(g.nproj),
                            _ptr(g.box_lo), _ptr(g.box_n), _ptr(g.proj), _ptr(g.proj_off), _ptr(dmat),
                            _ptr(g.dmat_off), _ptr(psi), nb, _ptr(out), _ptr(P))
    assert rc == 0
    return out


def gram(A: np.ndarray, B: np.ndarray, dV: float, nb: int) -> np.ndarray:
    """M[n][m] = dV sum_r conj(A_n(r)) B_m(r)."""
    cplx = np.iscomplexobj(A) or np.iscomplexobj(B)
    dt = np.complex128 if cplx else np.float64
    A = _c(A, dt)
    B = _c(B, dt)
    K = A.size // nb
    M = np.zeros((nb, nb), dtype=dt)
    rc = lib().oracle_gram(int(cplx), _ptr(A), _ptr(B), K, nb, float(dV), _ptr(M))
    assert rc == 0
    return M


class SubspaceError(RuntimeError):
    def __init__(self, code: int):
        super().__init__("Cholesky failed at column %d" % (-code - 1) if code > -1000000 else "Jacobi did not converge")
        self.code = code


def subspace_diag(Hnm: np.ndarray, Snm: np.ndarray):
    """(eps ascending, C) with H C = S C diag(eps), C^H S C = I; plus the Jacobi sweep count."""
    cplx = np.iscomplexobj(Hnm) or np.iscomplexobj(Snm)
    dt = np.complex128 if cplx else np.float64
    H = _c(Hnm, dt)
    S = _c(Snm, dt)
    n = H.shape[0]
    eps = np.zeros(n)
    C = np.zeros((n, n), dtype=dt)
    sweeps = ctypes.c_int(0)
    rc = lib().oracle_subspace_diag(int(cplx), n, _ptr(H), _ptr(S), _ptr(eps), _ptr(C), ctypes.byref(sweeps))
    if rc != 0:
        raise SubspaceError(rc)
    return eps, C, int(sweeps.value)


def cholesky(S: np.ndarray) -> np.ndarray:
    cplx = np.iscomplexobj(S)
    S = _c(S, np.complex128 if cplx else np.float64)
    L = np.zeros_like(S)
    rc = lib().oracle_cholesky(int(cplx), S.shape[0], _ptr(S), _ptr(L))
    if rc != 0:
        raise SubspaceError(rc)
    return L


def jacobi_eigh(A: np.ndarray):
    """(eigenvalues in Jacobi order, V, sweeps) with A = V diag V^H."""
    cplx = np.iscomplexobj(A)
    A = _c(A, np.complex128 if cplx else np.float64)
    n = A.shape[0]
    w = np.zeros(n)
    V = np.zeros_like(A)
    sweeps = ctypes.c_int(0)
    rc = lib().oracle_jacobi_eigh(int(cplx), n, _ptr(A), _ptr(w), _ptr(V), ctypes.byref(sweeps))
    if rc != 0:
        raise SubspaceError(-1000000)
    return w, V, int(sweeps.value)


def rotate(psi: np.ndarray, C: np.ndarray) -> np.ndarray:
    """psi'_m = sum_n psi_n C[n][m]."""
    cplx = np.iscomplexobj(psi) or np.iscomplexobj(C)
    dt = np.complex128 if cplx else np.float64
    psi = _c(psi, dt)
    C = _c(C, dt)
    nb = C.shape[0]
    K = psi.size // nb
    out = np.empty_like(psi)
    rc = lib().oracle_rotate(int(cplx), _ptr(psi), K, nb, _ptr(C), _ptr(out))
    assert rc == 0
    return out


def rayleigh_ritz(system, psi: np.ndarray) -> dict:
    """One eigensolver step: H psi, S psi, H_nm, S_nm, subspace diag, rotation (SCF step 1)."""
    psi, nb = _psi_in(system, psi)
    Hpsi, P = apply_H(system, psi)
    Spsi, _ = apply_S(system, psi)
    Hnm = gram(psi, Hpsi, system.dV, nb)
    Snm = gram(psi, Spsi, system.dV, nb)
    eps, C, sweeps = subspace_diag(Hnm, Snm)
    psi_rot = rotate(psi, C)
    return {"Hpsi": Hpsi, "Spsi": Spsi, "P": P, "Hnm": Hnm, "Snm": Snm, "eps": eps, "C": C, "sweeps": sweeps,
            "psi_rot": psi_rot}


def residual_norms(Hpsi: np.ndarray, Spsi: np.ndarray, eps: np.ndarray, dV: float) -> np.ndarray:
    """||r_n|| = sqrt(dV sum_r |(H psi)_n(r) - eps_n (S psi)_n(r)|^2) for every band n.

    The residual of the generalized eigenproblem H psi = eps S psi of the PAW section, the
    quantity an iterative eigensolver drives to zero (Kohn-Sham section, step 1)."""
    nb = len(eps)
    r = Hpsi.reshape(nb, -1) - np.asarray(eps, np.float64)[:, None] * Spsi.reshape(nb, -1)
    return np.sqrt(dV * np.sum(np.abs(r) ** 2, axis=1))


def density(system, psi: np.ndarray, f: np.ndarray) -> np.ndarray:
    """The pseudo density rho(r) = sum_n f_n |psi_n(r)|^2 of one spin channel (the PAW
    section's n~ without compensation charges; the density of step 4 of the Kohn-Sham
    section), [N3][N2][N1] float64."""
    psi, nb = _psi_in(system, psi)
    f = np.asarray(f, np.float64)
    rho = np.zeros(system.npoints)
    for n in range(nb):
        rho += f[n] * np.abs(psi.reshape(nb, -1)[n]) ** 2
    return rho.reshape(psi.shape[1:])


def atomic_density(system, P: np.ndarray, f: np.ndarray) -> np.ndarray:
    """Eq. (atomicdensitymatrix): D^a_ii' = sum_n f_n <psi_n|p_i^a> <p_i'^a|psi_n>
    = sum_n f_n conj(P[row_a + i][n]) P[row_a + i'][n] (P from ``project``), packed per atom
    like dH and dS (offsets system.dmat_off)."""
    f = np.asarray(f, np.float64)
    cplx = np.iscomplexobj(P)
    D = np.zeros(int(system.dmat_off[-1]) if system.natoms else 0, np.complex128 if cplx else np.float64)
    row = 0
    for a in range(system.natoms):
        I = int(system.nproj[a])
        Pa = P[row:row + I]
        Da = (np.conj(Pa) * f[None, :]) @ Pa.T
        D[int(system.dmat_off[a]):int(system.dmat_off[a]) + I * I] = Da.reshape(-1)
        row += I
    return D


def laplacian_symbol(system) -> np.ndarray:
    """The eigenvalues of the order-6 FD Laplacian on the periodic grid, [N3][N2][N1]:
    L(G) = sum_c (1/h_c^2) (c0 + 2 sum_m c_m cos(m G_c h_c)) for the grid's wave vectors G."""
    c = fd6_coefficients()
    h = system.h
    parts = []
    for ax in range(3):
        G = 2.0 * np.pi * np.fft.fftfreq(system.n[ax], d=h[ax])
        parts.append((c[0] + 2.0 * sum(c[m] * np.cos(m * G * h[ax]) for m in (1, 2, 3))) / (h[ax] * h[ax]))
    return parts[2][:, None, None] + parts[1][None, :, None] + parts[0][None, None, :]


def poisson(system, rho: np.ndarray) -> np.ndarray:
    """The zero-mean solution of lap_FD v = -4 pi (rho - <rho>) on the periodic grid with the
    order-6 Laplacian (the Poisson solve of the Kohn-Sham section's potential update, by its
    direct Fourier-transform route): v(G) = -4 pi rho(G) / L(G) for G != 0, v(0) = 0."""
    rho = np.asarray(rho, np.float64).reshape(system.n[2], system.n[1], system.n[0])
    L = laplacian_symbol(system)
    rg = np.fft.fftn(rho)
    vg = np.zeros_like(rg)
    nz = np.ones(L.shape, bool)
    nz[0, 0, 0] = False
    vg[nz] = -4.0 * np.pi * rg[nz] / L[nz]
    return np.real(np.fft.ifftn(vg))


def davidson_weights(system, eps: np.ndarray) -> np.ndarray:
    """Jacobi preconditioner weights w_n(r) = -1 / max(d(r) - eps_n, d0 / 10) of the block-Davidson
    step (a reading: the paper names the Davidson eigensolver of the Kohn-Sham and
    parallelization sections without its steps).  d(r) = v(r) + d0 is the diagonal of the
    kinetic + local operator, d0 = -1/2 c0 sum_c 1/h_c^2 the stencil's centre weight."""
    c0 = fd6_coefficients()[0]
    h = system.h
    d0 = -0.5 * c0 * (1.0 / (h[0] * h[0]) + 1.0 / (h[1] * h[1]) + 1.0 / (h[2] * h[2]))
    d = np.asarray(system.vloc, np.float64).reshape(-1) + d0
    e = np.asarray(eps, np.float64)
    floor = 0.1 * d0
    den = d[None, :] - e[:, None]
    den = np.where(den > floor, den, floor)
    return -1.0 / den


KINETIC_SHIFT = 0.5   # Hartree: sigma of the kinetic preconditioner (a reading)


def kinetic_symbol(system) -> np.ndarray:
    """t(k + G) = -1/2 L_FD(k + G), [N3][N2][N1]: the eigenvalue of the order-6 FD kinetic
    operator T on the Bloch wave e^{i(k+G).r} of the grid (G the grid's FFT wave vectors),
    t = -1/2 sum_c (1/h_c^2) (c0 + 2 sum_m c_m cos(m q_c h_c)) with q = k + G."""
    c = fd6_coefficients()
    h = system.h
    parts = []
    for ax in range(3):
        q = system.k[ax] + 2.0 * np.pi * np.fft.fftfreq(system.n[ax], d=h[ax])
        parts.append(-0.5 * (c[0] + 2.0 * sum(c[m] * np.cos(m * q * h[ax]) for m in (1, 2, 3))) / (h[ax] * h[ax]))
    return parts[2][:, None, None] + parts[1][None, :, None] + parts[0][None, None, :]


def kinetic_precondition(system, R: np.ndarray, sigma: float = KINETIC_SHIFT) -> np.ndarray:
    """The kinetic preconditioner of the block-Davidson step (a reading; the paper names the
    Davidson eigensolver without its steps): the correction -(T + sigma)^-1 R_n of each residual,
    with T the order-6 FD kinetic operator of the grid (Bloch boundary conditions) and sigma > 0.
    T is diagonal on the Bloch waves, so for R(r) = e^{ik.r} u(r):
    -(T + sigma)^-1 R = -e^{ik.r} IDFT[ DFT[u] / (t(k + G) + sigma) ]."""
    R = np.asarray(R)
    nb = R.shape[0]
    shape = (system.n[2], system.n[1], system.n[0])
    u = R.reshape((nb,) + shape).astype(np.complex128)
    ph = bloch_phase(system)
    u = u * np.conj(ph)[None]
    d = kinetic_symbol(system) + sigma
    out = -ph[None] * np.fft.ifftn(np.fft.fftn(u, axes=(1, 2, 3)) / d[None], axes=(1, 2, 3))
    if not system.complex_wf:
        out = out.real
    return out.reshape(R.shape)


def davidson_step(system, psi: np.ndarray, eps_in: np.ndarray, precond: str = "kinetic") -> dict:
    """One block-Davidson step in the order of its reading:

    1. H psi and S psi for the n input Ritz vectors psi (Ritz values eps_in);
    2. residuals R_n = H psi_n - eps_n S psi_n and their norms sqrt(dV sum_r |R_n|^2);
    3. corrections: -(T + sigma)^-1 R_n (``kinetic_precondition``, precond="kinetic") or
       w_n R_n with the Jacobi weights of ``davidson_weights`` (precond="jacobi");
    4. Rayleigh-Ritz on the 2n columns X = [psi, corrections]: Gram matrices dV X^H H X and
       dV X^H S X, the subspace diagonalization (2n Ritz pairs, ascending), and the n lowest
       Ritz vectors X C[:, :n].
    """
    psi, nb = _psi_in(system, psi)
    K = system.npoints
    Hpsi, _ = apply_H(system, psi)
    Spsi, _ = apply_S(system, psi)
    eps_in = np.asarray(eps_in, np.float64)[:nb]
    R = Hpsi.reshape(nb, K) - eps_in[:, None] * Spsi.reshape(nb, K)
    rnorm = np.sqrt(system.dV * np.sum(np.abs(R) ** 2, axis=1))
    if precond == "kinetic":
        corr = kinetic_precondition(system, R)
    else:
        corr = R * davidson_weights(system, eps_in)
    X = np.concatenate([psi.reshape(nb, K), corr.astype(psi.dtype)]).reshape((2 * nb,) + psi.shape[1:])
    HX, _ = apply_H(system, X)
    SX, _ = apply_S(system, X)
    Hnm = gram(X, HX, system.dV, 2 * nb)
    Snm = gram(X, SX, system.dV, 2 * nb)
    eps, C, sweeps = subspace_diag(Hnm, Snm)
    psi_out = rotate(X, C).reshape(2 * nb, K)[:nb].reshape(psi.shape)
    return {"X": X, "Hnm": Hnm, "Snm": Snm, "eps": eps, "C": C, "rnorm": rnorm, "psi_out": psi_out,
            "sweeps": sweeps}


def refine(system, psi_lo: np.ndarray, C_lo: Optional[np.ndarray] = None) -> dict:
    """Final refinement of the mixed form, in the order of its reading (the paper is silent):

    1. the FP32 / complex64 bands are promoted to FP64 (exactly).  When C_lo is given they are
       the INPUT bands of a mixed Rayleigh-Ritz step and C_lo that step's FP64 eigenvector
       matrix: the promoted bands are rotated by it in FP64, psi' = psi C_lo.  A rotation by a
       nonsingular matrix keeps the span of the bands, so the second Rayleigh-Ritz step below
       sees the subspace of the original input, not that of FP32-rounded rotated bands;
    2. H psi' and S psi' are applied in FP64 (Eq. (dh) and the overlap operator);
    3. FP64 Gram matrices H'_nm, S'_nm are formed;
    4. the Rayleigh quotients theta_n = H'_nn / S'_nn are taken from their diagonals;
    5. a second FP64 subspace diagonalization gives the refined eps (ascending) and C;
    6. the residual norms ||H psi'_n - eps_n S psi'_n|| are reported.
    """
    psi = np.asarray(psi_lo).astype(np.complex128 if system.complex_wf else np.float64)
    psi, nb = _psi_in(system, psi)
    if C_lo is not None:
        psi = rotate(psi, np.asarray(C_lo))
    Hpsi, P = apply_H(system, psi)
    Spsi, _ = apply_S(system, psi)
    Hnm = gram(psi, Hpsi, system.dV, nb)
    Snm = gram(psi, Spsi, system.dV, nb)
    theta = np.real(np.diag(Hnm)) / np.real(np.diag(Snm))
    eps, C, sweeps = subspace_diag(Hnm, Snm)
    resid = residual_norms(Hpsi, Spsi, eps, system.dV)
    return {"psi": psi, "Hpsi": Hpsi, "Spsi": Spsi, "Hnm": Hnm, "Snm": Snm, "theta": theta, "eps": eps, "C": C,
            "resid": resid}


# ------------------------------------------------------------------------------------------
# Plane-wave representation (the wave-function section: psi_kn(r) = sum_G C_nG e^{i(k+G).r})
# ------------------------------------------------------------------------------------------

def pw_wavevectors(system):
    """The components (k + G)_c on the FFT grid of the cell, each [N3][N2][N1]: G_c runs over
    2 pi j / L_c for the FFT frequencies j of N_c points (0, 1, ..., -1)."""
    q = []
    for c in range(3):
        g1 = system.k[c] + 2.0 * np.pi * np.fft.fftfreq(system.n[c], d=1.0 / system.n[c]) / system.cell[c]
        shape = [1, 1, 1]
        shape[2 - c] = system.n[c]
        q.append(np.broadcast_to(g1.reshape(shape), (system.n[2], system.n[1], system.n[0])))
    return q


def pw_kinetic(system) -> np.ndarray:
    """The plane-wave kinetic energies |k + G|^2 / 2 (Hartree), [N3][N2][N1]."""
    qx, qy, qz = pw_wavevectors(system)
    return 0.5 * (qx * qx + qy * qy + qz * qz)


def bloch_phase(system) -> np.ndarray:
    """e^{i k.r} at the grid points r = (i1 h1, i2 h2, i3 h3), [N3][N2][N1]."""
    z, y, x = np.meshgrid(*[np.arange(system.n[c]) * system.h[c] for c in (2, 1, 0)], indexing="ij")
    return np.exp(1j * (system.k[0] * x + system.k[1] * y + system.k[2] * z))


def pw_to_grid(system, C: np.ndarray) -> np.ndarray:
    """psi(r) = sum_G C_G e^{i(k+G).r} at the grid points, for every band of C [nb][N3][N2][N1]
    (G in FFT order): e^{ik.r} times the inverse discrete Fourier transform times K."""
    C = np.asarray(C, np.complex128)
    K = system.npoints
    return bloch_phase(system)[None] * np.fft.ifftn(C, axes=(1, 2, 3)) * K


def grid_to_pw(system, psi: np.ndarray) -> np.ndarray:
    """C_G = (1/K) sum_r e^{-i(k+G).r} psi(r), the inverse of pw_to_grid."""
    psi = np.asarray(psi, np.complex128)
    return np.fft.fftn(np.conj(bloch_phase(system))[None] * psi, axes=(1, 2, 3)) / system.npoints


def pw_apply(system, C: np.ndarray, which: str = "H", ecut: float = 0.0) -> np.ndarray:
    """H C or S C in the plane-wave representation (a reading of the PW mode: the
    generalized eigenproblem of Eq. (dh) in the basis e^{i(k+G).r} of the cell's FFT grid):
      (H C)_G = |k+G|^2 / 2 C_G + [v psi + sum_a |p^a> dH^a <p^a|psi>]_G,
      (S C)_G = C_G + [sum_a |p^a> dS^a <p^a|psi>]_G,
    with psi = pw_to_grid(C), [f]_G = grid_to_pw(f), and the projectors sampled on the grid
    (the same projector boxes as the finite-difference operator).  With ecut > 0 the basis is
    the sphere |k+G|^2 / 2 <= ecut: the output is zero outside it (C is taken as given)."""
    C = np.asarray(C, np.complex128)
    psi = pw_to_grid(system, C)
    if which == "H":
        v = np.asarray(system.vloc, np.float64).reshape(system.n[2], system.n[1], system.n[0])
        out = pw_kinetic(system)[None] * C + grid_to_pw(system, v[None] * psi + nonlocal_term(system, psi, "H"))
    else:
        out = C + grid_to_pw(system, nonlocal_term(system, psi, "S"))
    if ecut > 0:
        out = out * (pw_kinetic(system) <= ecut)[None]
    return out
