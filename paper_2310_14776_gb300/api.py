"""Python front end of the C ABI: torch tensors in, device pointers out.

PyTorch provides device memory and the current CUDA stream; every step of the eigensolver
step runs in the CUDA kernels of libpawfd.so.  This module only checks shapes, dtypes and
devices and passes pointers.
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np
import torch

from . import _lib
from ._lib import PawFDError


def _np_ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


class Context:
    """One system (cell, grid, local potential, projector boxes, dH/dS) resident on the GPU.

    ``system`` is a ``synth.System`` or any object with the same fields.  All band arrays are
    torch tensors on the context's device, shaped [nb, N3, N2, N1], contiguous: float64 /
    complex128 (Gamma point / Bloch vector) for ``precision="fp64"``, float32 / complex64
    for ``precision="mixed"``.  Gram matrices, eigenvalues and C are always FP64.
    """

    def __init__(self, system, max_bands: int, device: Optional[torch.device] = None, precision: str = "fp64"):
        self.lib = _lib.load()
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        if self.device.type != "cuda":
            raise ValueError("the PAW library runs on CUDA devices only")
        self.n = tuple(int(v) for v in system.n)
        self.K = self.n[0] * self.n[1] * self.n[2]
        self.complex = bool(system.complex_wf)
        if precision not in ("fp64", "mixed"):
            raise ValueError("precision must be 'fp64' or 'mixed'")
        self.precision = precision
        self.mat_dtype = torch.complex128 if self.complex else torch.float64
        if precision == "fp64":
            self.dtype = self.mat_dtype
        else:
            self.dtype = torch.complex64 if self.complex else torch.float32
        self.max_bands = int(max_bands)
        self._dmat_total = int(np.asarray(system.dmat_off)[-1]) if int(system.natoms) > 0 else 0
        h = [system.cell[c] / self.n[c] for c in range(3)]
        self.dV = h[0] * h[1] * h[2]
        keep = dict(
            nproj=np.ascontiguousarray(system.nproj, np.int32), box_lo=np.ascontiguousarray(system.box_lo, np.int32),
            box_n=np.ascontiguousarray(system.box_n, np.int32), proj=np.ascontiguousarray(system.proj, np.float64),
            proj_off=np.ascontiguousarray(system.proj_off, np.int64), dH=np.ascontiguousarray(system.dH, np.float64),
            dS=np.ascontiguousarray(system.dS, np.float64), dmat_off=np.ascontiguousarray(system.dmat_off, np.int64),
            vloc=np.ascontiguousarray(system.vloc, np.float64).reshape(-1))
        d = _lib.SystemDesc()
        d.n[:] = list(self.n)
        d.cell[:] = [float(v) for v in system.cell]
        d.k[:] = [float(v) for v in system.k]
        d.dtype = {("fp64", False): _lib.PAWFD_R64, ("fp64", True): _lib.PAWFD_C128,
                   ("mixed", False): _lib.PAWFD_R32, ("mixed", True): _lib.PAWFD_C64}[(precision, self.complex)]
        d.max_bands = self.max_bands
        d.natoms = int(len(keep["nproj"]))
        for name in ("nproj", "box_lo", "box_n", "proj", "proj_off", "dH", "dS", "dmat_off", "vloc"):
            setattr(d, name, _np_ptr(keep[name]) if keep[name].size else None)
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            rc = self.lib.pawfd_create(ctypes.byref(self._h), ctypes.byref(d), self._stream())
        if rc != 0:
            raise PawFDError(rc, "pawfd_create failed (see stderr)")
        self.Ip = int(self.lib.pawfd_nproj_total(self._h))

    # ------------------------------------------------------------------------------------
    def _stream(self):
        return ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    def _call(self, fn, *args):
        self.lib.pawfd_set_stream(self._h, self._stream())
        rc = fn(self._h, *args)
        if rc != 0:
            raise PawFDError(rc, self.lib.pawfd_last_error(self._h).decode())

    def _bands(self, t: torch.Tensor, name: str) -> int:
        if t.device != self.device or t.dtype != self.dtype or not t.is_contiguous():
            raise ValueError("%s must be a contiguous %s tensor on %s" % (name, self.dtype, self.device))
        if t.numel() % self.K:
            raise ValueError("%s size is not a multiple of the grid size" % name)
        return t.numel() // self.K

    def _mat(self, t: torch.Tensor, nb: int, name: str):
        if t.device != self.device or t.dtype != self.mat_dtype or not t.is_contiguous() or t.numel() != nb * nb:
            raise ValueError("%s must be a contiguous [%d, %d] %s tensor on %s" % (name, nb, nb, self.mat_dtype,
                                                                                   self.device))

    def _out_bands(self, t: torch.Tensor, nb: int, name: str):
        if self._bands(t, name) < nb:
            raise ValueError("%s must hold at least %d bands" % (name, nb))

    def _vec(self, t: torch.Tensor, n: int, name: str):
        if t.device != self.device or t.dtype != torch.float64 or not t.is_contiguous() or t.numel() < n:
            raise ValueError("%s must be a contiguous float64 tensor of at least %d values on %s" % (name, n, self.device))

    def _proj(self, P: torch.Tensor, nb: int, name: str = "P"):
        if P.device != self.device or P.dtype != self.dtype or not P.is_contiguous() or P.numel() < self.Ip * nb:
            raise ValueError("%s must be a contiguous [Ip, %d] tensor of the band dtype on %s" % (name, nb, self.device))

    def empty_bands(self, nb: int) -> torch.Tensor:
        return torch.empty((nb,) + self.n[::-1], dtype=self.dtype, device=self.device)

    # ------------------------------------------------------------------------------------
    def sync(self):
        """Wait for the context's work; raise the first device-side error (Cholesky, Jacobi, timeout)."""
        rc = self.lib.pawfd_sync(self._h)
        if rc != 0:
            raise PawFDError(rc, self.lib.pawfd_last_error(self._h).decode())

    def set_option(self, name: str, value: int):
        """Choose among equivalent implementations (see pawfd_set_option in include/pawfd.h)."""
        rc = self.lib.pawfd_set_option(self._h, name.encode(), int(value))
        if rc != 0:
            raise PawFDError(rc, self.lib.pawfd_last_error(self._h).decode())

    def launch_count(self) -> int:
        """CUDA kernels this context has launched (counted by the library)."""
        return int(self.lib.pawfd_launch_count(self._h))

    def kinetic_local(self, psi, out=None):
        nb = self._bands(psi, "psi")
        out = self.empty_bands(nb) if out is None else out
        self._out_bands(out, nb, "out")
        self._call(self.lib.pawfd_apply_kinetic_local, ctypes.c_void_p(psi.data_ptr()), nb,
                   ctypes.c_void_p(out.data_ptr()))
        return out

    def project(self, psi, P=None):
        nb = self._bands(psi, "psi")
        P = torch.empty((self.Ip, nb), dtype=self.dtype, device=self.device) if P is None else P
        if P.numel() != self.Ip * nb or P.dtype != self.dtype or not P.is_contiguous() or P.device != self.device:
            raise ValueError("P must be a contiguous [Ip, nb] tensor of the band dtype on the device")
        self._call(self.lib.pawfd_project, ctypes.c_void_p(psi.data_ptr()), nb, ctypes.c_void_p(P.data_ptr()))
        return P

    def _apply(self, fn, psi, out, P):
        nb = self._bands(psi, "psi")
        out = self.empty_bands(nb) if out is None else out
        self._out_bands(out, nb, "out")
        if P is not None:
            self._proj(P, nb)
        self._call(fn, ctypes.c_void_p(psi.data_ptr()), nb, ctypes.c_void_p(out.data_ptr()),
                   ctypes.c_void_p(P.data_ptr()) if P is not None else None)
        return out

    def apply_H(self, psi, out=None, P=None):
        return self._apply(self.lib.pawfd_apply_H, psi, out, P)

    def apply_S(self, psi, out=None, P=None):
        return self._apply(self.lib.pawfd_apply_S, psi, out, P)

    def apply_hs(self, psi, Hpsi=None, Spsi=None, P=None):
        """H psi and S psi with one set of projections (pawfd_apply_HS); returns (Hpsi, Spsi, P)."""
        nb = self._bands(psi, "psi")
        Hpsi = self.empty_bands(nb) if Hpsi is None else Hpsi
        Spsi = self.empty_bands(nb) if Spsi is None else Spsi
        self._out_bands(Hpsi, nb, "Hpsi")
        self._out_bands(Spsi, nb, "Spsi")
        P = torch.empty((max(self.Ip, 1), nb), dtype=self.dtype, device=self.device) if P is None else P
        self._proj(P, nb)
        self._call(self.lib.pawfd_apply_HS, ctypes.c_void_p(psi.data_ptr()), nb, ctypes.c_void_p(Hpsi.data_ptr()),
                   ctypes.c_void_p(Spsi.data_ptr()), ctypes.c_void_p(P.data_ptr()))
        return Hpsi, Spsi, P

    def gram_hs(self, psi, Hpsi, P, Hnm=None, Snm=None):
        """H_nm = dV psi^H H psi and S_nm = dV psi^H psi + sum_a P_a^H dS^a P_a (pawfd_gram_hs);
        P holds the projections of psi.  Returns (Hnm, Snm)."""
        nb = self._bands(psi, "psi")
        if self._bands(Hpsi, "Hpsi") != nb:
            raise ValueError("psi and Hpsi must hold the same number of bands")
        Hnm = torch.empty((nb, nb), dtype=self.mat_dtype, device=self.device) if Hnm is None else Hnm
        Snm = torch.empty((nb, nb), dtype=self.mat_dtype, device=self.device) if Snm is None else Snm
        self._mat(Hnm, nb, "Hnm")
        self._mat(Snm, nb, "Snm")
        if P is not None:
            self._proj(P, nb)
        self._call(self.lib.pawfd_gram_hs, ctypes.c_void_p(psi.data_ptr()), ctypes.c_void_p(Hpsi.data_ptr()), nb,
                   ctypes.c_void_p(P.data_ptr()) if P is not None else None, ctypes.c_void_p(Hnm.data_ptr()),
                   ctypes.c_void_p(Snm.data_ptr()))
        return Hnm, Snm

    def gram(self, A, B, M=None, hermitian: bool = False):
        """M = dV A^H B.  ``hermitian``: B = X A for a Hermitian X; only the upper half is
        computed and mirrored (pawfd_gram_hermitian)."""
        nb = self._bands(A, "A")
        if self._bands(B, "B") != nb:
            raise ValueError("A and B must hold the same number of bands")
        M = torch.empty((nb, nb), dtype=self.mat_dtype, device=self.device) if M is None else M
        self._mat(M, nb, "M")
        fn = self.lib.pawfd_gram_hermitian if hermitian else self.lib.pawfd_gram
        self._call(fn, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()), nb, ctypes.c_void_p(M.data_ptr()))
        return M

    def subspace_diag(self, Hnm, Snm, eps=None, C=None, overwrite: bool = False, check: bool = True):
        """(eps, C) of H C = S C diag(eps).  Inputs are copied unless ``overwrite``."""
        nb = Hnm.shape[0]
        self._mat(Hnm, nb, "Hnm")
        self._mat(Snm, nb, "Snm")
        if not overwrite:
            Hnm, Snm = Hnm.clone(), Snm.clone()
        eps = torch.empty(nb, dtype=torch.float64, device=self.device) if eps is None else eps
        self._vec(eps, nb, "eps")
        C = torch.empty((nb, nb), dtype=self.mat_dtype, device=self.device) if C is None else C
        self._mat(C, nb, "C")
        self._call(self.lib.pawfd_subspace_diag, nb, ctypes.c_void_p(Hnm.data_ptr()), ctypes.c_void_p(Snm.data_ptr()),
                   ctypes.c_void_p(eps.data_ptr()), ctypes.c_void_p(C.data_ptr()))
        if check:
            self.sync()
        return eps, C

    def rotate(self, psi, C, out=None):
        nb = self._bands(psi, "psi")
        self._mat(C, nb, "C")
        out = self.empty_bands(nb) if out is None else out
        self._out_bands(out, nb, "out")
        self._call(self.lib.pawfd_rotate, ctypes.c_void_p(psi.data_ptr()), nb, ctypes.c_void_p(C.data_ptr()),
                   ctypes.c_void_p(out.data_ptr()))
        return out

    def rotate_n(self, psi, C, nout: int, out=None):
        """psi_out_m = sum_n psi_n C[n][m] for m < nout (pawfd_rotate_n)."""
        nb = self._bands(psi, "psi")
        self._mat(C, nb, "C")
        out = self.empty_bands(nout) if out is None else out
        if self._bands(out, "out") != nout:
            raise ValueError("out must hold nout bands")
        self._call(self.lib.pawfd_rotate_n, ctypes.c_void_p(psi.data_ptr()), nb, ctypes.c_void_p(C.data_ptr()),
                   int(nout), ctypes.c_void_p(out.data_ptr()))
        return out

    def residual_precond(self, Hpsi, Spsi, eps, pr=None, rnorm=None):
        """Residuals H psi - eps S psi: their norms and the preconditioned corrections
        (pawfd_residual_precond).  Returns (pr, rnorm)."""
        nb = self._bands(Hpsi, "Hpsi")
        self._out_bands(Spsi, nb, "Spsi")
        if eps.numel() != nb:
            raise ValueError("eps must hold nb float64 values on the device")
        self._vec(eps, nb, "eps")
        pr = self.empty_bands(nb) if pr is None else pr
        self._out_bands(pr, nb, "pr")
        rnorm = torch.empty(nb, dtype=torch.float64, device=self.device) if rnorm is None else rnorm
        self._vec(rnorm, nb, "rnorm")
        self._call(self.lib.pawfd_residual_precond, ctypes.c_void_p(Hpsi.data_ptr()), ctypes.c_void_p(Spsi.data_ptr()),
                   nb, ctypes.c_void_p(eps.data_ptr()), ctypes.c_void_p(pr.data_ptr()),
                   ctypes.c_void_p(rnorm.data_ptr()))
        return pr, rnorm

    def kernel_timing(self, enable: bool):
        """Device time of the Gram MMA kernel launches timed since the previous call (ms, count),
        then timing on or off (pawfd_kernel_timing)."""
        ms = ctypes.c_double(0.0)
        n = ctypes.c_longlong(0)
        self._call(self.lib.pawfd_kernel_timing, int(bool(enable)), ctypes.byref(ms), ctypes.byref(n))
        return ms.value, n.value

    def poisson(self, rho, v=None, tol: float = 1e-11, maxiter: int = 5000):
        """The zero-mean Hartree potential of rho (pawfd_poisson); this context must be the
        free operator of its grid (see ``poisson_context``).  Returns (v, iterations, relative
        residual)."""
        if rho.numel() != self.K or rho.dtype != torch.float64 or rho.device != self.device:
            raise ValueError("rho must hold K float64 values on the device")
        rho = rho.contiguous()          # held until the call returns
        v = torch.empty(self.K, dtype=torch.float64, device=self.device) if v is None else v
        if v.numel() != self.K or v.dtype != torch.float64 or v.device != self.device or not v.is_contiguous():
            raise ValueError("v must be a contiguous float64 tensor of K values on the device")
        work = torch.empty(4 * self.K + 304, dtype=torch.float64, device=self.device)
        it = ctypes.c_int(0)
        res = ctypes.c_double(0.0)
        self._call(self.lib.pawfd_poisson, ctypes.c_void_p(rho.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                   float(tol), int(maxiter), ctypes.c_void_p(work.data_ptr()), ctypes.byref(it), ctypes.byref(res))
        return v, it.value, res.value

    def kinetic_precond(self, R, out=None, work=None):
        """-(T + sigma)^-1 R for every band of R (pawfd_kinetic_precond; FP32 transforms,
        sigma = 0.5 Ha).  ``out`` may be R."""
        nb = self._bands(R, "R")
        out = self.empty_bands(nb) if out is None else out
        self._out_bands(out, nb, "out")
        nt = nb if self.complex else (nb + 1) // 2
        work = torch.empty(nt * self.K, dtype=torch.complex64, device=self.device) if work is None else work
        if work.numel() * work.element_size() < 8 * self.K * nt or not work.is_contiguous():
            raise ValueError("work must be a contiguous device array of at least 8 K bytes per transform")
        self._call(self.lib.pawfd_kinetic_precond, ctypes.c_void_p(R.data_ptr()), nb, ctypes.c_void_p(out.data_ptr()),
                   ctypes.c_void_p(work.data_ptr()))
        return out

    def poisson_fft(self, rho, v=None, work=None):
        """The zero-mean Hartree potential of rho by the direct Fourier route
        (pawfd_poisson_fft); this context must be the free operator of its grid (see
        ``poisson_context``).  Returns v."""
        if rho.numel() != self.K or rho.dtype != torch.float64 or rho.device != self.device:
            raise ValueError("rho must hold K float64 values on the device")
        rho = rho.contiguous()          # held until the call returns
        v = torch.empty(self.K, dtype=torch.float64, device=self.device) if v is None else v
        if v.numel() != self.K or v.dtype != torch.float64 or v.device != self.device or not v.is_contiguous():
            raise ValueError("v must be a contiguous float64 tensor of K values on the device")
        work = torch.empty(self.K, dtype=torch.complex128, device=self.device) if work is None else work
        if (work.numel() < self.K or work.dtype != torch.complex128 or work.device != self.device
                or not work.is_contiguous()):
            raise ValueError("work must be a contiguous complex128 tensor of at least K values on the device")
        self._call(self.lib.pawfd_poisson_fft, ctypes.c_void_p(rho.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                   ctypes.c_void_p(work.data_ptr()))
        return v

    def density(self, psi, f, rho=None):
        """rho(r) = sum_n f_n |psi_n(r)|^2 (pawfd_density); f: device float64 [nb]."""
        nb = self._bands(psi, "psi")
        if f.numel() != nb or f.dtype != torch.float64 or f.device != self.device:
            raise ValueError("f must hold nb float64 values on the device")
        rho = torch.empty(self.K, dtype=torch.float64, device=self.device) if rho is None else rho
        if rho.numel() != self.K or rho.dtype != torch.float64 or not rho.is_contiguous() or rho.device != self.device:
            raise ValueError("rho must be a contiguous float64 tensor of K values on the device")
        self._call(self.lib.pawfd_density, ctypes.c_void_p(psi.data_ptr()), nb, ctypes.c_void_p(f.data_ptr()),
                   ctypes.c_void_p(rho.data_ptr()))
        return rho

    def atomic_density(self, P, f, D=None):
        """D^a = sum_n f_n conj(P_an) P_an^T per atom, packed like dH / dS (pawfd_atomic_density)."""
        nb = f.numel()
        if f.dtype != torch.float64 or f.device != self.device or not f.is_contiguous():
            raise ValueError("f must hold nb float64 values on the device")
        if P.numel() != self.Ip * nb or P.dtype != self.dtype or not P.is_contiguous() or P.device != self.device:
            raise ValueError("P must be a contiguous [Ip, nb] tensor of the band dtype on the device")
        total = int(self._dmat_total)
        D = torch.empty(max(total, 1), dtype=self.mat_dtype, device=self.device) if D is None else D
        if D.numel() < total or D.dtype != self.mat_dtype or not D.is_contiguous() or D.device != self.device:
            raise ValueError("D must be a contiguous %s tensor of at least %d values on the device"
                             % (self.mat_dtype, total))
        self._call(self.lib.pawfd_atomic_density, ctypes.c_void_p(P.data_ptr()), nb, ctypes.c_void_p(f.data_ptr()),
                   ctypes.c_void_p(D.data_ptr()))
        return D[:total]

    def alloc_davidson(self, nb: int) -> dict:
        """Device arrays of one block-Davidson step for nb bands (needs max_bands >= 2 nb)."""
        m = 2 * nb
        return {"X": self.empty_bands(m), "HX": self.empty_bands(m), "SX": self.empty_bands(nb),
                "P": torch.empty((max(self.Ip, 1), m), dtype=self.dtype, device=self.device),
                "Hnm": torch.empty((m, m), dtype=self.mat_dtype, device=self.device),
                "Snm": torch.empty((m, m), dtype=self.mat_dtype, device=self.device),
                "C": torch.empty((m, m), dtype=self.mat_dtype, device=self.device),
                "eps": torch.empty(m, dtype=torch.float64, device=self.device),
                "rnorm": torch.empty(nb, dtype=torch.float64, device=self.device),
                "psi_out": self.empty_bands(nb)}

    def davidson_step(self, work: dict, nb: int, eps_in) -> dict:
        """One block-Davidson step (pawfd_davidson_step) on work["X"][:nb] (Ritz vectors with
        Ritz values eps_in); fills the arrays of ``work`` (see alloc_davidson) and returns it.
        work["psi_out"] holds the nb lowest Ritz vectors, work["eps"][:nb] their Ritz values,
        work["rnorm"] the residual norms of the input vectors."""
        w = work
        for key, count in (("X", 2 * nb), ("HX", 2 * nb), ("SX", nb), ("psi_out", nb)):
            if self._bands(w[key], key) != count:
                raise ValueError("%s must hold %d bands" % (key, count))
        for key in ("Hnm", "Snm", "C"):
            self._mat(w[key], 2 * nb, key)
        self._vec(eps_in, nb, "eps_in")
        if w["eps"].numel() != 2 * nb or w["rnorm"].numel() != nb:
            raise ValueError("eps must hold 2 nb and rnorm nb float64 values")
        self._vec(w["eps"], 2 * nb, "eps")
        self._vec(w["rnorm"], nb, "rnorm")
        self._proj(w["P"], 2 * nb)
        p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
        self._call(self.lib.pawfd_davidson_step, p(w["X"]), nb, p(eps_in), p(w["HX"]), p(w["SX"]), p(w["P"]),
                   p(w["Hnm"]), p(w["Snm"]), p(w["eps"]), p(w["C"]), p(w["rnorm"]), p(w["psi_out"]))
        return w

    def rayleigh_ritz(self, psi, work: Optional[dict] = None, check: bool = True, keep_matrices: bool = False) -> dict:
        """One eigensolver step: H psi, S psi, H_nm, S_nm, subspace diag, rotation.

        ``work`` may hold preallocated outputs under the result's keys.  Unless
        ``keep_matrices`` the returned Hnm / Snm are the solver's workspace after the solve."""
        nb = self._bands(psi, "psi")
        w = work if work is not None else {}
        Hpsi, Spsi, P = self.apply_hs(psi, Hpsi=w.get("Hpsi"), Spsi=w.get("Spsi"), P=w.get("P"))
        Hnm, Snm = self.gram_hs(psi, Hpsi, P, Hnm=w.get("Hnm"), Snm=w.get("Snm"))
        eps, C = self.subspace_diag(Hnm, Snm, eps=w.get("eps"), C=w.get("C"), overwrite=not keep_matrices, check=check)
        psi_rot = self.rotate(psi, C, out=w.get("psi_rot"))
        return {"Hpsi": Hpsi, "Spsi": Spsi, "P": P, "Hnm": Hnm, "Snm": Snm, "eps": eps, "C": C, "psi_rot": psi_rot}

    def alloc_work(self, nb: int) -> dict:
        """Device arrays of one Rayleigh-Ritz step for nb bands (the keys rr_step fills)."""
        return {"Hpsi": self.empty_bands(nb), "Spsi": self.empty_bands(nb),
                "Hnm": torch.empty((nb, nb), dtype=self.mat_dtype, device=self.device),
                "Snm": torch.empty((nb, nb), dtype=self.mat_dtype, device=self.device),
                "eps": torch.empty(nb, dtype=torch.float64, device=self.device),
                "C": torch.empty((nb, nb), dtype=self.mat_dtype, device=self.device)}

    def _job_args(self, psi, out, work):
        nb = self._bands(psi, "psi")
        self._out_bands(out, nb, "out")
        for key in ("Hpsi", "Spsi"):
            self._out_bands(work[key], nb, key)
        for key in ("Hnm", "Snm", "C"):
            self._mat(work[key], nb, key)
        if work["eps"].numel() != nb:
            raise ValueError("eps must hold nb float64 values")
        self._vec(work["eps"], nb, "eps")
        p = lambda t: t.data_ptr()  # noqa: E731
        return nb, (p(psi), nb, p(work["Hpsi"]), p(work["Spsi"]), p(work["Hnm"]), p(work["Snm"]), p(work["eps"]),
                    p(work["C"]), p(out))

    def rr_step(self, psi, out=None, work: Optional[dict] = None) -> dict:
        """One whole Rayleigh-Ritz step in a single library call (pawfd_rr_step): returns the
        work dict (Hpsi, Spsi, Hnm/Snm as the solver's workspace, eps, C) plus psi_rot."""
        nb = self._bands(psi, "psi")
        work = work if work is not None else self.alloc_work(nb)
        out = self.empty_bands(nb) if out is None else out
        _, args = self._job_args(psi, out, work)
        self._call(self.lib.pawfd_rr_step, *[ctypes.c_void_p(a) if i != 1 else a for i, a in enumerate(args)])
        res = dict(work)
        res["psi_rot"] = out
        return res

    def refine(self, psi_lo, C_lo=None, work: Optional[dict] = None, check: bool = True) -> dict:
        """Final refinement of mixed-form bands on this FP64 context (pawfd_refine): FP64
        H psi', S psi', Gram matrices, Rayleigh quotients ``theta``, a second subspace solve
        (``eps``, ``C``) and residual norms ``resid``.  ``psi_lo`` is a float32 / complex64 band
        array of a mixed context of the same system.  With ``C_lo`` (the FP64 eigenvector
        matrix a mixed Rayleigh-Ritz step returned for the input bands ``psi_lo``) the bands
        refined are psi_lo C_lo rotated in FP64, which keeps the span of the input; without it,
        psi_lo as given."""
        if self.precision != "fp64":
            raise ValueError("refine runs on an fp64 context")
        lo = torch.complex64 if self.complex else torch.float32
        if psi_lo.device != self.device or psi_lo.dtype != lo or not psi_lo.is_contiguous():
            raise ValueError("psi_lo must be a contiguous %s tensor on %s" % (lo, self.device))
        if psi_lo.numel() % self.K:
            raise ValueError("psi_lo size is not a multiple of the grid size")
        nb = psi_lo.numel() // self.K
        if C_lo is not None:
            self._mat(C_lo, nb, "C_lo")
        w = work if work is not None else {}
        out = {}
        for key in ("psi", "Hpsi", "Spsi"):
            out[key] = w.get(key) if w.get(key) is not None else self.empty_bands(nb)
            self._out_bands(out[key], nb, key)
        for key in ("Hnm", "Snm", "C"):
            out[key] = w.get(key) if w.get(key) is not None else torch.empty((nb, nb), dtype=self.mat_dtype,
                                                                             device=self.device)
            self._mat(out[key], nb, key)
        for key in ("eps", "theta", "resid"):
            out[key] = w.get(key) if w.get(key) is not None else torch.empty(nb, dtype=torch.float64,
                                                                             device=self.device)
            self._vec(out[key], nb, key)
        p = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
        self._call(self.lib.pawfd_refine, p(psi_lo), nb, p(C_lo), p(out["psi"]), p(out["Hpsi"]), p(out["Spsi"]),
                   p(out["Hnm"]), p(out["Snm"]), p(out["eps"]), p(out["theta"]), p(out["resid"]), p(out["C"]))
        if check:
            self.sync()
        return out

    # -- plane-wave representation (pawfd_pw_*) ------------------------------------------
    def _pw_check(self, C, name):
        if not self.complex:
            raise ValueError("the plane-wave representation needs a complex context")
        return self._bands(C, name)

    def pw_apply(self, C, which: str = "H", ecut: float = 0.0, out=None, work=None):
        """H C or S C in the plane-wave representation (pawfd_pw_apply_H / _S): C holds the
        coefficients of nb bands on the cell's FFT grid, [nb, N3, N2, N1] in FFT order."""
        nb = self._pw_check(C, "C")
        out = self.empty_bands(nb) if out is None else out
        self._out_bands(out, nb, "out")
        work = self.empty_bands(2 * nb) if work is None else work
        self._out_bands(work, 2 * nb, "work")
        fn = {"H": self.lib.pawfd_pw_apply_H, "S": self.lib.pawfd_pw_apply_S}[which]
        self._call(fn, ctypes.c_void_p(C.data_ptr()), nb, float(ecut), ctypes.c_void_p(out.data_ptr()),
                   ctypes.c_void_p(work.data_ptr()))
        return out

    def pw_to_grid(self, C, out=None):
        """psi(r) = sum_G C_G e^{i(k+G).r} at the grid points (pawfd_pw_to_grid)."""
        nb = self._pw_check(C, "C")
        out = self.empty_bands(nb) if out is None else out
        self._out_bands(out, nb, "out")
        self._call(self.lib.pawfd_pw_to_grid, ctypes.c_void_p(C.data_ptr()), nb, ctypes.c_void_p(out.data_ptr()))
        return out

    def pw_from_grid(self, psi, out=None, work=None):
        """C_G = (1/K) sum_r e^{-i(k+G).r} psi(r) (pawfd_pw_from_grid)."""
        nb = self._pw_check(psi, "psi")
        out = self.empty_bands(nb) if out is None else out
        self._out_bands(out, nb, "out")
        work = self.empty_bands(nb) if work is None else work
        self._out_bands(work, nb, "work")
        self._call(self.lib.pawfd_pw_from_grid, ctypes.c_void_p(psi.data_ptr()), nb, ctypes.c_void_p(out.data_ptr()),
                   ctypes.c_void_p(work.data_ptr()))
        return out

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self.lib.pawfd_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Independent Rayleigh-Ritz steps of several contexts (pawfd_batch_*): every launch runs
    one step of every job, each job on a stream of its own so that their kernels overlap;
    with ``use_graph`` the sequence is captured once into a CUDA graph and each launch is a
    single graph launch (the arrays are then fixed).  ``entries``: (ctx, psi, out, work)."""

    def __init__(self, entries, use_graph: bool = True):
        if not entries:
            raise ValueError("a batch needs at least one job")
        self.lib = _lib.load()
        self.entries = list(entries)   # keeps the tensors alive
        jobs = (_lib.RrJob * len(entries))()
        for i, (ctx, psi, out, work) in enumerate(entries):
            nb, args = ctx._job_args(psi, out, work)
            j = jobs[i]
            j.ctx = ctx._h.value
            j.psi, j.nb, j.hpsi, j.spsi, j.Hnm, j.Snm, j.eps, j.C, j.psi_out = args
        self.device = entries[0][0].device
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            rc = self.lib.pawfd_batch_create(ctypes.byref(self._h), jobs, len(entries), int(use_graph))
        if rc != 0:
            raise PawFDError(rc, "pawfd_batch_create failed")

    @property
    def is_graph(self) -> bool:
        return bool(self.lib.pawfd_batch_is_graph(self._h))

    @property
    def kernel_count(self) -> int:
        return int(self.lib.pawfd_batch_kernel_count(self._h))

    @property
    def last_error(self) -> str:
        return self.lib.pawfd_batch_last_error(self._h).decode()

    def launch(self):
        stream = ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)
        rc = self.lib.pawfd_batch_launch(self._h, stream)
        if rc != 0:
            raise PawFDError(rc, self.last_error)

    def sync(self):
        """Wait for the device and raise the first error any job's context recorded."""
        torch.cuda.synchronize(self.device)
        for ctx, *_ in self.entries:
            ctx.sync()

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self.lib.pawfd_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def poisson_context(system, device=None) -> Context:
    """An FP64 context of the free operator T on ``system``'s grid (v = 0, no atoms): the
    operator of the Poisson solve."""
    from . import synth
    return Context(synth.free_grid(system), max_bands=1, device=device, precision="fp64")
