"""ctypes binding of libpawfd.so (include/pawfd.h).  Argument marshalling only."""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpawfd.so")

PAWFD_R64 = 0
PAWFD_C128 = 1
PAWFD_R32 = 2
PAWFD_C64 = 3
ERRORS = {0: "PAWFD_OK", -1: "PAWFD_EINVAL", -2: "PAWFD_ENOMEM", -3: "PAWFD_ENOTPD", -4: "PAWFD_ENOCONV",
          -5: "PAWFD_ETIMEDOUT", -6: "PAWFD_EDEVICE"}

# every symbol include/pawfd.h declares, with its argument types
VP, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double


class SystemDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("cell", ctypes.c_double * 3), ("k", ctypes.c_double * 3),
                ("dtype", ctypes.c_int), ("max_bands", ctypes.c_int), ("natoms", ctypes.c_int),
                ("nproj", VP), ("box_lo", VP), ("box_n", VP), ("proj", VP), ("proj_off", VP),
                ("dH", VP), ("dS", VP), ("dmat_off", VP), ("vloc", VP)]


class RrJob(ctypes.Structure):
    _fields_ = [("ctx", VP), ("psi", VP), ("nb", ctypes.c_int), ("hpsi", VP), ("spsi", VP), ("Hnm", VP),
                ("Snm", VP), ("eps", VP), ("C", VP), ("psi_out", VP)]


SIGNATURES = {
    "pawfd_create": ([ctypes.POINTER(VP), ctypes.POINTER(SystemDesc), VP], I),
    "pawfd_destroy": ([VP], I),
    "pawfd_set_stream": ([VP, VP], I),
    "pawfd_sync": ([VP], I),
    "pawfd_last_error": ([VP], ctypes.c_char_p),
    "pawfd_nproj_total": ([VP], I),
    "pawfd_launch_count": ([VP], ctypes.c_longlong),
    "pawfd_set_option": ([VP, ctypes.c_char_p, I], I),
    "pawfd_project": ([VP, VP, I, VP], I),
    "pawfd_apply_H": ([VP, VP, I, VP, VP], I),
    "pawfd_apply_S": ([VP, VP, I, VP, VP], I),
    "pawfd_apply_kinetic_local": ([VP, VP, I, VP], I),
    "pawfd_gram": ([VP, VP, VP, I, VP], I),
    "pawfd_gram_hermitian": ([VP, VP, VP, I, VP], I),
    "pawfd_apply_HS": ([VP, VP, I, VP, VP, VP], I),
    "pawfd_gram_hs": ([VP, VP, VP, I, VP, VP, VP], I),
    "pawfd_subspace_diag": ([VP, I, VP, VP, VP, VP], I),
    "pawfd_rotate": ([VP, VP, I, VP, VP], I),
    "pawfd_refine": ([VP, VP, I, VP, VP, VP, VP, VP, VP, VP, VP, VP, VP], I),
    "pawfd_rr_step": ([VP, VP, I, VP, VP, VP, VP, VP, VP, VP], I),
    "pawfd_rotate_n": ([VP, VP, I, VP, I, VP], I),
    "pawfd_residual_precond": ([VP, VP, VP, I, VP, VP, VP], I),
    "pawfd_davidson_step": ([VP, VP, I, VP, VP, VP, VP, VP, VP, VP, VP, VP, VP], I),
    "pawfd_density": ([VP, VP, I, VP, VP], I),
    "pawfd_kernel_timing": ([VP, I, ctypes.POINTER(D), ctypes.POINTER(ctypes.c_longlong)], I),
    "pawfd_poisson": ([VP, VP, VP, D, I, VP, ctypes.POINTER(I), ctypes.POINTER(D)], I),
    "pawfd_atomic_density": ([VP, VP, I, VP, VP], I),
    "pawfd_batch_create": ([ctypes.POINTER(VP), ctypes.POINTER(RrJob), I, I], I),
    "pawfd_batch_launch": ([VP, VP], I),
    "pawfd_batch_is_graph": ([VP], I),
    "pawfd_batch_kernel_count": ([VP], ctypes.c_longlong),
    "pawfd_batch_last_error": ([VP], ctypes.c_char_p),
    "pawfd_batch_destroy": ([VP], I),
    "pawfd_gram_noalloc": ([VP, VP, ctypes.c_longlong, I, I, D, VP, VP], I),
    "pawfd_pw_apply_H": ([VP, VP, I, D, VP, VP], I),
    "pawfd_pw_apply_S": ([VP, VP, I, D, VP, VP], I),
    "pawfd_pw_to_grid": ([VP, VP, I, VP], I),
    "pawfd_pw_from_grid": ([VP, VP, I, VP, VP], I),
    "pawfd_poisson_fft": ([VP, VP, VP, VP], I),
    "pawfd_kinetic_precond": ([VP, VP, I, VP, VP], I),
}

_lock = threading.Lock()
_lib = None


class PawFDError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


def load(path: str = LIB_PATH):
    """Load the CUDA library; raises if it has not been built (there is no CPU fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError("libpawfd.so not built: run paper_2310_14776_gb300.build.build() "
                                   "(needs nvcc); the library has no CPU fallback")
            L = ctypes.CDLL(path)
            for name, (args, res) in SIGNATURES.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib
