"""The C-ABI library builds, loads, and exports every symbol include/*.h declares (no GPU)."""
import glob
import os
import re
import subprocess

import pytest

from paper_2310_14776_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(pawfd_\w+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pawfd_apply_H", "pawfd_apply_S", "pawfd_project", "pawfd_subspace_diag", "pawfd_rotate",
                     "pawfd_gram", "pawfd_create", "pawfd_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\b(pawfd_\w+)\b", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(libpath):
    assert set(_lib.SIGNATURES) == set(declared_functions())
    L = _lib.load(libpath)
    for name in declared_functions():
        assert getattr(L, name) is not None


def test_binding_arity_matches_header():
    # every ctypes signature has as many arguments as the header's declaration
    decl = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for name, args in re.findall(r"\b(pawfd_\w+)\s*\(([^)]*)\)\s*;", text):
            args = args.strip()
            decl[name] = 0 if args in ("", "void") else args.count(",") + 1
    assert set(decl) == set(_lib.SIGNATURES)
    wrong = {n: (decl[n], len(_lib.SIGNATURES[n][0])) for n in decl if decl[n] != len(_lib.SIGNATURES[n][0])}
    assert not wrong, wrong


def test_header_compiles_as_c():
    src = '#include "pawfd.h"\nint main(void){ pawfd_system_desc d; (void)d; return PAWFD_OK; }\n'
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-fsyntax-only", "-I", os.path.join(ROOT, "include"),
                        "-x", "c", "-"], input=src, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


@pytest.mark.parametrize("cname,cls", [("pawfd_system_desc", "SystemDesc"), ("pawfd_rr_job", "RrJob")])
def test_struct_layout_matches_header(cname, cls):
    # field offsets of the ctypes mirrors equal those the C compiler gives the header's structs
    import ctypes
    mirror = getattr(_lib, cls)
    fields = [f[0] for f in mirror._fields_]
    prog = '#include <stdio.h>\n#include <stddef.h>\n#include "pawfd.h"\nint main(void){\n'
    for f in fields:
        prog += 'printf("%%zu\\n", offsetof(%s, %s));\n' % (cname, f)
    prog += 'printf("%%zu\\n", sizeof(%s)); return 0; }\n' % cname
    exe = "/tmp/pawfd_layout_check_" + cname
    r = subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), "-x", "c", "-", "-o", exe],
                       input=prog, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = [int(v) for v in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    want = [getattr(mirror, f).offset for f in fields] + [ctypes.sizeof(mirror)]
    assert got == want


def test_api_fails_loudly_without_cuda():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2310_14776_gb300 import api, synth
    s = synth.WORKLOADS["gamma-24c-16b"].system()
    with pytest.raises(Exception):
        api.Context(s, max_bands=4, device="cuda:0")


# ------------------------------------------------------------------------------------------
# error behaviour that is decided on the host (no device is touched)
# ------------------------------------------------------------------------------------------

EINVAL = -1


def _null_args(argtypes):
    import ctypes
    out = []
    for t in argtypes:
        if t in (ctypes.c_int, ctypes.c_longlong):
            out.append(1)
        elif t is ctypes.c_double:
            out.append(1.0)
        elif t is ctypes.c_char_p:
            out.append(b"stencil_fx")
        else:
            out.append(None)
    return out


def test_null_context_and_batch_are_rejected(libpath):
    # every entry point that takes a context or batch first: PAWFD_EINVAL (or the documented
    # fixed answers) for NULL, before any CUDA call
    L = _lib.load(libpath)
    fixed = {"pawfd_last_error": b"no context", "pawfd_batch_last_error": b"null batch",
             "pawfd_batch_is_graph": 0, "pawfd_batch_kernel_count": 0}
    takes_first = [n for n in declared_functions()
                   if n not in ("pawfd_create", "pawfd_batch_create", "pawfd_gram_noalloc")]
    for name in takes_first:
        args = _null_args(_lib.SIGNATURES[name][0])
        got = getattr(L, name)(*args)
        assert got == fixed.get(name, EINVAL), (name, got)
    import ctypes
    assert L.pawfd_create(None, None, None) == EINVAL
    assert L.pawfd_batch_create(None, None, 1, 0) == EINVAL
    assert L.pawfd_gram_noalloc(None, None, 1, 1, 0, 1.0, None, None) == EINVAL
    job = _lib.RrJob()
    h = ctypes.c_void_p()
    assert L.pawfd_batch_create(ctypes.byref(h), ctypes.byref(job), 1, 0) == EINVAL   # a job without a context
    assert h.value is None


def _desc(system, dtype, max_bands=4):
    """The ctypes description of a synthetic system, with the arrays it points to kept alive."""
    import ctypes
    import numpy as np
    keep = dict(
        nproj=np.ascontiguousarray(system.nproj, np.int32), box_lo=np.ascontiguousarray(system.box_lo, np.int32),
        box_n=np.ascontiguousarray(system.box_n, np.int32), proj=np.ascontiguousarray(system.proj, np.float64),
        proj_off=np.ascontiguousarray(system.proj_off, np.int64), dH=np.ascontiguousarray(system.dH, np.float64),
        dS=np.ascontiguousarray(system.dS, np.float64), dmat_off=np.ascontiguousarray(system.dmat_off, np.int64),
        vloc=np.ascontiguousarray(system.vloc, np.float64).reshape(-1))
    d = _lib.SystemDesc()
    d.n[:] = [int(v) for v in system.n]
    d.cell[:] = [float(v) for v in system.cell]
    d.k[:] = [float(v) for v in system.k]
    d.dtype = dtype
    d.max_bands = max_bands
    d.natoms = int(len(keep["nproj"]))
    for name, a in keep.items():
        setattr(d, name, ctypes.c_void_p(a.ctypes.data) if a.size else None)
    return d, keep


def _bad_descs(system):
    import numpy as np
    R64, C128 = _lib.PAWFD_R64, _lib.PAWFD_C128
    cases = {}

    def case(name, change, dtype=R64):
        d, keep = _desc(system, dtype)
        change(d, keep)
        cases[name] = (d, keep)

    case("grid size 0", lambda d, k: d.n.__setitem__(1, 0))
    case("cell length 0", lambda d, k: d.cell.__setitem__(2, 0.0))
    case("negative cell", lambda d, k: d.cell.__setitem__(0, -1.0))
    case("grid too large", lambda d, k: (d.n.__setitem__(0, 2048), d.n.__setitem__(1, 1024), d.n.__setitem__(2, 1024)))
    case("unknown dtype", lambda d, k: setattr(d, "dtype", 99))
    case("real with k", lambda d, k: d.k.__setitem__(0, 0.25))
    case("max_bands 0", lambda d, k: setattr(d, "max_bands", 0))
    case("vloc NULL", lambda d, k: setattr(d, "vloc", None))
    case("natoms < 0", lambda d, k: setattr(d, "natoms", -1))
    case("atom arrays missing", lambda d, k: setattr(d, "dS", None))

    def set_arr(name, i, v):
        def f(d, keep):
            a = keep[name].copy()
            a.reshape(-1)[i] = v
            keep[name + "_bad"] = a
            setattr(d, name, a.ctypes.data)
        return f

    case("nproj 0", set_arr("nproj", 0, 0))
    case("nproj 33", set_arr("nproj", 0, 33))
    case("box size 0", set_arr("box_n", 2, 0))
    case("proj_off mismatch", set_arr("proj_off", 1, int(np.asarray(system.proj_off)[1]) - 1))
    case("dmat_off mismatch", set_arr("dmat_off", 1, int(np.asarray(system.dmat_off)[1]) + 1))
    return cases


def test_create_rejects_invalid_descriptions_on_the_host(libpath):
    import ctypes
    from paper_2310_14776_gb300 import synth
    L = _lib.load(libpath)
    s = synth.WORKLOADS["gamma-24c-16b"].system()
    assert s.natoms > 0
    for name, (d, keep) in _bad_descs(s).items():
        h = ctypes.c_void_p(1234)
        assert L.pawfd_create(ctypes.byref(h), ctypes.byref(d), None) == EINVAL, name
        assert h.value is None, name
    # the unchanged description passes the host checks: without a device it reaches the
    # first CUDA call and fails there (PAWFD_EDEVICE), not in validation
    import torch
    if not torch.cuda.is_available():
        d, keep = _desc(s, _lib.PAWFD_R64)
        h = ctypes.c_void_p()
        assert L.pawfd_create(ctypes.byref(h), ctypes.byref(d), None) == -6   # PAWFD_EDEVICE
        assert h.value is None
