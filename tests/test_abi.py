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
