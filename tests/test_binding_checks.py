"""The Python binding checks shapes, dtypes, devices and layouts before it hands a pointer to
the library (no GPU): a context shell on the CPU device whose library refuses every call,
so a check that lets a bad argument through fails the test.  Also checks that good
arguments reach the library."""
import pytest
import torch

from paper_2310_14776_gb300 import api


class Refuse:
    """Stands in for libpawfd.so: records the entry point that would have been called."""

    def __init__(self):
        self.called = []

    def __getattr__(self, name):
        def fn(*args):
            self.called.append(name)
            return 0
        return fn


def shell(ip=6, complex_wf=False, mixed=False, dmat_total=72):
    c = object.__new__(api.Context)
    c.lib = Refuse()
    c.device = torch.device("cpu")
    c.n = (5, 4, 3)
    c.K = 60
    c.complex = complex_wf
    c.precision = "mixed" if mixed else "fp64"
    c.mat_dtype = torch.complex128 if complex_wf else torch.float64
    c.dtype = (torch.complex64 if complex_wf else torch.float32) if mixed else c.mat_dtype
    c.max_bands = 8
    c.Ip = ip
    c._dmat_total = dmat_total
    c._h = None
    c._stream = lambda: None
    return c


def bands(c, nb, dtype=None):
    return torch.zeros((nb,) + c.n[::-1], dtype=dtype or c.dtype)


def test_good_arguments_reach_the_library():
    c = shell()
    psi = bands(c, 4)
    P = c.project(psi)
    assert P.shape == (6, 4)
    f = torch.ones(4, dtype=torch.float64)
    c.density(psi, f)
    c.atomic_density(P, f)
    c.poisson(torch.zeros(60, dtype=torch.float64))
    assert c.lib.called == ["pawfd_set_stream", "pawfd_project", "pawfd_set_stream", "pawfd_density",
                            "pawfd_set_stream", "pawfd_atomic_density", "pawfd_set_stream", "pawfd_poisson"]


@pytest.mark.parametrize("case", ["P wrong size", "P wrong dtype", "P not contiguous"])
def test_project_rejects_bad_P(case):
    c = shell()
    psi = bands(c, 4)
    P = {"P wrong size": torch.zeros((6, 3)), "P wrong dtype": torch.zeros((6, 4), dtype=torch.float32),
         "P not contiguous": torch.zeros((4, 6), dtype=torch.float64).t()}[case]
    with pytest.raises(ValueError):
        c.project(psi, P=P)
    assert c.lib.called == []


@pytest.mark.parametrize("case", ["psi dtype", "psi size", "f length", "f dtype", "rho size", "rho dtype",
                                  "rho not contiguous"])
def test_density_rejects_bad_arguments(case):
    c = shell()
    psi, f, rho = bands(c, 4), torch.ones(4, dtype=torch.float64), torch.zeros(60, dtype=torch.float64)
    if case == "psi dtype":
        psi = bands(c, 4, torch.float32)
    elif case == "psi size":
        psi = torch.zeros(4 * 60 + 1, dtype=torch.float64)
    elif case == "f length":
        f = torch.ones(3, dtype=torch.float64)
    elif case == "f dtype":
        f = torch.ones(4, dtype=torch.float32)
    elif case == "rho size":
        rho = torch.zeros(59, dtype=torch.float64)
    elif case == "rho dtype":
        rho = torch.zeros(60, dtype=torch.float32)
    else:
        rho = torch.zeros(120, dtype=torch.float64)[::2]
    with pytest.raises(ValueError):
        c.density(psi, f, rho=rho)
    assert c.lib.called == []


@pytest.mark.parametrize("case", ["f dtype", "P size", "P dtype", "D too short", "D dtype", "D not contiguous"])
def test_atomic_density_rejects_bad_arguments(case):
    c = shell()
    P, f, D = torch.zeros((6, 4), dtype=torch.float64), torch.ones(4, dtype=torch.float64), None
    if case == "f dtype":
        f = torch.ones(4, dtype=torch.float32)
    elif case == "P size":
        P = torch.zeros((6, 5), dtype=torch.float64)
    elif case == "P dtype":
        P = torch.zeros((6, 4), dtype=torch.complex128)
    elif case == "D too short":
        D = torch.zeros(71, dtype=torch.float64)
    elif case == "D dtype":
        D = torch.zeros(72, dtype=torch.float32)
    else:
        D = torch.zeros(144, dtype=torch.float64)[::2]
    with pytest.raises(ValueError):
        c.atomic_density(P, f, D=D)
    assert c.lib.called == []


def test_atomic_density_without_atoms_accepts_an_empty_D():
    c = shell(ip=0, dmat_total=0)
    D = c.atomic_density(torch.zeros((0, 4), dtype=torch.float64), torch.ones(4, dtype=torch.float64))
    assert D.numel() == 0
    c.atomic_density(torch.zeros((0, 4), dtype=torch.float64), torch.ones(4, dtype=torch.float64), D=D)


@pytest.mark.parametrize("case", ["rho size", "rho dtype", "v size", "v dtype", "v not contiguous"])
def test_poisson_rejects_bad_arguments(case):
    c = shell(ip=0, dmat_total=0)
    rho, v = torch.zeros(60, dtype=torch.float64), None
    if case == "rho size":
        rho = torch.zeros(61, dtype=torch.float64)
    elif case == "rho dtype":
        rho = torch.zeros(60, dtype=torch.float32)
    elif case == "v size":
        v = torch.zeros(59, dtype=torch.float64)
    elif case == "v dtype":
        v = torch.zeros(60, dtype=torch.float32)
    else:
        v = torch.zeros(120, dtype=torch.float64)[1::2]
    with pytest.raises(ValueError):
        c.poisson(rho, v=v)
    assert c.lib.called == []


def test_poisson_passes_a_contiguous_copy_of_a_strided_rho():
    c = shell(ip=0, dmat_total=0)
    c.poisson(torch.zeros(120, dtype=torch.float64)[::2])
    assert c.lib.called[-1] == "pawfd_poisson"


def test_rotate_n_and_residual_checks():
    c = shell()
    psi = bands(c, 4)
    C = torch.zeros((4, 4), dtype=torch.float64)
    with pytest.raises(ValueError):
        c.rotate_n(psi, C, 2, out=bands(c, 3))
    with pytest.raises(ValueError):
        c.rotate_n(psi, torch.zeros((3, 3), dtype=torch.float64), 2)
    with pytest.raises(ValueError):
        c.residual_precond(psi, psi, torch.zeros(3, dtype=torch.float64))
    assert c.lib.called == []
    c.rotate_n(psi, C, 2)
    assert c.lib.called[-1] == "pawfd_rotate_n"
