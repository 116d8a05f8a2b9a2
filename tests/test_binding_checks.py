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


@pytest.mark.parametrize("case", ["apply_H out short", "apply_H P dtype", "apply_hs Spsi short", "apply_hs P short",
                                  "gram_hs P dtype", "subspace eps dtype", "subspace eps short", "rotate out short",
                                  "rr_step out short", "rr_step work Hpsi short", "rr_step eps dtype",
                                  "refine eps short", "refine Hpsi short", "refine C_lo shape",
                                  "residual rnorm dtype",
                                  "davidson eps_in not contiguous"])
def test_step_calls_reject_short_or_mistyped_outputs(case):
    c = shell()
    nb = 4
    psi = bands(c, nb)
    M = lambda: torch.zeros((nb, nb), dtype=torch.float64)  # noqa: E731
    f64 = lambda n: torch.zeros(n, dtype=torch.float64)  # noqa: E731
    calls = {
        "apply_H out short": lambda: c.apply_H(psi, out=bands(c, 3)),
        "apply_H P dtype": lambda: c.apply_H(psi, P=torch.zeros((6, nb), dtype=torch.float32)),
        "apply_hs Spsi short": lambda: c.apply_hs(psi, Spsi=bands(c, 3)),
        "apply_hs P short": lambda: c.apply_hs(psi, P=torch.zeros((6, 3), dtype=torch.float64)),
        "gram_hs P dtype": lambda: c.gram_hs(psi, psi, torch.zeros((6, nb), dtype=torch.complex128)),
        "subspace eps dtype": lambda: c.subspace_diag(M(), M(), eps=torch.zeros(nb, dtype=torch.float32)),
        "subspace eps short": lambda: c.subspace_diag(M(), M(), eps=f64(3)),
        "rotate out short": lambda: c.rotate(psi, M(), out=bands(c, 3)),
        "rr_step out short": lambda: c.rr_step(psi, out=bands(c, 3)),
        "rr_step work Hpsi short": lambda: c.rr_step(psi, work=dict(c.alloc_work(nb), Hpsi=bands(c, 3))),
        "rr_step eps dtype": lambda: c.rr_step(psi, work=dict(c.alloc_work(nb), eps=torch.zeros(nb, dtype=torch.float32))),
        "refine eps short": lambda: c.refine(bands(c, nb, torch.float32), work={"eps": f64(3)}),
        "refine Hpsi short": lambda: c.refine(bands(c, nb, torch.float32), work={"Hpsi": bands(c, 3)}),
        "refine C_lo shape": lambda: c.refine(bands(c, nb, torch.float32), torch.zeros((3, 3), dtype=torch.float64)),
        "residual rnorm dtype": lambda: c.residual_precond(psi, psi, f64(nb), rnorm=torch.zeros(nb, dtype=torch.float32)),
        "davidson eps_in not contiguous": lambda: c.davidson_step(c.alloc_davidson(nb), nb, f64(2 * nb)[::2]),
    }
    with pytest.raises(ValueError):
        calls[case]()
    assert c.lib.called == []


def test_step_calls_accept_their_own_allocations():
    c = shell()
    nb = 4
    psi = bands(c, nb)
    c.rayleigh_ritz(psi, check=False)
    c.rr_step(psi)
    c.refine(bands(c, nb, torch.float32), check=False)
    c.refine(bands(c, nb, torch.float32), torch.zeros((nb, nb), dtype=torch.float64), check=False)
    w = c.alloc_davidson(nb)
    c.davidson_step(w, nb, torch.zeros(nb, dtype=torch.float64))
    c.residual_precond(psi, psi, torch.zeros(nb, dtype=torch.float64))
    called = [n for n in c.lib.called if n != "pawfd_set_stream"]
    assert called == ["pawfd_apply_HS", "pawfd_gram_hs", "pawfd_subspace_diag", "pawfd_rotate", "pawfd_rr_step",
                      "pawfd_refine", "pawfd_refine", "pawfd_davidson_step", "pawfd_residual_precond"]
