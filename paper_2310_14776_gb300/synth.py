"""Seeded synthetic inputs for the real-space PAW eigensolver step.

This module only *makes inputs*: random numbers, atom and well positions,
the local potential sampled on the grid, the atom-centred projector functions
sampled on their grid boxes, and the random PAW correction matrices.  It holds
none of the method's arithmetic (no stencil, no projection, no Gram matrix, no
eigensolver); both the CUDA library and the CPU oracle consume what it writes.

Physical setting (the PAW operators of Eq. (dh) in the PAW section of the
paper):  H = -1/2 nabla^2 + v(r) + sum_a sum_ii' |p_i^a> dH^a_ii' <p_i'^a| and
S = 1 + sum_a sum_ii' |p_i^a> dS^a_ii' <p_i'^a|.  The projector functions
p_i^a are setup data ("stored in the setup file" in the same section), so here
they are synthetic setup functions sampled on the grid:

    p_{nu,l,m}(r) = N_{l,nu} * r^l Y_lm(r_hat) * exp(-r^2 / (2 sigma_nu^2)),  r < r_c
                  = 0                                                         r >= r_c

with N_{l,nu} normalising the untruncated function to 1, real solid harmonics
r^l Y_lm in the order s; p_y, p_z, p_x; d_xy, d_yz, d_{3z^2-r^2}, d_xz,
d_{x^2-y^2}, and projector index i = (nu, l, m) nu-major.

Grid convention: N = (N1, N2, N3) points along x, y, z; h_c = L_c / N_c;
point (i1, i2, i3) sits at (i1 h1, i2 h2, i3 h3); arrays are stored
[band][i3][i2][i1] (x fastest).  A projector box is an axis-aligned block of
*unwrapped* grid indices lo_c .. lo_c + n_c - 1 covering the sphere of radius
r_c around the atom; indices outside 0..N_c-1 stand for periodic images.

Random numbers: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) used as a counter-based generator, so any
element can be drawn independently of the others and the stream is identical
on every platform and numpy version.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

BOHR_PER_ANGSTROM = 1.8897261
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream tags (one independent counter stream per kind of random input)
STREAM_PSI_RE = 1
STREAM_PSI_IM = 2
STREAM_ATOMS = 3
STREAM_WELLS = 4
STREAM_DH = 5
STREAM_KPT = 6
STREAM_SIZES = 7


def _mix64(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniform01(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Doubles in [0, 1): element i is mix64(key + (start + i + 1) * gamma) >> 11 scaled by 2^-53."""
    with np.errstate(over="ignore"):
        key = _mix64(np.array([np.uint64(seed) * _GAMMA + np.uint64(stream) * np.uint64(0xD1B54A32D192ED03)],
                              dtype=np.uint64))[0]
        ctr = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = _mix64(key + ctr * _GAMMA)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform(seed: int, stream: int, count: int, lo: float, hi: float, start: int = 0) -> np.ndarray:
    return lo + (hi - lo) * uniform01(seed, stream, start, count)


# ----------------------------------------------------------------------------------------------
# synthetic setup functions
# ----------------------------------------------------------------------------------------------

def solid_harmonics(l: int, x: np.ndarray, y: np.ndarray, z: np.ndarray) -> List[np.ndarray]:
    """r^l Y_lm(r_hat) for real harmonics, in the order of the module docstring."""
    if l == 0:
        return [np.full_like(x, 1.0 / math.sqrt(4.0 * math.pi))]
    if l == 1:
        c = math.sqrt(3.0 / (4.0 * math.pi))
        return [c * y, c * z, c * x]
    if l == 2:
        c = math.sqrt(15.0 / (4.0 * math.pi))
        r2 = x * x + y * y + z * z
        return [c * x * y, c * y * z, math.sqrt(5.0 / (16.0 * math.pi)) * (3.0 * z * z - r2),
                c * x * z, math.sqrt(15.0 / (16.0 * math.pi)) * (x * x - y * y)]
    raise ValueError("l > 2 not provided")


def radial_norm(l: int, sigma: float) -> float:
    """N with N^2 * int_0^inf r^(2l+2) exp(-r^2/sigma^2) dr = 1, i.e. N^2 Gamma(l+3/2) sigma^(2l+3) / 2 = 1."""
    return math.sqrt(2.0 / (math.gamma(l + 1.5) * sigma ** (2 * l + 3)))


@dataclasses.dataclass(frozen=True)
class ProjectorSet:
    """Per-atom projector channels: a list of (l, sigma) radial functions, each giving 2l+1 projectors."""
    channels: Tuple[Tuple[int, float], ...]
    rcut: float

    @property
    def count(self) -> int:
        return sum(2 * l + 1 for l, _ in self.channels)


def projector_values(pset: ProjectorSet, dx: np.ndarray, dy: np.ndarray, dz: np.ndarray) -> np.ndarray:
    """Values of every projector of ``pset`` at displacements (dx, dy, dz) from the atom; shape [I, *dx.shape]."""
    r2 = dx * dx + dy * dy + dz * dz
    inside = r2 < pset.rcut * pset.rcut
    out = []
    for l, sigma in pset.channels:
        radial = radial_norm(l, sigma) * np.exp(-r2 / (2.0 * sigma * sigma)) * inside
        for ylm in solid_harmonics(l, dx, dy, dz):
            out.append(radial * ylm)
    return np.stack(out)


# ----------------------------------------------------------------------------------------------
# the system
# ----------------------------------------------------------------------------------------------

@dataclasses.dataclass
class System:
    """One periodic orthorhombic cell with its grid, local potential, atoms and PAW corrections."""
    n: Tuple[int, int, int]
    cell: Tuple[float, float, float]
    k: Tuple[float, float, float]
    complex_wf: bool
    vloc: np.ndarray                 # [N3][N2][N1] float64
    pos: np.ndarray                  # [A][3] bohr
    nproj: np.ndarray                # [A] int32
    box_lo: np.ndarray               # [A][3] int32 (x, y, z), unwrapped grid indices
    box_n: np.ndarray                # [A][3] int32
    proj: np.ndarray                 # concatenated [I_a][bn3][bn2][bn1] float64 per atom
    proj_off: np.ndarray             # [A+1] int64 offsets into proj
    dH: np.ndarray                   # concatenated [I_a][I_a] per atom
    dS: np.ndarray
    dmat_off: np.ndarray             # [A+1] int64 offsets into dH / dS
    pset: Optional[ProjectorSet] = None
    wells: Optional[np.ndarray] = None

    @property
    def h(self) -> Tuple[float, float, float]:
        return tuple(self.cell[c] / self.n[c] for c in range(3))

    @property
    def dV(self) -> float:
        h = self.h
        return h[0] * h[1] * h[2]

    @property
    def npoints(self) -> int:
        return self.n[0] * self.n[1] * self.n[2]

    @property
    def natoms(self) -> int:
        return int(self.pos.shape[0])

    @property
    def nproj_total(self) -> int:
        return int(self.nproj.sum())

    @property
    def proj_row_off(self) -> np.ndarray:
        """First global projector row of each atom in the [Ip][nb] projection matrix."""
        return np.concatenate([[0], np.cumsum(self.nproj)]).astype(np.int64)


def vloc_gaussian_wells(n, cell, wells: np.ndarray, depth: float = 1.0, width: float = 1.0) -> np.ndarray:
    """v(r) = -depth * sum_w sum_T exp(-|r - R_w - T|^2 / (2 width^2)), periodic images until < 1e-18.

    The Gaussian factorises over axes, so the image sum is taken per axis.
    """
    reach = width * math.sqrt(2.0 * math.log(1e18))
    v = np.zeros((n[2], n[1], n[0]))
    for w in wells:
        f = []
        for c in range(3):
            x = np.arange(n[c]) * (cell[c] / n[c])
            tmax = int(math.ceil(reach / cell[c])) + 1
            s = np.zeros(n[c])
            for t in range(-tmax, tmax + 1):
                d = x - w[c] - t * cell[c]
                s += np.exp(-d * d / (2.0 * width * width))
            f.append(s)
        v -= depth * f[2][:, None, None] * f[1][None, :, None] * f[0][None, None, :]
    return v


def make_system(n: Sequence[int], cell: Sequence[float], natoms: int, pset: ProjectorSet, seed: int,
                nwells: int = 2, k: Sequence[float] = (0.0, 0.0, 0.0), complex_wf: bool = False,
                dH_scale: float = 0.1, dS_diag: float = 0.05) -> System:
    """Seeded atoms and wells uniform in the cell; dH^a = (B + B^T)/2 with B_ij ~ U(-dH_scale, dH_scale);
    dS^a = dS_diag * I."""
    cell_a = np.array([float(v) for v in cell])
    pos = uniform(seed, STREAM_ATOMS, 3 * natoms, 0.0, 1.0).reshape(natoms, 3) * cell_a
    wells = uniform(seed, STREAM_WELLS, 3 * nwells, 0.0, 1.0).reshape(nwells, 3) * cell_a
    I = pset.count
    dH, dS = [], []
    for a in range(natoms):
        B = uniform(seed, STREAM_DH, I * I, -dH_scale, dH_scale, start=a * I * I).reshape(I, I)
        dH.append((B + B.T) / 2.0)
        dS.append(dS_diag * np.eye(I))
    return build_system(n, cell, pos, wells, pset, dH, dS, k=k, complex_wf=complex_wf)


def projector_box(center: Sequence[float], rcut: float, h: Sequence[float]):
    """Unwrapped index range lo_c .. lo_c + n_c - 1 of the grid points within rcut of ``center`` per axis."""
    lo = [math.ceil((center[c] - rcut) / h[c]) for c in range(3)]
    hi = [math.floor((center[c] + rcut) / h[c]) for c in range(3)]
    return lo, [hi[c] - lo[c] + 1 for c in range(3)]


def build_system(n: Sequence[int], cell: Sequence[float], pos: np.ndarray, wells: np.ndarray, pset: ProjectorSet,
                 dH: Sequence[np.ndarray], dS: Sequence[np.ndarray], k: Sequence[float] = (0.0, 0.0, 0.0),
                 complex_wf: bool = False) -> System:
    """A system with given atom and well positions and per-atom correction matrices."""
    n = tuple(int(v) for v in n)
    cell = tuple(float(v) for v in cell)
    h = [cell[c] / n[c] for c in range(3)]
    pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    natoms = pos.shape[0]
    vloc = vloc_gaussian_wells(n, cell, np.asarray(wells, dtype=np.float64).reshape(-1, 3))
    I = pset.count
    box_lo = np.zeros((natoms, 3), np.int32)
    box_n = np.zeros((natoms, 3), np.int32)
    projs = []
    for a in range(natoms):
        lo, bn = projector_box(pos[a], pset.rcut, h)
        box_lo[a], box_n[a] = lo, bn
        axes = [np.arange(lo[c], lo[c] + bn[c]) * h[c] - pos[a, c] for c in range(3)]
        dz, dy, dx = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
        projs.append(projector_values(pset, dx, dy, dz).reshape(-1))
    proj_off = np.concatenate([[0], np.cumsum([p.size for p in projs])]).astype(np.int64)
    dmat_off = (np.arange(natoms + 1) * I * I).astype(np.int64)
    flat = lambda blocks: np.concatenate([np.asarray(b, np.float64).reshape(-1) for b in blocks]) if natoms else np.zeros(0)
    return System(n=n, cell=cell, k=tuple(float(v) for v in k), complex_wf=bool(complex_wf), vloc=vloc, pos=pos,
                  nproj=np.full(natoms, I, np.int32), box_lo=box_lo, box_n=box_n,
                  proj=np.concatenate(projs) if projs else np.zeros(0), proj_off=proj_off,
                  dH=flat(dH), dS=flat(dS), dmat_off=dmat_off, pset=pset, wells=np.asarray(wells).reshape(-1, 3))

def make_psi(system: System, nb: int, seed: int, band0: int = 0) -> np.ndarray:
    """Seeded uniform(-1, 1) noise, [nb][N3][N2][N1]; float64, or complex128 with independent real/imag parts."""
    K = system.npoints
    shape = (nb, system.n[2], system.n[1], system.n[0])
    re = np.empty(nb * K)
    for b in range(nb):
        re[b * K:(b + 1) * K] = uniform(seed, STREAM_PSI_RE, K, -1.0, 1.0, start=(band0 + b) * K)
    if not system.complex_wf:
        return re.reshape(shape)
    im = np.empty(nb * K)
    for b in range(nb):
        im[b * K:(b + 1) * K] = uniform(seed, STREAM_PSI_IM, K, -1.0, 1.0, start=(band0 + b) * K)
    return (re + 1j * im).reshape(shape)


def with_corrections(system: System, dH: Optional[np.ndarray] = None, dS: Optional[np.ndarray] = None) -> System:
    """A copy of ``system`` with its PAW correction matrices replaced (used for the NCPP special cases)."""
    return dataclasses.replace(system, dH=system.dH.copy() if dH is None else dH,
                               dS=system.dS.copy() if dS is None else dS)


def without_atoms(system: System) -> System:
    return dataclasses.replace(system, pos=np.zeros((0, 3)), nproj=np.zeros(0, np.int32),
                               box_lo=np.zeros((0, 3), np.int32), box_n=np.zeros((0, 3), np.int32),
                               proj=np.zeros(0), proj_off=np.zeros(1, np.int64), dH=np.zeros(0), dS=np.zeros(0),
                               dmat_off=np.zeros(1, np.int64))


def free_grid(system: System) -> System:
    """The same cell and grid with v = 0, no atoms and k = 0: the operator T alone (the
    Laplacian of the Poisson solve)."""
    s = without_atoms(system)
    return dataclasses.replace(s, vloc=np.zeros_like(system.vloc), k=(0.0, 0.0, 0.0), complex_wf=False, wells=None)


# ----------------------------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------------------------

PSET_SP = ProjectorSet(channels=((0, 0.5), (1, 0.5)), rcut=2.0)                    # 4 projectors: s + 3 p
PSET_SPD2 = ProjectorSet(channels=((0, 0.5), (1, 0.5), (2, 0.5), (0, 0.8), (1, 0.8), (2, 0.8)), rcut=2.0)  # 18

H_02A = 0.2 * BOHR_PER_ANGSTROM     # grid spacing 0.2 Angstrom in bohr


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    n: Tuple[int, int, int]
    cell: Tuple[float, float, float]
    nbands: int
    natoms: int
    pset: ProjectorSet
    seed: int
    complex_wf: bool = False
    k: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    iterations: int = 1

    def system(self) -> System:
        return make_system(self.n, self.cell, self.natoms, self.pset, self.seed, k=self.k, complex_wf=self.complex_wf)

    def psi(self, system: System, nb: Optional[int] = None, band0: int = 0) -> np.ndarray:
        return make_psi(system, self.nbands if nb is None else nb, self.seed, band0=band0)


def _bloch_k(cell):
    return (2 * math.pi * 0.25 / cell[0], 2 * math.pi * 0.125 / cell[1], 2 * math.pi * 0.375 / cell[2])


WORKLOADS = {
    # 10 bohr cube, 24^3 grid, 16 real bands, 2 atoms x (s + p), one apply_H/apply_S + Rayleigh-Ritz
    "gamma-24c-16b": Workload("gamma-24c-16b", (24, 24, 24), (10.0, 10.0, 10.0), 16, 2, PSET_SP, seed=0),
    # 96^3 grid at 0.2 Angstrom, 256 real bands, 32 atoms x 18 projectors, ten iterations
    "gamma-96c-256b": Workload("gamma-96c-256b", (96, 96, 96), (96 * H_02A,) * 3, 256, 32, PSET_SPD2, seed=1,
                               iterations=10),
    # 64^3 grid at 0.2 Angstrom, 128 real bands, 8 atoms x 18 projectors: the small case for
    # profiler captures (band arrays of 268 MB, larger than L2)
    "gamma-64c-128b": Workload("gamma-64c-128b", (64, 64, 64), (64 * H_02A,) * 3, 128, 8, PSET_SPD2, seed=5),
    # 144^3 grid at 0.2 Angstrom, 1024 complex bands at one Bloch k-point, 128 atoms x 18 projectors
    "bloch-144c-1024b": Workload("bloch-144c-1024b", (144, 144, 144), (144 * H_02A,) * 3, 1024, 128, PSET_SPD2,
                                 seed=2, complex_wf=True, k=_bloch_k((144 * H_02A,) * 3)),
}


# ------------------------------------------------------------------------------------------
# Batched and served instances: independent systems of different sizes
# ------------------------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class Instance:
    """One eigensolver instance of a batch or of the served stream: grid, cell at 0.2 Angstrom
    spacing, band count, atoms (18 projectors each), Bloch vector, seed."""
    n: Tuple[int, int, int]
    nbands: int
    natoms: int
    seed: int
    complex_wf: bool
    k: Tuple[float, float, float]

    @property
    def cell(self) -> Tuple[float, float, float]:
        return tuple(self.n[c] * H_02A for c in range(3))

    @property
    def npoints(self) -> int:
        return self.n[0] * self.n[1] * self.n[2]

    def system(self) -> System:
        return make_system(self.n, self.cell, self.natoms, PSET_SPD2, self.seed, k=self.k,
                           complex_wf=self.complex_wf)

    def psi(self, system: System) -> np.ndarray:
        return make_psi(system, self.nbands, self.seed)


def batch_instance(seed: int, complex_wf: bool = True, grid=(32, 80), bands=(32, 256), atoms=(2, 24)) -> Instance:
    """Seeded sizes of one batched instance: each grid axis and the band and atom counts are
    independent uniform integers in the given inclusive ranges; for Bloch instances each
    component of k is uniform in [0, pi / L_c)."""
    u = uniform01(seed, STREAM_SIZES, 0, 5)
    n = tuple(int(grid[0] + min(grid[1] - grid[0], int(u[c] * (grid[1] - grid[0] + 1)))) for c in range(3))
    nb = int(bands[0] + min(bands[1] - bands[0], int(u[3] * (bands[1] - bands[0] + 1))))
    na = int(atoms[0] + min(atoms[1] - atoms[0], int(u[4] * (atoms[1] - atoms[0] + 1))))
    k = (0.0, 0.0, 0.0)
    if complex_wf:
        uk = uniform01(seed, STREAM_KPT, 0, 3)
        k = tuple(float(uk[c] * math.pi / (n[c] * H_02A)) for c in range(3))
    return Instance(n, nb, na, seed, complex_wf, k)


def batch_instances(count: int = 64, seed0: int = 3, complex_wf: bool = True, **ranges) -> List[Instance]:
    """The batched workload: `count` instances with seeds seed0, seed0 + 1, ..."""
    return [batch_instance(seed0 + i, complex_wf, **ranges) for i in range(count)]


def served_job(job_id: int, seed0: int = 4, complex_wf: bool = True, large_fraction: float = 0.1,
               large=((128, 128, 128), 512, 24), **ranges) -> Instance:
    """One job of the served stream: with probability `large_fraction` a large job (grid,
    bands, atoms of `large`), otherwise sized as a batched instance."""
    seed = seed0 + job_id
    if uniform01(seed, STREAM_SIZES, 5, 1)[0] < large_fraction:
        n, nb, na = large
        k = (0.0, 0.0, 0.0)
        if complex_wf:
            uk = uniform01(seed, STREAM_KPT, 0, 3)
            k = tuple(float(uk[c] * math.pi / (n[c] * H_02A)) for c in range(3))
        return Instance(tuple(n), nb, na, seed, complex_wf, k)
    return batch_instance(seed, complex_wf, **ranges)


def poisson_arrivals(rate: float, count: int, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson stream: cumulative exponential gaps -ln(1 - u) / rate."""
    u = uniform01(seed, STREAM_SIZES, 1 << 20, count)
    return np.cumsum(-np.log1p(-u) / rate)
