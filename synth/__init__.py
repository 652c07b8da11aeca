"""Seeded synthetic inputs for the Spectral Quadrature hot path.

This module is the ONLY code shared by the CPU oracle (``oracle/``) and the
CUDA path (``paper_1708_07913_gb300``).  It builds input data and holds none
of the method's arithmetic: atom positions, the local potential V on the
finite-difference grid, projector parameters and the per-workload constants.

The paper's workloads are aluminium and lithium hydride with Troullier-Martins
pseudopotentials (Section 4); those pseudopotentials are not available, so the
stand-in is an FCC aluminium-like crystal (lattice constant 7.65 bohr, 4 atoms
per cubic cell, seeded Gaussian displacements) whose local potential is a sum
of Gaussians over all periodic images, plus optional Gaussian s and p
Kleinman-Bylander projectors.  The grid is the uniform periodic grid of
Section 3.1 with node (i, j, k) at position (i h, j h, k h); arrays are stored
x-fastest, i.e. flat index ``i + n1*(j + n2*k)``, numpy shape ``(n3, n2, n1)``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

LATTICE_A = 7.65          # bohr, FCC cubic lattice constant
V_AMP = -3.0              # Ha, depth of each Gaussian well
V_WIDTH = 0.8             # bohr, Gaussian width of each well
V_CUTOFF = 7.0            # bohr, image-sum cutoff radius (term < 1e-16 * |V_AMP| beyond)
PROJ_RC = 1.5             # bohr, Gaussian width of the projectors
PROJ_RNL = 4.5            # bohr, projector support radius (3 rc)
GAMMA_S = 0.5             # Ha, s-channel Kleinman-Bylander energy
GAMMA_P = -0.3            # Ha, p-channel Kleinman-Bylander energy
ELECTRONS_PER_ATOM = 3.0  # Al 3s2 3p1 valence


@dataclass(frozen=True)
class Workload:
    """One synthetic SQ workload: crystal, grid and SQ parameters."""
    name: str
    cells: int            # FCC cubic cells per axis
    n: int                # grid points per axis
    r_cut: float          # bohr, half-side of the region of influence
    npl: int              # Chebyshev / quadrature degree (multiple of 4)
    kT: float             # Ha, smearing sigma
    sigma_disp: float     # bohr, std-dev of atom displacements
    nonlocal_: bool       # include s + 3p projectors per atom
    seed: int
    n_lanczos: int = 40   # Lanczos iterations for the spectral bounds
    margin: float = 0.01  # relative widening of the Lanczos interval
    fd_half_order: int = 6

    @property
    def L(self) -> float:
        return LATTICE_A * self.cells

    @property
    def h(self) -> float:
        return self.L / self.n

    @property
    def m(self) -> int:
        """Region half-width in grid points: floor(R_cut / h)."""
        return int(math.floor(self.r_cut / self.h + 1e-12))

    @property
    def n_atoms(self) -> int:
        return 4 * self.cells ** 3

    @property
    def n_electrons(self) -> float:
        return ELECTRONS_PER_ATOM * self.n_atoms

    @property
    def n_nodes(self) -> int:
        return self.n ** 3


# The three hot-path workloads: a tiny one-cell case, the 3x3x3-cell case with
# projectors, and the 8x8x8-cell scale case.  Seeds are 1708 + workload index.
WORKLOADS = {
    "al4_16": Workload("al4_16", cells=1, n=16, r_cut=3.0, npl=24, kT=0.1,
                       sigma_disp=0.1, nonlocal_=False, seed=1708),
    "al108_48": Workload("al108_48", cells=3, n=48, r_cut=6.0, npl=48, kT=0.05,
                         sigma_disp=0.15, nonlocal_=True, seed=1709),
    "al2048_128": Workload("al2048_128", cells=8, n=128, r_cut=7.0, npl=64, kT=0.1,
                           sigma_disp=0.2, nonlocal_=True, seed=1712),
    # the learned-warm-start SCF target: 4x4x4 cells (256 atoms), 64^3 grid,
    # with the region, degree and temperature of al108_48
    "al256_64": Workload("al256_64", cells=4, n=64, r_cut=6.0, npl=48, kT=0.05,
                         sigma_disp=0.15, nonlocal_=True, seed=1711),
    # profiling case: same region size, degree and projectors as al108_48 on a
    # 2x2x2-cell (32^3) grid, so the same kernels run on 30% of the nodes
    "al32_32": Workload("al32_32", cells=2, n=32, r_cut=6.0, npl=48, kT=0.05,
                        sigma_disp=0.15, nonlocal_=True, seed=1713),
    # profiling case of the scale workload: its region (29^3), degree,
    # temperature, displacements and projectors on a 2x2x2-cell (32^3) grid
    "al32_32_r7": Workload("al32_32_r7", cells=2, n=32, r_cut=7.0, npl=64, kT=0.1,
                           sigma_disp=0.2, nonlocal_=True, seed=1714),
}


def fcc_positions(cells: int, sigma: float, seed: int, a: float = LATTICE_A) -> np.ndarray:
    """FCC positions (bohr), shape (4*cells^3, 3), displaced by N(0, sigma^2)
    per coordinate and wrapped into [0, L)."""
    basis = np.array([[0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]]) * a
    cell_idx = np.array([(i, j, k) for k in range(cells) for j in range(cells) for i in range(cells)],
                        dtype=np.float64)
    pos = (cell_idx[:, None, :] * a + basis[None, :, :]).reshape(-1, 3)
    rng = np.random.default_rng(seed)
    pos = pos + rng.normal(0.0, sigma, size=pos.shape)
    L = a * cells
    return np.mod(pos, L)


def local_potential(n: int, L: float, pos: np.ndarray, amp: float = V_AMP,
                    width: float = V_WIDTH, cutoff: float = V_CUTOFF) -> np.ndarray:
    """V(x) = sum over atoms and periodic images of amp*exp(-|x-R|^2/(2 width^2)),
    terms with |x-R| >= cutoff dropped.  Returns shape (n, n, n) = (z, y, x)."""
    h = L / n
    V = np.zeros((n, n, n), dtype=np.float64)
    for R in pos:
        lo = [int(math.ceil((R[d] - cutoff) / h)) for d in range(3)]
        hi = [int(math.floor((R[d] + cutoff) / h)) for d in range(3)]
        gi = [np.arange(lo[d], hi[d] + 1) for d in range(3)]
        dx = [gi[d] * h - R[d] for d in range(3)]
        r2 = (dx[2][:, None, None] ** 2 + dx[1][None, :, None] ** 2 + dx[0][None, None, :] ** 2)
        val = np.where(r2 < cutoff * cutoff, amp * np.exp(-r2 / (2.0 * width * width)), 0.0)
        iz, iy, ix = (np.mod(gi[2], n), np.mod(gi[1], n), np.mod(gi[0], n))
        np.add.at(V, np.ix_(iz, iy, ix), val)
    return V


@dataclass
class System:
    """Materialised inputs of one workload."""
    wl: Workload
    positions: np.ndarray
    V: np.ndarray                      # (n, n, n) float64, x fastest
    proj_types: list = field(default_factory=list)   # [(l, gamma, rc, r_nl), ...]


def projector_types(nonlocal_: bool) -> list:
    """Projector channels per atom as (l, gamma [Ha], rc [bohr], r_nl [bohr])."""
    if not nonlocal_:
        return []
    return [(0, GAMMA_S, PROJ_RC, PROJ_RNL), (1, GAMMA_P, PROJ_RC, PROJ_RNL)]


def make_system(wl: Workload | str) -> System:
    if isinstance(wl, str):
        wl = WORKLOADS[wl]
    pos = fcc_positions(wl.cells, wl.sigma_disp, wl.seed)
    V = local_potential(wl.n, wl.L, pos)
    return System(wl=wl, positions=pos, V=np.ascontiguousarray(V),
                  proj_types=projector_types(wl.nonlocal_))


def custom_workload(name: str = "custom", **kw) -> Workload:
    """A workload with explicit parameters (tests use this for edge cases)."""
    base = dict(cells=1, n=16, r_cut=3.0, npl=24, kT=0.1, sigma_disp=0.1,
                nonlocal_=False, seed=1708)
    base.update(kw)
    return Workload(name, **base)


def sample_nodes(n_nodes: int, count: int, seed: int = 7) -> np.ndarray:
    """A seeded, sorted sample of distinct node indices (int64)."""
    rng = np.random.default_rng(seed)
    count = min(count, n_nodes)
    return np.sort(rng.choice(n_nodes, size=count, replace=False)).astype(np.int64)


def batch_workloads(count: int = 16, seed: int = 1724) -> list:
    """Seeded uneven systems for the batched launch: 1^3..4^3 FCC cells,
    nominal h in {0.45, 0.5} (n = round(a c / h)), R_cut in {4, 5, 6, 7} bohr,
    n_pl in {24, 32, 48, 64}, kT uniform in [0.03, 0.2] Ha, displacements
    sigma 0.15 bohr, s + 3p projectors.  The Lanczos bounds are widened by
    2 % rather than 1 %: after the fixed 40 steps a few nodes of these
    systems keep an extreme Ritz value up to ~1 % of the spectrum width
    inside the spectrum (found by the enclosure check |rho^j| <= 1)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        cells = int(rng.integers(1, 5))
        h_nom = float(rng.choice([0.45, 0.5]))
        n = int(round(LATTICE_A * cells / h_nom))
        out.append(Workload(f"batch{count}_{i}", cells=cells, n=n, r_cut=float(rng.choice([4.0, 5.0, 6.0, 7.0])),
                            npl=int(rng.choice([24, 32, 48, 64])), kT=float(rng.uniform(0.03, 0.2)),
                            sigma_disp=0.15, nonlocal_=True, seed=seed + 1 + i, margin=0.02))
    return out
