"""Seeded synthetic inputs for the five workloads of the robust spectral-MsFEM solve.

This module holds NO arithmetic of the method: it only draws designs, boundary-condition
masks and load vectors.  Both the CUDA library's tests/benchmark and the CPU oracle take
their inputs from here, so that the two sides never share anything else.

Layouts (shared with the oracle and the CUDA library; plain row-major numpy arrays):
  element field   [nely][nelx]            row 0 = bottom row of elements (y upwards)
  nodal vector    [nely+1][nelx+1][2]     component 0 = x, 1 = y
  design field    [cy][cx] for a periodic unit cell, else the element field itself

Workloads (plane stress, unit square Q4 elements, E0 = 1, Emin = 1e-9, nu = 0.3, p = 3):
  mbb_c1     192x64 MBB beam, 16x16 unit cells, each solid with a centred circular void of
             radius 5 +- U{-1,0,1} elements; full-field design, filter radius 2, beta 8,
             eta 0.5; coarse cells H = 16 with 4 eigenvectors each.
  mbb_c2     1024x512 MBB beam; one 32x32 unit cell whose elements are void with
             probability 0.4 (Bernoulli), tiled periodically; periodic design on the cell,
             filter radius 3, beta 8, eta 0.5; H = 32, 6 eigenvectors.
  mbb_c3     2048x1024 MBB beam of horizontal solid/void layers of thickness U{4..12};
             full-field design, filter radius 3, beta 16, eta in {0.3,0.5,0.7}; H = 32, 6.
  cant_c4    64 cantilevers of sizes drawn from {256x128, 384x192, 512x256, 768x384,
             1024x512}, each a periodic circular-void cell (size from {8,16,32}, void radius
             5/16 of the cell +- 1); filter radius 2, beta 8, eta 0.5; H = 16, 4.
  mbb_c5     3200x4096 MBB beam, periodic 32x32 cell with a void of radius 10; filter radius
             3, beta 8, eta in {0.3,0.5,0.7}; H = 32, 6.

Boundary conditions (the problem statement, Sec. 2.1, fixes only that Dirichlet DOFs are zero):
  MBB        u_x = 0 on the left edge, u_y = 0 at the bottom-right node, F_y = -1 at the
             top-left node.
  cantilever u = 0 on the whole left edge, F_y = -1 at the bottom-right node.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

CONFIG_NAMES = ("mbb_c1", "mbb_c2", "mbb_c3", "cant_c4", "mbb_c5")


@dataclasses.dataclass
class Workload:
    name: str
    nelx: int
    nely: int
    rho: np.ndarray                 # design field (float64), [nely][nelx] or [cy][cx]
    cell: Optional[tuple]           # (cx, cy) when the design is one periodic unit cell
    fixed: np.ndarray               # uint8 [nely+1][nelx+1][2]
    force: np.ndarray               # float64 [nely+1][nelx+1][2]
    nu: float = 0.3
    E0: float = 1.0
    Emin: float = 1e-9
    penal: float = 3.0
    rmin: float = 2.0
    beta: float = 8.0
    etas: tuple = (0.5,)
    H: int = 16
    n_eig: int = 4
    tol: float = 1e-8

    @property
    def n_dof(self) -> int:
        return 2 * (self.nelx + 1) * (self.nely + 1)

    @property
    def n_design(self) -> int:
        return int(self.rho.size)


def mbb_bc(nelx: int, nely: int):
    """MBB half-beam supports and load (see module docstring)."""
    fixed = np.zeros((nely + 1, nelx + 1, 2), dtype=np.uint8)
    fixed[:, 0, 0] = 1
    fixed[0, nelx, 1] = 1
    force = np.zeros((nely + 1, nelx + 1, 2), dtype=np.float64)
    force[nely, 0, 1] = -1.0
    return fixed, force


def cantilever_bc(nelx: int, nely: int):
    """Cantilever clamped on the left edge, tip load at the bottom-right node."""
    fixed = np.zeros((nely + 1, nelx + 1, 2), dtype=np.uint8)
    fixed[:, 0, :] = 1
    force = np.zeros((nely + 1, nelx + 1, 2), dtype=np.float64)
    force[0, nelx, 1] = -1.0
    return fixed, force


def circular_void_cell(size: int, radius: float) -> np.ndarray:
    """One square unit cell, solid (1) with a centred circular void (0); an element is void
    when its centroid lies strictly inside the circle."""
    c = np.arange(size) + 0.5 - size / 2.0
    d2 = c[None, :] ** 2 + c[:, None] ** 2
    return np.where(d2 < radius * radius, 0.0, 1.0)


def jittered_void_tiling(nelx: int, nely: int, cell: int, radius: float, rng) -> np.ndarray:
    """Tiling of circular-void cells whose radius is jittered per cell by U{-1,0,1}."""
    rho = np.empty((nely, nelx))
    for cy in range(nely // cell):
        for cx in range(nelx // cell):
            r = radius + float(rng.integers(-1, 2))
            rho[cy * cell:(cy + 1) * cell, cx * cell:(cx + 1) * cell] = circular_void_cell(cell, r)
    return rho


def layered(nelx: int, nely: int, rng, tmin: int = 4, tmax: int = 12, period: int = 32,
            strut: int = 8) -> np.ndarray:
    """Horizontal layers, alternately solid and void from the bottom, thickness U{tmin..tmax}.
    Every void layer is crossed by solid struts ``strut`` elements wide, one per ``period``
    elements along x, at a seeded offset per layer, so that the stiff layers form one
    connected structure (without them each stiff layer floats on the void material)."""
    rho = np.empty((nely, nelx))
    x = np.arange(nelx)
    y, solid = 0, True
    while y < nely:
        t = int(rng.integers(tmin, tmax + 1))
        if solid:
            rho[y:y + t, :] = 1.0
        else:
            off = int(rng.integers(0, period))
            rho[y:y + t, :] = np.where((x - off) % period < strut, 1.0, 0.0)[None, :]
        y += t
        solid = not solid
    return rho


def make(name: str, scale: int = 1) -> Workload:
    """Build a named workload.  ``scale`` > 1 divides every mesh dimension (and keeps the
    cell / coarse-cell sizes) to make a smaller copy of the same structure for tests."""
    if name == "mbb_c1":
        rng = np.random.default_rng(1)
        nelx, nely = 192 // scale, 64 // scale
        rho = jittered_void_tiling(nelx, nely, 16, 5.0, rng)
        fixed, force = mbb_bc(nelx, nely)
        return Workload(name, nelx, nely, rho, None, fixed, force, rmin=2.0, beta=8.0,
                        etas=(0.5,), H=16, n_eig=4)
    if name == "mbb_c2":
        rng = np.random.default_rng(2)
        nelx, nely = 1024 // scale, 512 // scale
        cell = np.where(rng.random((32, 32)) < 0.4, 0.0, 1.0)
        fixed, force = mbb_bc(nelx, nely)
        return Workload(name, nelx, nely, cell, (32, 32), fixed, force, rmin=3.0, beta=8.0,
                        etas=(0.5,), H=32, n_eig=6)
    if name in ("mbb_c3", "mbb_c3_literal"):
        # mbb_c3_literal: the layers as the configuration states them, without struts (every
        # stiff layer floats on the void material: a mechanism up to Emin)
        rng = np.random.default_rng(3)
        nelx, nely = 2048 // scale, 1024 // scale
        rho = layered(nelx, nely, rng, strut=0 if name == "mbb_c3_literal" else 8)
        fixed, force = mbb_bc(nelx, nely)
        return Workload(name, nelx, nely, rho, None, fixed, force, rmin=3.0, beta=16.0,
                        etas=(0.3, 0.5, 0.7), H=32, n_eig=6)
    if name == "mbb_c5":
        # reduced copies keep whole 32-element cells (and coarse cells)
        nelx, nely = max(64, 3200 // scale // 32 * 32), max(64, 4096 // scale // 32 * 32)
        cell = circular_void_cell(32, 10.0)
        fixed, force = mbb_bc(nelx, nely)
        return Workload(name, nelx, nely, cell, (32, 32), fixed, force, rmin=3.0, beta=8.0,
                        etas=(0.3, 0.5, 0.7), H=32, n_eig=6)
    raise KeyError(name)


def cantilever_batch(n: int = 64, seed: int = 4, scale: int = 1):
    """The uneven-size batch: ``n`` cantilever workloads with seeded sizes and cells."""
    rng = np.random.default_rng(seed)
    sizes = [(256, 128), (384, 192), (512, 256), (768, 384), (1024, 512)]
    out = []
    for b in range(n):
        nelx, nely = sizes[int(rng.integers(0, len(sizes)))]
        nelx, nely = nelx // scale, nely // scale
        csize = int(rng.choice([8, 16, 32]))
        radius = 5.0 / 16.0 * csize + float(rng.integers(-1, 2))
        cell = circular_void_cell(csize, radius)
        fixed, force = cantilever_bc(nelx, nely)
        out.append(Workload(f"cant_c4_{b}", nelx, nely, cell, (csize, csize), fixed, force,
                            rmin=2.0, beta=8.0, etas=(0.5,), H=16, n_eig=4))
    return out


def small(nelx: int, nely: int, seed: int = 0, kind: str = "random", bc: str = "mbb",
          H: int = 4, n_eig: int = 4, rmin: float = 1.5, beta: float = 4.0,
          etas=(0.5,), cell: Optional[tuple] = None, Emin: float = 1e-9) -> Workload:
    """Tiny seeded workloads for tests.  ``kind``: 'random' (U(0,1) densities), 'solid'
    (all ones), 'voids' (circular voids in cells of size H)."""
    rng = np.random.default_rng(seed)
    shape = (cell[1], cell[0]) if cell else (nely, nelx)
    if kind == "random":
        rho = rng.random(shape)
    elif kind == "solid":
        rho = np.ones(shape)
    elif kind == "voids":
        if cell:
            rho = circular_void_cell(cell[0], cell[0] * 5.0 / 16.0)
        else:
            rho = jittered_void_tiling(nelx, nely, H, H * 5.0 / 16.0, rng)
    else:
        raise KeyError(kind)
    fixed, force = (mbb_bc if bc == "mbb" else cantilever_bc)(nelx, nely)
    return Workload(f"small_{kind}_{nelx}x{nely}", nelx, nely, rho, cell, fixed, force,
                    rmin=rmin, beta=beta, etas=tuple(etas), H=H, n_eig=n_eig, Emin=Emin)
