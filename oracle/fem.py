"""Oracle, part 1: Q4 plane-stress finite elements (paper Sec. 2.1, Eq. for K_e in Sec. 2.2).

TEST INFRASTRUCTURE ONLY -- plain FP64 NumPy/SciPy, no blocking or fusion.

The element stiffness K0 (unit Young's modulus, unit square, plane stress, unit thickness)
is obtained by 2x2 Gauss quadrature of B^T C0 B, which integrates the bilinear element
exactly.  The global matrix is assembled in CSR from K_e = E_e K0 (modified SIMP, Sec. 2.2)
and solved with a sparse direct factorisation (SuperLU) on the free DOFs.

Numbering (private to the oracle): node (i, j) -> n = i*(nely+1) + j (column-major),
DOFs 2n (x) and 2n+1 (y); element (ex, ey) -> ex*nely + ey with local nodes
(ex,ey), (ex+1,ey), (ex+1,ey+1), (ex,ey+1).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

# local node offsets (dx, dy), counter-clockwise from the lower-left corner
_LOCAL = ((0, 0), (1, 0), (1, 1), (0, 1))


def shape_gradients(xi: float, eta: float) -> np.ndarray:
    """Gradients of the four bilinear shape functions on [0,1]^2 at (xi, eta): rows = nodes,
    columns = (d/dx, d/dy).  N_a = (1-x or x)(1-y or y)."""
    g = np.empty((4, 2))
    for a, (dx, dy) in enumerate(_LOCAL):
        fx = xi if dx else 1.0 - xi
        fy = eta if dy else 1.0 - eta
        sx = 1.0 if dx else -1.0
        sy = 1.0 if dy else -1.0
        g[a, 0] = sx * fy
        g[a, 1] = sy * fx
    return g


def plane_stress_C(nu: float) -> np.ndarray:
    """Isotropic plane-stress constitutive matrix for unit Young's modulus (Sec. 2.1: C = E C0)."""
    return np.array([[1.0, nu, 0.0], [nu, 1.0, 0.0], [0.0, 0.0, (1.0 - nu) / 2.0]]) / (1.0 - nu * nu)


def element_stiffness(nu: float) -> np.ndarray:
    """K0: 8x8 stiffness of a unit-E unit-square Q4 element by 2x2 Gauss quadrature."""
    C = plane_stress_C(nu)
    gp = (0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0))
    K0 = np.zeros((8, 8))
    for xi in gp:
        for eta in gp:
            g = shape_gradients(xi, eta)
            B = np.zeros((3, 8))
            for a in range(4):
                B[0, 2 * a] = g[a, 0]
                B[1, 2 * a + 1] = g[a, 1]
                B[2, 2 * a] = g[a, 1]
                B[2, 2 * a + 1] = g[a, 0]
            K0 += 0.25 * B.T @ C @ B
    return 0.5 * (K0 + K0.T)   # exact K0 is symmetric; remove quadrature round-off asymmetry


class Grid:
    """A nelx x nely structured mesh of unit-square Q4 elements."""

    def __init__(self, nelx: int, nely: int):
        self.nelx, self.nely = nelx, nely
        self.n_nodes = (nelx + 1) * (nely + 1)
        self.n_dof = 2 * self.n_nodes
        self.n_el = nelx * nely
        ex, ey = np.meshgrid(np.arange(nelx), np.arange(nely), indexing="ij")
        ex, ey = ex.ravel(), ey.ravel()           # oracle element order: ex*nely + ey
        nodes = [self.node(ex + dx, ey + dy) for dx, dy in _LOCAL]
        edof = np.empty((self.n_el, 8), dtype=np.int64)
        for a in range(4):
            edof[:, 2 * a] = 2 * nodes[a]
            edof[:, 2 * a + 1] = 2 * nodes[a] + 1
        self.edof = edof

    def node(self, i, j):
        return i * (self.nely + 1) + j

    # --- conversions between the neutral layouts and the oracle numbering ---------------
    def nodal_from_neutral(self, v: np.ndarray) -> np.ndarray:
        v = np.asarray(v).reshape(self.nely + 1, self.nelx + 1, 2)
        return np.ascontiguousarray(v.transpose(1, 0, 2)).reshape(-1)

    def nodal_to_neutral(self, v: np.ndarray) -> np.ndarray:
        return np.ascontiguousarray(v.reshape(self.nelx + 1, self.nely + 1, 2).transpose(1, 0, 2))

    def element_from_neutral(self, e: np.ndarray) -> np.ndarray:
        return np.ascontiguousarray(np.asarray(e).reshape(self.nely, self.nelx).T).reshape(-1)

    def element_to_neutral(self, e: np.ndarray) -> np.ndarray:
        return np.ascontiguousarray(e.reshape(self.nelx, self.nely).T)


def assemble(grid: Grid, E_el: np.ndarray, K0: np.ndarray) -> sp.csr_matrix:
    """Global stiffness K = sum_e E_e K0 (no boundary conditions).  E_el in oracle order."""
    iK = np.repeat(grid.edof, 8, axis=1).ravel()
    jK = np.tile(grid.edof, (1, 8)).ravel()
    sK = (E_el[:, None] * K0.ravel()[None, :]).ravel()
    return sp.coo_matrix((sK, (iK, jK)), shape=(grid.n_dof, grid.n_dof)).tocsr()


def matvec_unconstrained(grid: Grid, E_el: np.ndarray, K0: np.ndarray, u: np.ndarray) -> np.ndarray:
    """y = K u element by element (the definition Sec. 2.1 gives), oracle numbering."""
    ue = u[grid.edof]                      # [n_el, 8]
    fe = (ue @ K0.T) * E_el[:, None]
    y = np.zeros(grid.n_dof)
    np.add.at(y, grid.edof.ravel(), fe.ravel())
    return y


def element_energy(grid: Grid, K0: np.ndarray, u: np.ndarray) -> np.ndarray:
    """u_e^T K0 u_e per element (oracle element order)."""
    ue = u[grid.edof]
    return np.einsum("ei,ij,ej->e", ue, K0, ue)


class Problem:
    """K(E) u = f with homogeneous Dirichlet conditions given by a per-DOF mask."""

    def __init__(self, grid: Grid, K0: np.ndarray, fixed_neutral: np.ndarray):
        self.grid, self.K0 = grid, K0
        self.fixed = grid.nodal_from_neutral(fixed_neutral).astype(bool)
        self.free = np.flatnonzero(~self.fixed)

    def stiffness(self, E_neutral: np.ndarray) -> sp.csr_matrix:
        return assemble(self.grid, self.grid.element_from_neutral(E_neutral), self.K0)

    def free_matrix(self, E_neutral: np.ndarray) -> sp.csr_matrix:
        K = self.stiffness(E_neutral)
        return K[self.free][:, self.free].tocsc()

    def solve_direct(self, E_neutral: np.ndarray, f_neutral: np.ndarray) -> np.ndarray:
        """u = K^{-1} f on the free DOFs (sparse LU), zero on fixed DOFs; neutral layout."""
        Kf = self.free_matrix(E_neutral)
        f = self.grid.nodal_from_neutral(f_neutral)
        u = np.zeros(self.grid.n_dof)
        u[self.free] = spla.splu(Kf).solve(f[self.free])
        return self.grid.nodal_to_neutral(u)

    def apply(self, E_neutral: np.ndarray, u_neutral: np.ndarray) -> np.ndarray:
        """Constrained operator: y = K u restricted to free DOFs (fixed DOFs of u are taken as
        zero, fixed DOFs of y are set to zero); neutral layout."""
        g = self.grid
        u = g.nodal_from_neutral(u_neutral).copy()
        u[self.fixed] = 0.0
        y = matvec_unconstrained(g, g.element_from_neutral(E_neutral), self.K0, u)
        y[self.fixed] = 0.0
        return g.nodal_to_neutral(y)
