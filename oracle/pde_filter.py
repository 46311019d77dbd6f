"""Oracle, part 5: the PDE (Helmholtz) density filter with periodicity and connectivity
imposed by collapsing degrees of freedom (Sec. 4.3 and 4.5, the filter the paper takes from
Lazarov & Sigmund for designs of several microstructure blocks).

TEST INFRASTRUCTURE ONLY -- plain FP64 NumPy/SciPy.

The filter (restated from its published definition; the paper cites it without equations):
    -r^2 lap(phi) + phi = rho    in the filter domain, natural (Neumann) boundary conditions,
    r = r_min / (2 sqrt(3))      (the length scale that matches a cone filter of radius r_min),
discretised with bilinear Q4 elements of unit size on the design elements:
    K_F = sum_e (r^2 K_e^lap + M_e),    b = T_F rho  (each element adds rho_e / 4 to its nodes),
    rho_tilde_e = (1/4) sum of phi over the element's four nodes  (= T_F^T phi).
Periodicity and connectivity: nodes on edges that are identified share one unknown. With a
collapse matrix P (nodes x collapsed unknowns, one 1 per row) the filter is
    rho_tilde = T_F^T P (P^T K_F P)^-1 P^T T_F rho,
a symmetric operator, so the sensitivity chain uses the same operator.

Domains:
  - ``periodic_cell(nx, ny)``: one unit cell, left/right and bottom/top edges identified (a
    torus): the single periodic microstructure.
  - ``stacked_blocks(nx, heights)``: cells of equal width nx and heights ny_b stacked along y
    (one design cell per block). Each cell's left and right edges are identified
    (horizontal periodicity within its block). The top and bottom edges of all cells are one
    collapsed set (vertical periodicity within each block and connectivity across the
    interfaces). This is the three-layer arrangement of the paper's multi-block figure.
  - ``plain(nx, ny)``: no identification (Neumann on the whole boundary).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def element_matrices() -> tuple[np.ndarray, np.ndarray]:
    """Q4 Laplacian stiffness and consistent mass of the unit square, local nodes
    (0,0), (1,0), (1,1), (0,1): closed forms of int grad N_a . grad N_b and int N_a N_b."""
    Kl = np.array([[4, -1, -2, -1], [-1, 4, -1, -2], [-2, -1, 4, -1], [-1, -2, -1, 4]]) / 6.0
    Me = np.array([[4, 2, 1, 2], [2, 4, 2, 1], [1, 2, 4, 2], [2, 1, 2, 4]]) / 36.0
    return Kl, Me


class Mesh:
    """A set of rectangular cells, each an nx x ny grid of unit elements with its own nodes.
    Elements are numbered cell by cell, row by row (x fastest); the design vector follows the
    same order."""

    def __init__(self, cells: list[tuple[int, int]]):
        self.cells = cells
        self.node_off, self.el_off = [], []
        n_nodes = n_el = 0
        for nx, ny in cells:
            self.node_off.append(n_nodes)
            self.el_off.append(n_el)
            n_nodes += (nx + 1) * (ny + 1)
            n_el += nx * ny
        self.n_nodes, self.n_el = n_nodes, n_el
        conn = []
        for c, (nx, ny) in enumerate(cells):
            o = self.node_off[c]
            for ey in range(ny):
                for ex in range(nx):
                    n0 = o + ey * (nx + 1) + ex
                    conn.append((n0, n0 + 1, n0 + nx + 2, n0 + nx + 1))
        self.conn = np.array(conn, dtype=np.int64)

    def node(self, c: int, i: int, j: int) -> int:
        nx, _ = self.cells[c]
        return self.node_off[c] + j * (nx + 1) + i


def _union_find_collapse(n: int, pairs) -> sp.csr_matrix:
    parent = np.arange(n)

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for a, b in pairs:
        ra, rb = find(a), find(b)
        if ra != rb:
            parent[max(ra, rb)] = min(ra, rb)
    roots = np.array([find(a) for a in range(n)])
    uniq, col = np.unique(roots, return_inverse=True)
    return sp.csr_matrix((np.ones(n), (np.arange(n), col)), shape=(n, uniq.size))


class PDEFilter:
    """rho_tilde = T_F^T P (P^T K_F P)^-1 P^T T_F rho on a Mesh with a collapse matrix P."""

    def __init__(self, mesh: Mesh, rmin: float, pairs=()):
        self.mesh = mesh
        self.r = rmin / (2.0 * np.sqrt(3.0))
        Kl, Me = element_matrices()
        Ke = self.r ** 2 * Kl + Me
        conn = mesh.conn
        rows = np.repeat(conn, 4, axis=1).ravel()
        cols = np.tile(conn, (1, 4)).ravel()
        self.KF = sp.coo_matrix((np.tile(Ke.ravel(), mesh.n_el), (rows, cols)),
                                shape=(mesh.n_nodes, mesh.n_nodes)).tocsr()
        self.TF = sp.coo_matrix((np.full(4 * mesh.n_el, 0.25),
                                 (conn.ravel(), np.repeat(np.arange(mesh.n_el), 4))),
                                shape=(mesh.n_nodes, mesh.n_el)).tocsr()
        self.P = _union_find_collapse(mesh.n_nodes, pairs)
        self.Kc = (self.P.T @ self.KF @ self.P).tocsc()
        self.lu = spla.splu(self.Kc)

    def nodal(self, rho: np.ndarray) -> np.ndarray:
        """The filtered nodal field phi (one value per mesh node)."""
        return self.P @ self.lu.solve(self.P.T @ (self.TF @ rho))

    def apply(self, rho: np.ndarray) -> np.ndarray:
        return self.TF.T @ self.nodal(rho)


def plain(nx: int, ny: int, rmin: float) -> PDEFilter:
    return PDEFilter(Mesh([(nx, ny)]), rmin)


def periodic_cell(nx: int, ny: int, rmin: float) -> PDEFilter:
    m = Mesh([(nx, ny)])
    pairs = [(m.node(0, 0, j), m.node(0, nx, j)) for j in range(ny + 1)]
    pairs += [(m.node(0, i, 0), m.node(0, i, ny)) for i in range(nx + 1)]
    return PDEFilter(m, rmin, pairs)


def stacked_blocks(nx: int, heights, rmin: float) -> PDEFilter:
    m = Mesh([(nx, ny) for ny in heights])
    pairs = []
    for c, ny in enumerate(heights):
        pairs += [(m.node(c, 0, j), m.node(c, nx, j)) for j in range(ny + 1)]   # left = right
        pairs += [(m.node(c, i, 0), m.node(0, i, 0)) for i in range(nx + 1)]     # all bottoms
        pairs += [(m.node(c, i, ny), m.node(0, i, 0)) for i in range(nx + 1)]    # all tops
    return PDEFilter(m, rmin, pairs)
