"""Oracle, part 2: the design chain and its adjoint (paper Sec. 2.2, 4.1-4.4).

TEST INFRASTRUCTURE ONLY -- plain FP64 NumPy/SciPy.

  density filter     rho~_e = sum_j w_ej rho_j / sum_j w_ej,  w_ej = max(0, rmin - |x_e - x_j|)
                     (the standard neighbourhood filter of Sec. 4.3; centroid distances in
                     element units; the sum runs over elements inside the design domain).
                     Periodic mode (Sec. 4.3, single periodic microstructure): the design is
                     one unit cell and neighbours wrap around it, which equals filtering a
                     3x3 block of cells and keeping the centre cell.
  projection         rho_bar = (tanh(beta eta) + tanh(beta (rho~ - eta)))
                               / (tanh(beta eta) + tanh(beta (1 - eta)))         (Sec. 4.3)
  modified SIMP      E = Emin + (E0 - Emin) rho_bar^p                             (Sec. 2.2)
  compliance         c = f^T u                                                    (Sec. 2.2)
  sensitivity        dc/drho_bar_e = -p (E0 - Emin) rho_bar_e^(p-1) u_e^T K0 u_e  (Sec. 4.2)
  periodic designs   a design variable's sensitivity is the sum over all fine elements it
                     controls (Sec. 4.1)
  robust objective   f = mean_k c_k + kappa * std_k c_k, equal weights, population
                     variance, kappa = 1, eta in {0.3, 0.5, 0.7}                  (Sec. 4.4)
Element fields use the neutral [ny][nx] layout, flattened row-major for the filter matrix.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def filter_weights(nx: int, ny: int, rmin: float, periodic: bool) -> sp.csr_matrix:
    """Unnormalised weight matrix W[e, j] = max(0, rmin - dist(e, j)) on an nx x ny element
    grid (row-major flattening e = y*nx + x).  Periodic: indices wrap around the grid."""
    R = int(np.ceil(rmin))
    rows, cols, vals = [], [], []
    ey, ex = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    ex, ey = ex.ravel(), ey.ravel()
    for dy in range(-R, R + 1):
        for dx in range(-R, R + 1):
            w = rmin - np.hypot(dx, dy)
            if w <= 0.0:
                continue
            jx, jy = ex + dx, ey + dy
            if periodic:
                jx, jy = jx % nx, jy % ny
                ok = np.ones_like(jx, dtype=bool)
            else:
                ok = (jx >= 0) & (jx < nx) & (jy >= 0) & (jy < ny)
            rows.append((ey * nx + ex)[ok])
            cols.append((jy * nx + jx)[ok])
            vals.append(np.full(int(ok.sum()), w))
    n = nx * ny
    W = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n)).tocsr()
    W.sum_duplicates()
    return W


def filter_matrix(nx: int, ny: int, rmin: float, periodic: bool) -> sp.csr_matrix:
    """Row-normalised filter H = diag(1 / W 1) W."""
    W = filter_weights(nx, ny, rmin, periodic)
    s = np.asarray(W.sum(axis=1)).ravel()
    return sp.diags(1.0 / s) @ W


def heaviside(rt, beta: float, eta: float):
    den = np.tanh(beta * eta) + np.tanh(beta * (1.0 - eta))
    return (np.tanh(beta * eta) + np.tanh(beta * (rt - eta))) / den


def heaviside_deriv(rt, beta: float, eta: float):
    den = np.tanh(beta * eta) + np.tanh(beta * (1.0 - eta))
    return beta * (1.0 - np.tanh(beta * (rt - eta)) ** 2) / den


def simp(rb, E0: float, Emin: float, p: float):
    return Emin + (E0 - Emin) * rb ** p


def simp_deriv(rb, E0: float, Emin: float, p: float):
    return p * (E0 - Emin) * rb ** (p - 1.0)


class DesignChain:
    """rho (design) -> rho~ -> rho_bar_k -> E_k on the full nelx x nely mesh."""

    def __init__(self, nelx: int, nely: int, rmin: float, beta: float, etas, cell=None,
                 E0: float = 1.0, Emin: float = 1e-9, penal: float = 3.0):
        self.nelx, self.nely, self.cell = nelx, nely, cell
        self.beta, self.etas = beta, tuple(etas)
        self.E0, self.Emin, self.penal = E0, Emin, penal
        if cell is None:
            self.dx, self.dy = nelx, nely
        else:
            self.dx, self.dy = cell
            assert nelx % self.dx == 0 and nely % self.dy == 0
        self.H = filter_matrix(self.dx, self.dy, rmin, periodic=cell is not None)

    def to_mesh(self, d: np.ndarray) -> np.ndarray:
        """Design-domain field -> fine mesh (tiling for periodic designs)."""
        d = d.reshape(self.dy, self.dx)
        if self.cell is None:
            return d.copy()
        return np.tile(d, (self.nely // self.dy, self.nelx // self.dx))

    def tile_sum(self, g: np.ndarray) -> np.ndarray:
        """Adjoint of to_mesh: sum the fine-mesh field over all copies of the cell."""
        if self.cell is None:
            return g.reshape(self.dy, self.dx).copy()
        ty, tx = self.nely // self.dy, self.nelx // self.dx
        return g.reshape(ty, self.dy, tx, self.dx).sum(axis=(0, 2))

    def forward(self, rho: np.ndarray) -> dict:
        rt = (self.H @ rho.reshape(-1)).reshape(self.dy, self.dx)
        rbar = [heaviside(rt, self.beta, eta) for eta in self.etas]
        E = [simp(self.to_mesh(rb), self.E0, self.Emin, self.penal) for rb in rbar]
        return {"rho_tilde": rt, "rho_bar": rbar, "E": E}

    def element_sensitivity(self, rb_mesh: np.ndarray, energy_mesh: np.ndarray) -> np.ndarray:
        """dc/drho_bar_e = -dE/drho_bar * u_e^T K0 u_e (self-adjoint compliance, Sec. 4.2)."""
        return -simp_deriv(rb_mesh, self.E0, self.Emin, self.penal) * energy_mesh

    def backward(self, rho: np.ndarray, dcdrb_mesh: list, weights) -> np.ndarray:
        """d/drho of sum_k weights_k c_k given per-realisation fine-mesh dc_k/drho_bar."""
        fw = self.forward(rho)
        g = np.zeros((self.dy, self.dx))
        for k, eta in enumerate(self.etas):
            g += weights[k] * self.tile_sum(dcdrb_mesh[k]) * heaviside_deriv(fw["rho_tilde"], self.beta, eta)
        return (self.H.T @ g.reshape(-1)).reshape(self.dy, self.dx)


def robust_combine(c, kappa: float = 1.0):
    """f = mean(c) + kappa*std(c) (population std) and df/dc_k (Sec. 4.4)."""
    c = np.asarray(c, dtype=np.float64)
    n = c.size
    mu = c.mean()
    sigma = np.sqrt(np.mean((c - mu) ** 2))
    if sigma > 1e-300 * max(abs(mu), 1e-300) and n > 1:
        w = 1.0 / n + kappa * (c - mu) / (n * sigma)
    else:
        w = np.full(n, 1.0 / n)
    return mu + kappa * sigma, w
