"""Oracle, part 3: spectral MsFEM coarse space and the two-level preconditioned CG
(paper Sec. 2.4, 2.4.1, 2.4.2, 3.2).

TEST INFRASTRUCTURE ONLY -- plain FP64 NumPy/SciPy.

Steps, in the order of Sec. 2.4:
  1. coarse mesh of H x H cells; coarse node y_i = (I*H, J*H), I in [0, nelx/H], J in [0, nely/H]
  2. agglomerate omega_i = union of the coarse cells touching y_i (clipped at the domain edge)
  3. local generalised eigenproblem K_omega psi = lambda M_omega psi (Eq. discrete_aggeigenprob)
     with M_omega = diag(K_omega) (Sec. 3.2).  K_omega is assembled from the elements inside
     omega_i only (no condition on the artificial boundary) and keeps the physical Dirichlet
     conditions by dropping those DOFs (Sec. 2.4).  Eigenvalues ascending; either a fixed
     number k per agglomerate or all lambda < lambda_Omega, capped at k.
  4. partition of unity chi_i: the bilinear coarse hat of y_i (chi in H^1, |grad chi| <= 1/H,
     sum_i chi_i = 1); phi_ij = I_h(chi_i psi_j) at the fine nodes
  5. R_c^T = [phi_1 ... phi_Nt], K_c = R_c K R_c^T (Eq. coarse_projection), dense Cholesky
  6. two-level additive Schwarz preconditioner (Galvis & Efendiev, cited in Sec. 2.4.2):
     M^-1 r = R_c^T K_c^-1 R_c r + sum_i R_i^T K_i^-1 R_i r, where K_i = K restricted to the
     free DOFs of the nodes of omega_i that are not on its artificial boundary (zero
     Dirichlet there, physical conditions kept); exact local solves by sparse LU
  7. preconditioned CG on the free DOFs (Sec. 2.4.2 notes K and M are SPD so PCG applies),
     x0 = 0, stopped on the true relative residual ||f - K u|| / ||f||.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem


class Agglomerate:
    def __init__(self, I: int, J: int, H: int, nelx: int, nely: int):
        self.I, self.J = I, J
        self.x0, self.x1 = max(0, (I - 1) * H), min(nelx, (I + 1) * H)
        self.y0, self.y1 = max(0, (J - 1) * H), min(nely, (J + 1) * H)
        self.nx, self.ny = self.x1 - self.x0, self.y1 - self.y0   # elements
        # nodes of the closed box, local column-major numbering
        ii, jj = np.meshgrid(np.arange(self.x0, self.x1 + 1), np.arange(self.y0, self.y1 + 1), indexing="ij")
        self.node_i, self.node_j = ii.ravel(), jj.ravel()
        # a box side is artificial when it lies inside the domain
        art = np.zeros(self.node_i.size, dtype=bool)
        if self.x0 > 0:
            art |= self.node_i == self.x0
        if self.x1 < nelx:
            art |= self.node_i == self.x1
        if self.y0 > 0:
            art |= self.node_j == self.y0
        if self.y1 < nely:
            art |= self.node_j == self.y1
        self.artificial = art

    def chi(self, H: int) -> np.ndarray:
        """Bilinear coarse hat of y_i at the box nodes."""
        cx, cy = self.I * H, self.J * H
        return (np.maximum(0.0, 1.0 - np.abs(self.node_i - cx) / H)
                * np.maximum(0.0, 1.0 - np.abs(self.node_j - cy) / H))

    def global_dofs(self, grid: fem.Grid) -> np.ndarray:
        n = grid.node(self.node_i, self.node_j)
        return np.stack([2 * n, 2 * n + 1], axis=1).ravel()

    def local_stiffness(self, E_neutral: np.ndarray, K0: np.ndarray) -> sp.csr_matrix:
        """Neumann matrix of the agglomerate: sum of E_e K0 over its own elements."""
        g = fem.Grid(self.nx, self.ny)
        E = E_neutral[self.y0:self.y1, self.x0:self.x1]
        return fem.assemble(g, g.element_from_neutral(E), K0)


def local_eigenpairs(Kw: sp.spmatrix, k: int, dense_limit: int = 900):
    """k smallest eigenpairs of Kw psi = lambda diag(Kw) psi, psi^T D psi = 1.
    Dense generalised eigh for small problems; otherwise shift-invert Lanczos around a
    slightly negative shift (K_omega is singular for floating agglomerates)."""
    n = Kw.shape[0]
    D = Kw.diagonal()
    k = min(k, n)
    if n <= dense_limit or k >= n - 1:
        lam, psi = sla.eigh(Kw.toarray(), np.diag(D))
        lam, psi = lam[:k], psi[:, :k]
    else:
        # shift-invert Lanczos for a block of 2k vectors, then a few steps of block inverse
        # iteration with the same shifted factor and a Rayleigh-Ritz projection to polish
        sigma = -1e-6
        m = min(2 * k + 2, n - 2)
        Dm = sp.diags(D).tocsc()
        _, X = spla.eigsh(Kw.tocsc(), k=m, M=Dm, sigma=sigma, which="LM", tol=1e-12, maxiter=10000)
        lu = spla.splu((Kw - sigma * Dm).tocsc())
        for _ in range(3):
            X = lu.solve(D[:, None] * X)
            X, _ = np.linalg.qr(X)
        A = X.T @ (Kw @ X)
        B = X.T @ (D[:, None] * X)
        lam, Y = sla.eigh(0.5 * (A + A.T), 0.5 * (B + B.T))
        lam, psi = lam[:k], X @ Y[:, :k]
    nrm = np.sqrt(np.einsum("ij,i,ij->j", psi, D, psi))
    return lam, psi / nrm


class TwoLevel:
    """The spectral coarse space and the additive two-level preconditioner on free DOFs.

    basis: another TwoLevel whose coarse basis (agglomerates, eigenvectors, R_c) is taken as
    it is, while K_c = R_c K R_c^T and the patch matrices come from E_neutral.  This is the
    robust formulation's shared preconditioner (Sec. 5.3): the basis of the dilated design
    serves every realisation, each realisation keeping its own operator K.

    Identical local matrices have identical eigenpairs and factors, so each distinct
    agglomerate matrix is eigen-solved once and each distinct patch matrix factorised once
    (the unique agglomerates of a periodic microstructure, Sec. 2.4.1); the key is the
    matrix itself (its CSR arrays, byte for byte)."""

    def __init__(self, prob: fem.Problem, E_neutral: np.ndarray, H: int, n_eig: int,
                 lam_thresh: float | None = None, with_patches: bool = True,
                 dense_limit: int = 900, basis: "TwoLevel | None" = None):
        g = prob.grid
        assert g.nelx % H == 0 and g.nely % H == 0, "mesh must be a whole number of coarse cells"
        self.prob, self.H = prob, H
        self.ncx, self.ncy = g.nelx // H, g.nely // H
        self.K = prob.free_matrix(E_neutral)
        if basis is not None:
            assert basis.prob is prob and basis.H == H
            self.aggs, self.eigvals, self.Nt = basis.aggs, basis.eigvals, basis.Nt
            self.RcT, patch_dofs = basis.RcT, basis.patch_dofs
        else:
            n_free = prob.free.size
            pos = -np.ones(g.n_dof, dtype=np.int64)
            pos[prob.free] = np.arange(n_free)
            self.aggs, self.eigvals = [], []
            cols, rows, vals = [], [], []
            patch_dofs = []
            memo = {}
            t = 0
            for J in range(self.ncy + 1):
                for I in range(self.ncx + 1):
                    a = Agglomerate(I, J, H, g.nelx, g.nely)
                    gd = a.global_dofs(g)
                    keep = ~prob.fixed[gd]
                    Kw = sp.csr_matrix(a.local_stiffness(E_neutral, prob.K0)[keep][:, keep])
                    key = _matrix_key(Kw)
                    if key not in memo:
                        memo[key] = local_eigenpairs(Kw, n_eig, dense_limit)
                    lam, psi = memo[key]
                    if lam_thresh is not None:
                        m = max(1, int(np.sum(lam < lam_thresh)))
                        lam, psi = lam[:m], psi[:, :m]
                    chi = np.repeat(a.chi(H), 2)[keep]
                    phi = chi[:, None] * psi
                    fr = pos[gd[keep]]
                    for j in range(phi.shape[1]):
                        nz = phi[:, j] != 0.0
                        rows.append(fr[nz])
                        cols.append(np.full(int(nz.sum()), t))
                        vals.append(phi[nz, j])
                        t += 1
                    self.aggs.append(a)
                    self.eigvals.append(lam)
                    interior = ~np.repeat(a.artificial, 2)
                    patch_dofs.append(pos[gd[keep & interior]])
            self.Nt = t
            self.RcT = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                                     shape=(n_free, t)).tocsr()
        self.Kc = np.asarray((self.RcT.T @ (self.K @ self.RcT)).todense())
        self.Kc = 0.5 * (self.Kc + self.Kc.T)
        self.Kc_chol = sla.cho_factor(self.Kc, lower=True)
        self.patch_dofs = patch_dofs
        # patch solves grouped by identical matrix: (factor, [n_patch_dofs x patches] indices)
        self.patch_groups = []
        if with_patches:
            Kr = sp.csr_matrix(self.K)
            groups = {}
            for d in patch_dofs:
                Ki = sp.csr_matrix(Kr[d][:, d])
                key = _matrix_key(Ki)
                if key not in groups:
                    groups[key] = (spla.splu(Ki.tocsc()), [])
                groups[key][1].append(d)
            self.patch_groups = [(lu, np.stack(ds, axis=1)) for lu, ds in groups.values()]

    # --- operators on free-DOF vectors ---------------------------------------------------
    def coarse(self, r: np.ndarray) -> np.ndarray:
        """R_c^T K_c^-1 R_c r."""
        return self.RcT @ sla.cho_solve(self.Kc_chol, self.RcT.T @ r)

    def local(self, r: np.ndarray) -> np.ndarray:
        """sum_i R_i^T K_i^-1 R_i r (patches with the same matrix solved as one block of
        right-hand sides)."""
        z = np.zeros_like(r)
        for lu, D in self.patch_groups:
            np.add.at(z, D, lu.solve(r[D]))
        return z

    def apply(self, r: np.ndarray) -> np.ndarray:
        return self.coarse(r) + self.local(r)


def _matrix_key(A: sp.csr_matrix):
    A.sort_indices()
    return (A.shape, A.indptr.tobytes(), A.indices.tobytes(), A.data.tobytes())


def pcg(K: sp.spmatrix, f: np.ndarray, Minv, tol: float = 1e-8, maxit: int = 1000, x0=None):
    """Standard preconditioned CG; stops when the TRUE relative residual ||f - K x||/||f||
    is at most tol.  Returns (x, iterations, true relative residual)."""
    x = np.zeros_like(f) if x0 is None else x0.copy()
    r = f - K @ x
    nf = np.linalg.norm(f)
    if nf == 0.0:
        return x, 0, 0.0
    z = Minv(r)
    p = z.copy()
    rz = r @ z
    it = 0
    while it < maxit:
        if np.linalg.norm(r) <= tol * nf:
            rt = f - K @ x
            if np.linalg.norm(rt) <= tol * nf:
                break
            r = rt
            z = Minv(r)
            p = z.copy()
            rz = r @ z
        q = K @ p
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        z = Minv(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
    return x, it, np.linalg.norm(f - K @ x) / nf


def energy_error(K: sp.spmatrix, u: np.ndarray, ua: np.ndarray) -> float:
    """||u - u_a||_K / ||u||_K (the square-rooted energy-norm ratio of Sec. 3.1)."""
    e = u - ua
    return float(np.sqrt((e @ (K @ e)) / (u @ (K @ u))))
