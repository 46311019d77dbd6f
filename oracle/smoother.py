"""Oracle, part 4: the paper's own two-level preconditioner (Sec. 2.4.2): the spectral coarse
solve of part 3 with one symmetric Gauss-Seidel sweep before it and one after it, applied
multiplicatively.

TEST INFRASTRUCTURE ONLY -- plain FP64 NumPy/SciPy.

Definitions, on the free DOFs of K with K = D + L + U:
  - Forward Gauss-Seidel sweep for K x = r, starting from x:   x <- x + (D + L)^-1 (r - K x).
  - Backward sweep:                                            x <- x + (D + U)^-1 (r - K x).
  - Symmetric sweep (SGS): the forward sweep, then the backward sweep.

D, L and U depend on the order in which the unknowns are visited and on their blocking:
  - "lex": point Gauss-Seidel in the oracle's own DOF numbering. The paper's (Matlab)
    smoother is read this way.
  - "colour": node blocks. The two free DOFs of a node are solved together (D = the 2x2 node
    blocks), and nodes are visited colour by colour, colour = (i mod 2) + 2 (j mod 2). Two
    nodes of one colour share no element, so within a colour the visiting order does not
    change the result. This is the smoother the GPU runs.

Multiplicative two-level preconditioner (Sec. 2.4.2: coarse solve, one SGS sweep before and
one after):
    x = SGS(0; r);   x <- x + R_c^T K_c^-1 R_c (r - K x);   x <- SGS(x; r)
With a symmetric smoother before and after, the operator is symmetric positive definite
(error propagation (I - S K)(I - C K)(I - S K), S the symmetric sweep), so PCG applies to it,
as the paper remarks for its preconditioner.

The paper's outer method is GMRES (Sec. 2.4.2): ``gmres`` is right-preconditioned restarted
GMRES(m) written from its textbook definition (Arnoldi with modified Gram-Schmidt, Givens
rotations), stopped on the true residual.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem


class SymmetricGaussSeidel:
    """One symmetric Gauss-Seidel sweep on the free-DOF system K x = r."""

    def __init__(self, prob: fem.Problem, Kf: sp.spmatrix, order: str = "colour"):
        if order not in ("lex", "colour"):
            raise ValueError(order)
        self.K = sp.csr_matrix(Kf)
        self.order = order
        if order == "lex":
            self.lower = sp.tril(self.K, format="csr")
            self.upper = sp.triu(self.K, format="csr")
            return
        # node blocks by colour, free-DOF positions
        g = prob.grid
        n_free = prob.free.size
        pos = -np.ones(g.n_dof, dtype=np.int64)
        pos[prob.free] = np.arange(n_free)
        self.colours = []
        for c in range(4):
            ci, cj = c & 1, c >> 1
            nodes = [g.node(i, j) for j in range(cj, g.nely + 1, 2)
                     for i in range(ci, g.nelx + 1, 2)]
            blocks = []
            for n in nodes:
                d = [p for p in (pos[2 * n], pos[2 * n + 1]) if p >= 0]
                if d:
                    blocks.append(np.array(d, dtype=np.int64))
            self.colours.append(blocks)
        Kd = self.K.toarray() if n_free <= 4000 else None
        self._blk = []
        for blocks in self.colours:
            inv = []
            for d in blocks:
                B = (Kd[np.ix_(d, d)] if Kd is not None else self.K[d][:, d].toarray())
                inv.append(np.linalg.inv(B))
            self._blk.append(inv)

    def _colour_pass(self, x: np.ndarray, r: np.ndarray, c: int) -> None:
        res = r - self.K @ x
        for d, Binv in zip(self.colours[c], self._blk[c]):
            x[d] += Binv @ res[d]

    def forward(self, x: np.ndarray, r: np.ndarray) -> np.ndarray:
        x = x.copy()
        if self.order == "lex":
            x += spla.spsolve_triangular(self.lower, r - self.K @ x, lower=True)
        else:
            for c in range(4):
                self._colour_pass(x, r, c)
        return x

    def backward(self, x: np.ndarray, r: np.ndarray) -> np.ndarray:
        x = x.copy()
        if self.order == "lex":
            x += spla.spsolve_triangular(self.upper, r - self.K @ x, lower=False)
        else:
            for c in (3, 2, 1, 0):
                self._colour_pass(x, r, c)
        return x

    def sweep(self, x: np.ndarray, r: np.ndarray) -> np.ndarray:
        """SGS(x; r): forward then backward."""
        return self.backward(self.forward(x, r), r)


class MultiplicativeTwoLevel:
    """x = SGS(0; r); x += R_c^T K_c^-1 R_c (r - K x); x = SGS(x; r).  ``coarse`` is any
    callable r -> R_c^T K_c^-1 R_c r on free-DOF vectors (part 3's TwoLevel.coarse)."""

    def __init__(self, K: sp.spmatrix, smoother: SymmetricGaussSeidel, coarse):
        self.K, self.S, self.coarse = sp.csr_matrix(K), smoother, coarse

    def apply(self, r: np.ndarray) -> np.ndarray:
        x = self.S.sweep(np.zeros_like(r), r)
        x = x + self.coarse(r - self.K @ x)
        return self.S.sweep(x, r)


def gmres(K: sp.spmatrix, f: np.ndarray, Minv, tol: float = 1e-8, restart: int = 50,
          maxit: int = 1000, x0=None, history: list | None = None):
    """Right-preconditioned restarted GMRES(m), the paper's outer method (Sec. 2.4.2):
    Arnoldi on K M^-1 with modified Gram-Schmidt, Givens rotations for the small least-squares
    problem, x = x0 + M^-1 V y.  Stops when the TRUE relative residual ||f - K x|| / ||f|| is
    at most tol (checked at every restart and whenever the recurrence estimate reaches tol).
    ``history`` (optional) receives the recurrence residual norm after every iteration.
    Returns (x, iterations, true relative residual)."""
    x = np.zeros_like(f) if x0 is None else x0.copy()
    nf = np.linalg.norm(f)
    if nf == 0.0:
        return x, 0, 0.0
    it = 0
    while it < maxit:
        r = f - K @ x
        beta = np.linalg.norm(r)
        if beta <= tol * nf:
            break
        m = min(restart, maxit - it)
        V = np.zeros((m + 1, f.size))
        Z = np.zeros((m, f.size))
        Hm = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        for j in range(m):
            Z[j] = Minv(V[j])
            w = K @ Z[j]
            for i in range(j + 1):                     # modified Gram-Schmidt
                Hm[i, j] = w @ V[i]
                w = w - Hm[i, j] * V[i]
            Hm[j + 1, j] = np.linalg.norm(w)
            if Hm[j + 1, j] > 0.0:
                V[j + 1] = w / Hm[j + 1, j]
            for i in range(j):                         # earlier rotations on the new column
                a, b = Hm[i, j], Hm[i + 1, j]
                Hm[i, j], Hm[i + 1, j] = cs[i] * a + sn[i] * b, -sn[i] * a + cs[i] * b
            d = np.hypot(Hm[j, j], Hm[j + 1, j])        # new rotation zeroes H[j+1, j]
            cs[j], sn[j] = Hm[j, j] / d, Hm[j + 1, j] / d
            Hm[j, j], Hm[j + 1, j] = d, 0.0
            g[j], g[j + 1] = cs[j] * g[j], -sn[j] * g[j]
            it += 1
            j_done = j + 1
            if history is not None:
                history.append(abs(g[j + 1]))
            if abs(g[j + 1]) <= tol * nf or Hm[j, j] == 0.0:
                break
        y = np.linalg.solve(np.triu(Hm[:j_done, :j_done]), g[:j_done])
        x = x + Z[:j_done].T @ y
    return x, it, np.linalg.norm(f - K @ x) / nf
