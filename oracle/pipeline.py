"""Oracle, part 4: the whole hot path on one workload (paper Sec. 2.2, 2.4, 4.2-4.4, 5.3).

TEST INFRASTRUCTURE ONLY.

  design chain (filter -> projection per eta -> SIMP)
  -> state solves K(E_k) u_k = f   (sparse LU, or PCG with the two-level preconditioner
     whose coarse basis comes from the dilated realisation, i.e. the smallest eta, as
     Sec. 5.3 prescribes, and whose K_c and patch matrices are those of realisation k)
  -> compliances c_k = f^T u_k, robust objective and its gradient w.r.t. the design.
"""
from __future__ import annotations

import numpy as np

from . import design, fem, msfem


def build(wl):
    grid = fem.Grid(wl.nelx, wl.nely)
    K0 = fem.element_stiffness(wl.nu)
    prob = fem.Problem(grid, K0, wl.fixed)
    chain = design.DesignChain(wl.nelx, wl.nely, wl.rmin, wl.beta, wl.etas, wl.cell,
                               wl.E0, wl.Emin, wl.penal)
    return grid, K0, prob, chain


def run(wl, solver: str = "direct", kappa: float = 1.0, tol: float | None = None,
        with_grad: bool = True, precond=None):
    """Returns a dict with the design fields, displacements (neutral layout), compliances,
    robust objective, its design gradient, and PCG iteration counts when solver='pcg'."""
    grid, K0, prob, chain = build(wl)
    fw = chain.forward(wl.rho)
    tol = wl.tol if tol is None else tol
    us, its, res = [], [], []
    precs = None
    if solver == "pcg":
        if precond is not None:   # one operator for every realisation (caller's choice)
            precs = [precond] * len(fw["E"])
        else:
            ref = int(np.argmin(wl.etas))
            basis = msfem.TwoLevel(prob, fw["E"][ref], wl.H, wl.n_eig)
            precs = [basis if k == ref else msfem.TwoLevel(prob, E, wl.H, wl.n_eig, basis=basis)
                     for k, E in enumerate(fw["E"])]
    f_or = grid.nodal_from_neutral(wl.force)
    for k, E in enumerate(fw["E"]):
        if solver == "direct":
            us.append(prob.solve_direct(E, wl.force))
        else:
            Kf = prob.free_matrix(E)
            x, it, rr = msfem.pcg(Kf, f_or[prob.free], precs[k].apply, tol=tol)
            u = np.zeros(grid.n_dof)
            u[prob.free] = x
            us.append(grid.nodal_to_neutral(u))
            its.append(it)
            res.append(rr)
    c = np.array([float(np.sum(wl.force * u)) for u in us])
    fr, w = design.robust_combine(c, kappa)
    out = dict(rho_tilde=fw["rho_tilde"], rho_bar=fw["rho_bar"], E=fw["E"], u=us, c=c,
               f_robust=fr, weights=w, iterations=its, rel_residual=res)
    if with_grad:
        dc = []
        for k, u in enumerate(us):
            en = grid.element_to_neutral(fem.element_energy(grid, K0, grid.nodal_from_neutral(u)))
            dc.append(chain.element_sensitivity(chain.to_mesh(fw["rho_bar"][k]), en))
        out["dc_drho_bar"] = dc
        out["dfdrho"] = chain.backward(wl.rho, dc, w)
    return out
