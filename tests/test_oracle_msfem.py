"""Pins for oracle/msfem.py: the spectral coarse space and two-level PCG (Sec. 2.4, 3.1, 3.2)."""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads
from oracle import design, fem, msfem, pipeline


def setup(nelx=16, nely=8, H=4, kind="voids", Emin=1e-9, seed=0, bc="mbb"):
    wl = workloads.small(nelx, nely, seed=seed, kind=kind, H=H, Emin=Emin, bc=bc)
    grid, K0, prob, chain = pipeline.build(wl)
    E = chain.forward(wl.rho)["E"][0]
    return wl, grid, K0, prob, E


def test_partition_of_unity():
    """sum_i chi_i = 1 at every node and |grad chi_i| <= 1/H (Sec. 2.4)."""
    H, nelx, nely = 4, 12, 8
    s = np.zeros((nelx + 1, nely + 1))
    for J in range(nely // H + 1):
        for I in range(nelx // H + 1):
            a = msfem.Agglomerate(I, J, H, nelx, nely)
            chi = a.chi(H)
            s[a.node_i, a.node_j] += chi
            assert np.all(chi[a.artificial] == 0.0)
            c = chi.reshape(a.nx + 1, a.ny + 1)
            assert np.abs(np.diff(c, axis=0)).max() <= 1.0 / H + 1e-15
            assert np.abs(np.diff(c, axis=1)).max() <= 1.0 / H + 1e-15
    assert np.allclose(s, 1.0, atol=1e-15)


def test_floating_agglomerate_has_three_rigid_modes():
    """An interior agglomerate has no Dirichlet DOFs, so its three rigid motions are
    eigenvectors with eigenvalue 0 (Sec. 2.4.1)."""
    wl, grid, K0, prob, E = setup(kind="solid")
    a = msfem.Agglomerate(2, 1, 4, 16, 8)
    Kw = a.local_stiffness(E, K0)
    lam, psi = msfem.local_eigenpairs(Kw, 5)
    assert np.all(np.abs(lam[:3]) < 1e-12) and lam[3] > 1e-4
    i, j = a.node_i.astype(float), a.node_j.astype(float)
    rot = np.zeros(2 * i.size); rot[0::2] = -j; rot[1::2] = i
    D = Kw.diagonal()
    proj = psi[:, :3] @ (psi[:, :3].T @ (D * rot))
    assert np.linalg.norm(proj - rot) < 1e-10 * np.linalg.norm(rot)


@pytest.mark.parametrize("I,J", [(0, 0), (2, 1), (4, 2)])
def test_eigenpairs_residual_orthonormality_and_brute_force(I, J):
    wl, grid, K0, prob, E = setup(kind="voids", seed=2)
    a = msfem.Agglomerate(I, J, 4, 16, 8)
    keep = ~prob.fixed[a.global_dofs(grid)]
    Kw = a.local_stiffness(E, K0)[keep][:, keep]
    D = Kw.diagonal()
    lam, psi = msfem.local_eigenpairs(Kw, 6, dense_limit=0)     # shift-invert Lanczos
    R = Kw @ psi - (D[:, None] * psi) * lam[None, :]
    assert np.abs(R).max() < 1e-9 * abs(Kw).max()
    assert np.allclose(psi.T @ (D[:, None] * psi), np.eye(6), atol=1e-9)
    ref = sla.eigh(Kw.toarray(), np.diag(D), eigvals_only=True)[:6]   # dense brute force
    assert np.allclose(lam, ref, rtol=1e-8, atol=1e-12)


def test_pcg_converges_to_direct_solution():
    wl, grid, K0, prob, E = setup(kind="voids", seed=3)
    tl = msfem.TwoLevel(prob, E, 4, 4)
    Kf = prob.free_matrix(E)
    f = grid.nodal_from_neutral(wl.force)[prob.free]
    # cond(K) is ~1e10 at this contrast, so an FP64 true residual of 1e-10 is near the floor
    x, it, rr = msfem.pcg(Kf, f, tl.apply, tol=1e-10)
    xd = sla.solve(Kf.toarray(), f, assume_a="pos")
    assert rr <= 1e-10
    assert msfem.energy_error(Kf, xd, x) < 1e-8


def test_preconditioner_symmetric_positive_definite():
    wl, grid, K0, prob, E = setup(kind="voids", seed=4)
    tl = msfem.TwoLevel(prob, E, 4, 3)
    rng = np.random.default_rng(0)
    n = prob.free.size
    for _ in range(5):
        x, y = rng.standard_normal(n), rng.standard_normal(n)
        My, Mx = tl.apply(y), tl.apply(x)
        # K_c has condition ~1e10 here, so FP64 round-off leaves ~1e-10 relative asymmetry
        assert abs(x @ My - y @ Mx) <= 1e-8 * np.linalg.norm(x) * np.linalg.norm(My)
        assert x @ Mx > 0.0


def test_coarse_only_energy_error_decreases_with_basis_size():
    """Nested coarse spaces (first k eigenvectors of every agglomerate) give a non-increasing
    Galerkin energy error (Sec. 3.1 reports the same trend against lambda_Omega)."""
    wl, grid, K0, prob, E = setup(kind="voids", seed=5)
    Kf = prob.free_matrix(E)
    f = grid.nodal_from_neutral(wl.force)[prob.free]
    u = sla.solve(Kf.toarray(), f, assume_a="pos")
    errs = []
    # cuts at 3 and above: the rigid-mode eigenvalue 0 is triple on floating agglomerates,
    # and a cut inside a degenerate cluster does not give nested spaces
    for k in (3, 4, 6, 8, 12):
        tl = msfem.TwoLevel(prob, E, 4, k, with_patches=False)
        errs.append(msfem.energy_error(Kf, u, tl.coarse(f)))
    assert all(e2 <= e1 * (1 + 1e-9) for e1, e2 in zip(errs, errs[1:]))
    assert errs[-1] < 0.5 * errs[0]


def test_coarse_only_solve_exact_when_basis_is_complete():
    """With every local eigenvector kept, span{chi_i psi_j} is the whole fine space (the
    chi_i sum to one), so the MsFEM coarse-only solve returns the exact solution."""
    wl, grid, K0, prob, E = setup(nelx=8, nely=4, H=4, kind="voids", seed=6, Emin=1e-3)
    Kf = prob.free_matrix(E)
    f = grid.nodal_from_neutral(wl.force)[prob.free]
    u = sla.solve(Kf.toarray(), f, assume_a="pos")
    # Kc is singular here (the spanning set is redundant): use a least-squares coarse solve
    g = grid
    n_free = prob.free.size
    pos = -np.ones(g.n_dof, dtype=np.int64); pos[prob.free] = np.arange(n_free)
    cols = []
    for J in range(2):
        for I in range(3):
            a = msfem.Agglomerate(I, J, 4, 8, 4)
            gd = a.global_dofs(g); keep = ~prob.fixed[gd]
            Kw = a.local_stiffness(E, K0)[keep][:, keep]
            lam, psi = msfem.local_eigenpairs(Kw, 10 ** 6)
            phi = np.repeat(a.chi(4), 2)[keep][:, None] * psi
            block = np.zeros((n_free, phi.shape[1])); block[pos[gd[keep]]] = phi
            cols.append(block)
    RcT = np.hstack(cols)
    Kc = RcT.T @ Kf.toarray() @ RcT
    uc = np.linalg.lstsq(Kc, RcT.T @ f, rcond=1e-13)[0]
    assert np.linalg.norm(RcT @ uc - u) < 1e-8 * np.linalg.norm(u)


def test_iterations_contrast_independent():
    """Sec. 3.1: for Emin <= 1e-6 the iteration count does not grow with the contrast."""
    its = []
    for Emin in (1e-6, 1e-9, 1e-12):
        wl, grid, K0, prob, E = setup(nelx=24, nely=8, H=4, kind="voids", seed=7, Emin=Emin)
        tl = msfem.TwoLevel(prob, E, 4, 6)
        Kf = prob.free_matrix(E)
        f = grid.nodal_from_neutral(wl.force)[prob.free]
        its.append(msfem.pcg(Kf, f, tl.apply, tol=1e-8)[1])
    assert max(its) - min(its) <= 2, its


def test_config_sizes():
    """Mesh sizes of the workloads: DOF counts 2 (nelx+1)(nely+1) and coarse node counts."""
    wl = workloads.make("mbb_c1")
    assert wl.n_dof == 25090 and (wl.nelx // wl.H + 1) * (wl.nely // wl.H + 1) == 65
    wl = workloads.make("mbb_c2")
    assert wl.n_dof == 1051650 and (wl.nelx // wl.H + 1) * (wl.nely // wl.H + 1) == 561


def test_grouped_patch_solves_equal_one_solve_per_patch():
    """local() solves the patches that share a matrix as one block of right-hand sides; the
    sum must equal the plain definition sum_i R_i^T K_i^-1 R_i r with one sparse LU per patch
    (periodic design: most patches share their matrix)."""
    import scipy.sparse.linalg as spla
    wl = workloads.small(48, 24, seed=5, kind="voids", cell=(8, 8), H=8, n_eig=4)
    grid, K0, prob, chain = pipeline.build(wl)
    E = chain.forward(wl.rho)["E"][0]
    tl = msfem.TwoLevel(prob, E, 8, 4)
    assert len(tl.patch_groups) < len(tl.patch_dofs)
    r = np.random.default_rng(3).standard_normal(prob.free.size)
    z = np.zeros_like(r)
    K = prob.free_matrix(E).tocsr()
    for d in tl.patch_dofs:
        z[d] += spla.splu(K[d][:, d].tocsc()).solve(r[d])
    assert np.linalg.norm(tl.local(r) - z) <= 1e-12 * np.linalg.norm(z)


def test_robust_pcg_with_the_dilated_basis_converges_on_every_realisation():
    """Sec. 5.3: the coarse basis of the dilated design (smallest eta) serves all three
    realisations, while K_c and the patch matrices are each realisation's own.  On a 192x256
    copy of the 26.2M-DOF periodic workload (H = 32, six eigenvectors, contrast 1e9) PCG with
    that preconditioner reaches the sparse-LU solution of every realisation: energy-norm error
    1e-8 and compliance 1e-10 at true residual 1e-10, in a number of iterations close to the
    single-design count (the eroded realisation included)."""
    wl = workloads.make("mbb_c5", 16)
    grid, K0, prob, chain = pipeline.build(wl)
    out = pipeline.run(wl, "pcg", tol=1e-10, with_grad=False)
    ref = pipeline.run(wl, "direct", with_grad=False)
    assert max(out["iterations"]) <= 2 * min(out["iterations"]) <= 100, out["iterations"]
    for k in range(3):
        Kf = prob.free_matrix(ref["E"][k])
        e = msfem.energy_error(Kf, grid.nodal_from_neutral(ref["u"][k])[prob.free],
                               grid.nodal_from_neutral(out["u"][k])[prob.free])
        assert out["rel_residual"][k] <= 1e-10 and e <= 1e-8
        assert out["c"][k] == pytest.approx(ref["c"][k], rel=1e-10)


def test_shared_basis_keeps_the_basis_and_rebuilds_the_operators():
    wl = workloads.small(32, 16, seed=6, kind="voids", H=8, n_eig=4, etas=(0.3, 0.7),
                         rmin=2.0, beta=8.0)
    grid, K0, prob, chain = pipeline.build(wl)
    E = chain.forward(wl.rho)["E"]
    b = msfem.TwoLevel(prob, E[0], 8, 4)
    t = msfem.TwoLevel(prob, E[1], 8, 4, basis=b)
    assert t.RcT is b.RcT and t.Nt == b.Nt
    Kf = prob.free_matrix(E[1])
    assert np.allclose(t.Kc, (b.RcT.T @ (Kf @ b.RcT)).toarray(), rtol=1e-12, atol=1e-14 * abs(t.Kc).max())
    assert not np.allclose(t.Kc, b.Kc)
