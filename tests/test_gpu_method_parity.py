"""GPU parity of the preconditioner's operators and of the solver's iteration counts at the
workloads' own coarse-cell size (H = 32 and 16, six and four eigenvectors), on designs with
interior agglomerates and periodic microstructure.

The additive two-level preconditioner (Sec. 2.4, 2.4.2) is a fixed linear operator once the
agglomerate types, eigenbases, coarse matrix and patch factors are built, so its parts can be
compared with the oracle's operator by operator:
  patches   sum_i R_i^T K_i^-1 R_i r            1e-9 relative in FP64 (same matrices, block
                                                Cholesky vs sparse LU)
  coarse    R_c^T K_c^-1 R_c r                  1e-6 (both coarse spaces come from eigen-solves
                                                converged to residual 1e-7)
  eigen     lambda of K_w psi = lambda D psi    1e-6 relative
and the flexible CG with it needs the same number of iterations as the oracle's PCG with the
oracle's operator (FCG(1) with a fixed SPD preconditioner reproduces PCG in exact arithmetic):
within 10 % in FP64 and MIXED.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads
from oracle import fem, msfem, pipeline


def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1411_3923_gb300 as m
    return m


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def make_problem(m, wl, precision="fp64", **kw):
    return m.Problem(wl.nelx, wl.nely, wl.fixed, nu=wl.nu, E0=wl.E0, Emin=wl.Emin, penal=wl.penal,
                     H=wl.H, n_eig=wl.n_eig, precision=precision, tol=kw.pop("tol", 1e-8), **kw)


def exact_type_count(wl, Es):
    """Distinct agglomerates under the exact key of Sec. 2.4.1's de-duplication, counted on the
    CPU from raw bytes: the moduli of every realisation over the box (out-of-mesh elements
    marked), the Dirichlet flags of the box nodes, and which box sides lie inside the mesh
    (those are the patch's artificial boundary)."""
    H = wl.H
    ncx, ncy = wl.nelx // H, wl.nely // H
    fixed = np.asarray(wl.fixed, dtype=np.int64)
    mask = fixed[..., 0] | (fixed[..., 1] << 1)
    keys = set()
    for J in range(ncy + 1):
        for I in range(ncx + 1):
            ox, oy = (I - 1) * H, (J - 1) * H
            x0, x1 = max(ox, 0), min(ox + 2 * H, wl.nelx)
            y0, y1 = max(oy, 0), min(oy + 2 * H, wl.nely)
            parts = []
            for E in Es:
                ev = np.full((2 * H, 2 * H), -1.0)
                ev[y0 - oy:y1 - oy, x0 - ox:x1 - ox] = E[y0:y1, x0:x1]
                parts.append(ev.tobytes())
            mv = np.full((2 * H + 1, 2 * H + 1), 7)
            mv[y0 - oy:y1 - oy + 1, x0 - ox:x1 - ox + 1] = mask[y0:y1 + 1, x0:x1 + 1]
            sides = (ox > 0, ox + 2 * H < wl.nelx, oy > 0, oy + 2 * H < wl.nely)
            keys.add((tuple(parts), mv.tobytes(), sides))
    return len(keys)


class _Case:
    """One workload with its GPU problem (built) and the oracle's preconditioner."""

    def __init__(self, m, wl, precision="fp64"):
        self.wl = wl
        self.grid, self.K0, self.oprob, chain = pipeline.build(wl)
        fw = chain.forward(wl.rho)
        self.E = fw["E"]
        self.prob = make_problem(m, wl, precision)
        self.prob.set_design(cuda(wl.rho), wl.rmin, wl.beta, wl.etas, wl.cell)
        self.info = self.prob.build_preconditioner()
        self.tl = msfem.TwoLevel(self.oprob, self.E[0], wl.H, wl.n_eig)

    def free(self, v):
        return self.grid.nodal_from_neutral(np.asarray(v))[self.oprob.free]

    def neutral(self, vf):
        z = np.zeros(self.grid.n_dof)
        z[self.oprob.free] = vf
        return self.grid.nodal_to_neutral(z)


@pytest.fixture(scope="module")
def c2_copy():
    """The 1024x512 bench workload's structure on a 256x128 copy: one 32x32 Bernoulli cell
    tiled periodically, filter radius 3 (periodic), H = 32, six eigenvectors.  Coarse nodes
    I = 2..6 of row J = 2 have agglomerates whose four box sides are all artificial."""
    m = _gpu()
    wl = workloads.make("mbb_c2", 4)
    assert (wl.nelx, wl.nely, wl.H, wl.n_eig) == (256, 128, 32, 6)
    return _Case(m, wl)


def test_type_count_keys_on_artificial_sides(c2_copy):
    c = c2_copy
    n = exact_type_count(c.wl, c.E)
    print("types", c.info["n_types"], "exact key", n)
    assert c.info["n_types"] == n == 25


def test_full_size_bench_workload_types_and_residual_certificate():
    """The 1024x512 workload as the benchmark runs it (MIXED, tol 1e-8): the type count equals
    the exact key's, and the oracle's assembled FP64 K certifies the returned u: the true
    relative residual over the free DOFs is at most the tolerance (plus FP64 round-off of the
    residual itself), and the library's compliance equals f^T u."""
    m = _gpu()
    wl = workloads.make("mbb_c2")
    grid, K0, oprob, chain = pipeline.build(wl)
    E = chain.forward(wl.rho)["E"]
    prob = make_problem(m, wl, "mixed")
    prob.set_design(cuda(wl.rho), wl.rmin, wl.beta, wl.etas, wl.cell)
    info = prob.build_preconditioner()
    n = exact_type_count(wl, E)
    print("1024x512 types", info["n_types"], "exact key", n)
    assert info["n_agglomerates"] == 561 and info["n_types"] == n
    u, infos = prob.solve(cuda(wl.force), -1)
    uf = grid.nodal_from_neutral(u[0].cpu().numpy())[oprob.free]
    ff = grid.nodal_from_neutral(wl.force)[oprob.free]
    rr = np.linalg.norm(ff - oprob.free_matrix(E[0]) @ uf) / np.linalg.norm(ff)
    print("oracle residual", rr, "library", infos[0]["rel_residual"], "iterations", infos[0]["iterations"])
    assert infos[0]["status"] == 0 and rr <= 1.01e-8
    assert abs(rr - infos[0]["rel_residual"]) <= 1e-3 * rr
    assert infos[0]["compliance"] == pytest.approx(float(ff @ uf), rel=1e-12)


def test_patch_operator_at_H32_on_a_periodic_design(c2_copy):
    m = _gpu()
    c = c2_copy
    rng = np.random.default_rng(40)
    for _ in range(2):
        r = rng.standard_normal((c.wl.nely + 1, c.wl.nelx + 1, 2))
        z_ref = c.neutral(c.tl.local(c.free(r)))
        z = c.prob.apply_precond(cuda(r), m.FP64, 2).cpu().numpy()
        err = np.linalg.norm(z - z_ref) / np.linalg.norm(z_ref)
        print("patch operator rel. error", err)
        assert err <= 1e-9


def test_coarse_operator_at_H32_on_a_periodic_design(c2_copy):
    m = _gpu()
    c = c2_copy
    r = np.random.default_rng(41).standard_normal((c.wl.nely + 1, c.wl.nelx + 1, 2))
    z_ref = c.neutral(c.tl.coarse(c.free(r)))
    z = c.prob.apply_precond(cuda(r), m.FP64, 1).cpu().numpy()
    err = np.linalg.norm(z - z_ref) / np.linalg.norm(z_ref)
    print("coarse operator rel. error", err)
    assert err <= 1e-6


def test_whole_operator_at_H32_on_a_periodic_design(c2_copy):
    m = _gpu()
    c = c2_copy
    r = np.random.default_rng(42).standard_normal((c.wl.nely + 1, c.wl.nelx + 1, 2))
    z_ref = c.neutral(c.tl.apply(c.free(r)))
    z = c.prob.apply_precond(cuda(r), m.FP64, 0).cpu().numpy()
    assert np.linalg.norm(z - z_ref) <= 1e-6 * np.linalg.norm(z_ref)
    z32 = c.prob.apply_precond(cuda(r), m.MIXED, 0).cpu().numpy()
    err32 = np.linalg.norm(z32 - z_ref) / np.linalg.norm(z_ref)
    print("FP32 operator rel. error", err32)
    assert err32 <= 1e-3


@pytest.mark.parametrize("IJ", [(0, 0), (1, 1), (2, 1), (3, 2), (4, 2), (8, 4), (7, 3)])
def test_eigenvalues_at_H32_on_a_periodic_design(c2_copy, IJ):
    c = c2_copy
    I, J = IJ
    lam, psi, k = c.prob.get_eigenpairs(I, J, c.wl.n_eig, c.wl.H)
    ia = I + J * (c.tl.ncx + 1)
    lam_ref = c.tl.eigvals[ia]
    assert k == lam_ref.size
    print(IJ, lam, lam_ref)
    assert np.allclose(lam, lam_ref, rtol=1e-6, atol=1e-12 * max(1.0, abs(lam_ref).max()))


def _oracle_iterations(c, tol=1e-8):
    Kf = c.oprob.free_matrix(c.E[0])
    f = c.free(c.wl.force)
    _, it, rr = msfem.pcg(Kf, f, c.tl.apply, tol=tol)
    assert rr <= tol
    return it


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_iteration_count_matches_oracle_pcg_on_the_c2_copy(c2_copy, precision):
    m = _gpu()
    c = c2_copy
    it_ref = _oracle_iterations(c)
    prob = make_problem(m, c.wl, precision, tol=1e-8)
    prob.set_design(cuda(c.wl.rho), c.wl.rmin, c.wl.beta, c.wl.etas, c.wl.cell)
    prob.build_preconditioner()
    _, infos = prob.solve(cuda(c.wl.force), -1)
    it = infos[0]["iterations"]
    print(precision, "GPU iterations", it, "oracle", it_ref)
    assert infos[0]["status"] == 0
    assert abs(it - it_ref) <= max(1, int(np.ceil(0.1 * it_ref)))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_iteration_count_matches_oracle_pcg_on_c1_full_size(precision):
    m = _gpu()
    wl = workloads.make("mbb_c1")
    c = _Case(m, wl, precision)
    it_ref = _oracle_iterations(c)
    assert c.info["n_types"] == exact_type_count(wl, c.E)
    _, infos = c.prob.solve(cuda(wl.force), -1)
    it = infos[0]["iterations"]
    print(precision, "C1 GPU iterations", it, "oracle", it_ref)
    assert infos[0]["status"] == 0
    assert abs(it - it_ref) <= max(1, int(np.ceil(0.1 * it_ref)))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_three_realisation_iteration_counts_match_the_oracle(precision):
    """The robust batch (Sec. 5.3): basis of the dilated realisation, K_c and patches per
    realisation.  On a 192x256 copy of the 26.2M-DOF periodic workload each realisation needs
    the oracle's PCG iteration count (within 10 %) and reaches its compliance."""
    m = _gpu()
    wl = workloads.make("mbb_c5", 16)
    out = pipeline.run(wl, "pcg", tol=1e-8, with_grad=False)
    prob = make_problem(m, wl, precision, tol=1e-8)
    prob.set_design(cuda(wl.rho), wl.rmin, wl.beta, wl.etas, wl.cell)
    prob.build_preconditioner()
    _, infos = prob.solve(cuda(wl.force), -1)
    its = [i["iterations"] for i in infos]
    print(precision, "GPU iterations", its, "oracle", out["iterations"])
    for it, it_ref, inf, c in zip(its, out["iterations"], infos, out["c"]):
        assert inf["status"] == 0
        assert abs(it - it_ref) <= max(1, int(np.ceil(0.1 * it_ref)))
        assert inf["compliance"] == pytest.approx(c, rel=1e-7)
