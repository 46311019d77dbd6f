"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle, element by element.

Tolerances (derived from the arithmetic):
  design chain (FP64)      1e-12 relative: a few roundings of tanh/pow/filter sums
  FP64 matvec              1e-12 of sum_e |E_e K0| |u_e| per DOF (summation order only)
  FP32 matvec              2e-6 of the same scale (FP32 unit round-off x ~30 terms)
  patch solves (FP64)      1e-9 relative (block Cholesky vs sparse LU of the same matrix)
  solve u (FP64 and MIXED) energy-norm error <= 1e-8 at true residual 1e-10, compliance 1e-10
  design gradient          2-norm relative 1e-7 against the oracle's chain on the same u
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads
from oracle import design, fem, msfem, pipeline, smoother


def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1411_3923_gb300 as m
    return m


def make_problem(m, wl, precision="fp64", **kw):
    return m.Problem(wl.nelx, wl.nely, wl.fixed, nu=wl.nu, E0=wl.E0, Emin=wl.Emin, penal=wl.penal,
                     H=wl.H, n_eig=wl.n_eig, precision=precision, tol=kw.pop("tol", 1e-10), **kw)


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def assert_energy(Kf, u_ref, u, bound=1e-8):
    """u against the direct solution in the energy norm ||e||_K / ||u||_K (Sec. 3.1)."""
    err = msfem.energy_error(Kf, u_ref, u)
    print(f"energy-norm error {err:.3e}")
    assert err <= bound


@pytest.mark.parametrize("cell", [None, (8, 4)])
@pytest.mark.parametrize("size", [(24, 12), (40, 16)])
def test_design_chain(cell, size):
    m = _gpu()
    wl = workloads.small(*size, seed=11, kind="random", cell=cell, etas=(0.3, 0.5, 0.7),
                         rmin=2.3, beta=8.0, H=4)
    prob = make_problem(m, wl)
    prob.set_design(cuda(wl.rho), wl.rmin, wl.beta, wl.etas, wl.cell)
    _, _, _, chain = pipeline.build(wl)
    ref = chain.forward(wl.rho)
    rt = prob.get_field(m.FIELD_RHO_TILDE).cpu().numpy()
    assert np.allclose(rt, ref["rho_tilde"], rtol=1e-12, atol=1e-14)
    for k in range(3):
        rb = prob.get_field(m.FIELD_RHO_BAR, k).cpu().numpy()
        assert np.allclose(rb, ref["rho_bar"][k], rtol=1e-12, atol=1e-14)
        E = prob.get_field(m.FIELD_YOUNG, k).cpu().numpy()
        assert np.allclose(E, ref["E"][k], rtol=1e-12, atol=1e-20)


@pytest.mark.parametrize("size", [(7 * 4, 3 * 4), (33 * 4, 5 * 4), (64, 64)])
def test_matvec_fp64_and_fp32(size):
    m = _gpu()
    wl = workloads.small(*size, seed=3, kind="random", H=4)
    prob = make_problem(m, wl)
    prob.set_design(cuda(wl.rho), wl.rmin, wl.beta, wl.etas, wl.cell)
    E = prob.get_field(m.FIELD_YOUNG, 0).cpu().numpy()
    grid, K0, oprob, _ = pipeline.build(wl)
    rng = np.random.default_rng(5)
    u = rng.standard_normal((wl.nely + 1, wl.nelx + 1, 2))
    y_ref = oprob.apply(E, u)
    # scale: sum_e |E_e K0| |u_e| per DOF
    ue = np.abs(grid.nodal_from_neutral(u)); ue[oprob.fixed] = 0
    scale = grid.nodal_to_neutral(fem.matvec_unconstrained(grid, grid.element_from_neutral(E), np.abs(K0), ue))
    y64 = prob.apply_K(cuda(u), 0, m.FP64).cpu().numpy()
    assert np.all(np.abs(y64 - y_ref) <= 1e-12 * scale + 1e-300)
    y32 = prob.apply_K(cuda(u), 0, m.MIXED).cpu().numpy()
    assert np.all(np.abs(y32 - y_ref) <= 2e-6 * scale + 1e-30)


def test_patch_solves_match_sparse_lu():
    m = _gpu()
    wl = workloads.small(32, 16, seed=4, kind="voids", H=8, n_eig=4)
    prob = make_problem(m, wl)
    prob.set_design(cuda(wl.rho), wl.rmin, wl.beta, wl.etas, wl.cell)
    prob.build_preconditioner()
    grid, K0, oprob, chain = pipeline.build(wl)
    E = chain.forward(wl.rho)["E"][0]
    tl = msfem.TwoLevel(oprob, E, wl.H, wl.n_eig)
    rng = np.random.default_rng(1)
    r = rng.standard_normal((wl.nely + 1, wl.nelx + 1, 2))
    rf = grid.nodal_from_neutral(r)[oprob.free]
    z_ref = np.zeros(grid.n_dof)
    z_ref[oprob.free] = tl.local(rf)
    z_ref = grid.nodal_to_neutral(z_ref)
    z = prob.apply_precond(cuda(r), m.FP64, 2).cpu().numpy()
    assert np.linalg.norm(z - z_ref) <= 1e-9 * np.linalg.norm(z_ref)
    z32 = prob.apply_precond(cuda(r), m.MIXED, 2).cpu().numpy()
    # FP32 factors of a contrast-1e9 matrix: compare in the energy of the patch matrices
    assert np.linalg.norm(z32 - z_ref) <= 1e-2 * np.linalg.norm(z_ref)


@pytest.mark.parametrize("size,H,etas", [
    ((128, 64), 32, (0.5,)),             # nb = 130: 17 K-steps, N = 144, partial groups
    ((256, 128), 16, (0.5,)),            # nb = 66: 9 K-steps
    ((192, 96), 8, (0.3, 0.5, 0.7)),     # nb = 34: 5 K-steps, three realisations
    ((1024, 768), 32, (0.3, 0.5, 0.7)),  # 825 patches per realisation: several full groups
])
def test_tensor_core_patch_solves(size, H, etas):
    """The FP32 patch solves on the tensor cores (up to 128 patches of one type as the MMA's
    rows, the two-sided elimination of Sec. 3.2) against the FP64 patch solves of the same
    factors, next to the FP32 CUDA-core solves; both must stay far below the preconditioner's
    own approximation error.  Every line product sums 3 KS tensor-core MMAs (KS = ceil(nb / 8)
    K-steps, TF32 high and low parts of both operands) in one FP32 accumulator, each of which
    may drop up to one FP32 unit of the running sum, so the bound is 3 KS 2^-23 on top of four
    times the CUDA-core FP32 error."""
    m = _gpu()
    wl = workloads.small(*size, seed=21, kind="voids", H=H, n_eig=4, etas=etas, Emin=1e-3)
    rng = np.random.default_rng(5)
    r = cuda(rng.standard_normal((wl.nely + 1, wl.nelx + 1, 2)))
    err = {}
    for tc in ("1", "0"):
        prob = make_problem(m, wl, precision="mixed",
                            patch_kernel="tensor_cores" if tc == "1" else "cuda_cores")
        prob.set_design(cuda(wl.rho), wl.rmin, wl.beta, wl.etas, wl.cell)
        prob.build_preconditioner()
        z64 = prob.apply_precond(r, m.FP64, 2)
        z32 = prob.apply_precond(r, m.MIXED, 2)
        assert torch.isfinite(z32).all()
        err[tc] = (torch.linalg.norm(z32 - z64) / torch.linalg.norm(z64)).item()
        del prob
    print(f"tensor-core patch solves {size} H={H}: rel. error {err['1']:.3e} "
          f"(CUDA-core FP32 {err['0']:.3e})")
    assert err["1"] < 1e-5, err
    ks = (2 * (2 * H + 1) + 7) // 8
    assert err["1"] <= 3 * ks * 2.0 ** -23 + 4.0 * err["0"], err


def test_tensor_core_patch_solves_reject_other_line_sizes():
    """The tensor-core kernel is compiled for H = 8, 16 and 32; forcing it with another H is an
    invalid argument, while the automatic choice falls back to the CUDA cores."""
    m = _gpu()
    wl = workloads.small(40, 24, seed=21, kind="voids", H=4, n_eig=4)
    prob = make_problem(m, wl, precision="mixed", patch_kernel="tensor_cores")
    prob.set_design(cuda(wl.rho), wl.rmin, wl.beta, wl.etas, wl.cell)
    with pytest.raises(m.MstopoError, match="H = 8, 16 or 32"):
        prob.build_preconditioner()
    prob = make_problem(m, wl, precision="mixed", patch_kernel="auto")
    prob.set_design(cuda(wl.rho), wl.rmin, wl.beta, wl.etas, wl.cell)
    prob.build_preconditioner()


def test_eigenpairs_satisfy_generalised_eigenproblem():
    """Every kept pair satisfies K_w psi = lambda diag(K_w) psi (Sec. 2.4, 3.2) with the
    oracle's assembled agglomerate matrix, and the eigenvalues match the oracle's."""
    m = _gpu()
    wl = workloads.small(32, 16, seed=8, kind="random", H=8, n_eig=4)
    prob = make_problem(m, wl)
    prob.set_design(cuda(wl.rho), wl.rmin, wl.beta, wl.etas, wl.cell)
    prob.build_preconditioner()
    grid, K0, oprob, chain = pipeline.build(wl)
    E = chain.forward(wl.rho)["E"][0]
    for (I, J) in [(0, 0), (2, 1), (4, 2), (1, 2)]:
        lam, psi, k = prob.get_eigenpairs(I, J, wl.n_eig, wl.H)
        a = msfem.Agglomerate(I, J, wl.H, wl.nelx, wl.nely)
        keep = ~oprob.fixed[a.global_dofs(grid)]
        Kw = a.local_stiffness(E, K0)[keep][:, keep]
        D = Kw.diagonal()
        # gather the GPU vectors on the (clipped) agglomerate nodes, oracle local order
        bx, by = (I - 1) * wl.H, (J - 1) * wl.H
        P = psi[a.node_j - by, a.node_i - bx]            # [nodes, 2, k]
        P = P.reshape(-1, k)[keep]
        R = Kw @ P - (D[:, None] * P) * lam[None, :]
        assert np.sqrt(np.sum(R * R / D[:, None], axis=0)).max() < 1e-6
        assert np.allclose(P.T @ (D[:, None] * P), np.eye(k), atol=1e-8)
        lam_ref, _ = msfem.local_eigenpairs(Kw, k)
        assert np.allclose(lam, lam_ref, rtol=1e-6, atol=1e-9)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["voids", "random_periodic"])
def test_solve_compliance_and_gradient(precision, case):
    m = _gpu()
    if case == "voids":
        wl = workloads.small(48, 16, seed=6, kind="voids", H=8, n_eig=4, etas=(0.3, 0.5, 0.7),
                             rmin=2.0, beta=8.0)
    else:
        wl = workloads.small(48, 24, seed=7, kind="random", H=8, n_eig=6, cell=(8, 8),
                             etas=(0.5,), rmin=1.5, beta=4.0)
    prob = make_problem(m, wl, precision, tol=1e-10)
    prob.set_design(cuda(wl.rho), wl.rmin, wl.beta, wl.etas, wl.cell)
    prob.build_preconditioner()
    u, infos = prob.solve(cuda(wl.force), -1)
    ref = pipeline.run(wl, "direct")
    grid, K0, oprob, _ = pipeline.build(wl)
    for k, info in enumerate(infos):
        assert info["status"] == 0 and info["rel_residual"] <= 1e-10
        Kf = oprob.free_matrix(ref["E"][k])
        ug = grid.nodal_from_neutral(u[k].cpu().numpy())[oprob.free]
        ur = grid.nodal_from_neutral(ref["u"][k])[oprob.free]
        assert_energy(Kf, ur, ug)
        assert info["compliance"] == pytest.approx(ref["c"][k], rel=1e-10)
    c, fr, g = prob.compliance_and_sensitivity(1.0)
    assert np.allclose(c, ref["c"], rtol=1e-10)
    assert fr == pytest.approx(ref["f_robust"], rel=1e-10)
    g = g.cpu().numpy()
    assert np.linalg.norm(g - ref["dfdrho"]) <= 1e-7 * np.linalg.norm(ref["dfdrho"]) + 1e-12


def test_host_pointer_solve_matches_device_solve():
    m = _gpu()
    wl = workloads.small(32, 16, seed=9, kind="voids", H=8, n_eig=4)
    prob = make_problem(m, wl, "mixed", tol=1e-8)
    prob.set_design(cuda(wl.rho), wl.rmin, wl.beta, wl.etas, wl.cell)
    prob.build_preconditioner()
    u_d, _ = prob.solve(cuda(wl.force), 0)
    u_h, _ = prob.solve_host(wl.force, 0)
    assert np.array_equal(u_d.cpu().numpy(), u_h)   # same kernels, deterministic reductions


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_mbb_c1_full_size_against_direct_solve(precision):
    """The 192x64 MBB workload (25,090 DOFs) against sparse LU: u to energy-norm 1e-8 and the
    compliance to 1e-10 (solved to true residual 1e-10)."""
    m = _gpu()
    wl = workloads.make("mbb_c1")
    prob = make_problem(m, wl, precision, tol=1e-10)
    prob.set_design(cuda(wl.rho), wl.rmin, wl.beta, wl.etas, wl.cell)
    info = prob.build_preconditioner()
    assert info["n_agglomerates"] == 65 and info["n_coarse"] == 260
    u, infos = prob.solve(cuda(wl.force), -1)
    ref = pipeline.run(wl, "direct", with_grad=False)
    assert infos[0]["status"] == 0 and infos[0]["rel_residual"] <= 1e-10
    grid, K0, oprob, _ = pipeline.build(wl)
    Kf = oprob.free_matrix(ref["E"][0])
    assert_energy(Kf, grid.nodal_from_neutral(ref["u"][0])[oprob.free],
                  grid.nodal_from_neutral(u[0].cpu().numpy())[oprob.free])
    print("compliance rel. error", abs(infos[0]["compliance"] / ref["c"][0] - 1))
    assert infos[0]["compliance"] == pytest.approx(ref["c"][0], rel=1e-10)


@pytest.mark.parametrize("n_eig", [4, 12])
def test_coarse_solve_matches_oracle(n_eig):
    """The coarse correction R_c^T K_c^-1 R_c r (Sec. 2.4) through the explicit inverse and
    through the block sweeps over lines of coarse nodes: 13 nodes x n_eig = 52 or 156
    unknowns per line (ragged 32-column Cholesky panels), 25 lines.  Against the oracle the
    bound is set by the eigen-solve (residual 1e-7: the coarse spaces differ at that level);
    the two GPU solvers share the coarse space and agree to FP64 round-off."""
    m = _gpu()
    wl = workloads.small(96, 48, seed=12, kind="random", H=4, n_eig=n_eig, Emin=1e-3)
    grid, K0, oprob, chain = pipeline.build(wl)
    E = chain.forward(wl.rho)["E"][0]
    tl = msfem.TwoLevel(oprob, E, wl.H, n_eig, with_patches=False)
    rng = np.random.default_rng(2)
    r = rng.standard_normal((wl.nely + 1, wl.nelx + 1, 2))
    rf = grid.nodal_from_neutral(r)[oprob.free]
    z_ref = np.zeros(grid.n_dof)
    z_ref[oprob.free] = tl.coarse(rf)
    z_ref = grid.nodal_to_neutral(z_ref)
    z = {}
    for coarse in ("dense", "blocktri"):
        prob = make_problem(m, wl, coarse_solver=coarse)
        prob.set_design(cuda(wl.rho), wl.rmin, wl.beta, wl.etas, wl.cell)
        info = prob.build_preconditioner()
        assert info["coarse_solver"] == {"dense": 1, "blocktri": 2}[coarse]
        assert info["coarse_line"] == 13 * n_eig and info["coarse_lines"] == 25
        z[coarse] = prob.apply_precond(cuda(r), m.FP64, 1).cpu().numpy()
        assert np.linalg.norm(z[coarse] - z_ref) <= 1e-6 * np.linalg.norm(z_ref)
    assert np.linalg.norm(z["blocktri"] - z["dense"]) <= 1e-11 * np.linalg.norm(z["dense"])


def test_blocktri_and_dense_coarse_agree_at_full_contrast():
    """Both coarse solvers factor the same assembled K_c (contrast 1e9): the corrections agree
    to the conditioning of K_c times FP64 round-off."""
    m = _gpu()
    wl = workloads.small(128, 64, seed=14, kind="voids", H=8, n_eig=6)
    z = {}
    for coarse in ("dense", "blocktri"):
        prob = make_problem(m, wl, coarse_solver=coarse)
        prob.set_design(cuda(wl.rho), wl.rmin, wl.beta, wl.etas, wl.cell)
        prob.build_preconditioner()
        r = torch.from_numpy(np.random.default_rng(3).standard_normal(prob.n_dof)).cuda()
        z[coarse] = prob.apply_precond(r, m.FP64, 1).cpu().numpy()
    assert np.linalg.norm(z["blocktri"] - z["dense"]) <= 1e-6 * np.linalg.norm(z["dense"])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solve_with_blocktri_coarse_solver(precision):
    """Three realisations (one cooperative sweep launch carries all three right-hand sides)
    solved with the block-tridiagonal coarse solver against sparse LU."""
    m = _gpu()
    wl = workloads.small(96, 48, seed=13, kind="voids", H=8, n_eig=6, etas=(0.3, 0.5, 0.7),
                         rmin=2.0, beta=8.0)
    prob = make_problem(m, wl, precision, tol=1e-10, coarse_solver="blocktri")
    prob.set_design(cuda(wl.rho), wl.rmin, wl.beta, wl.etas, wl.cell)
    info = prob.build_preconditioner()
    assert info["coarse_solver"] == 2 and info["coarse_line"] == 42
    u, infos = prob.solve(cuda(wl.force), -1)
    ref = pipeline.run(wl, "direct", with_grad=False)
    grid, K0, oprob, _ = pipeline.build(wl)
    for k, inf in enumerate(infos):
        assert inf["status"] == 0 and inf["rel_residual"] <= 1e-10
        Kf = oprob.free_matrix(ref["E"][k])
        ug = grid.nodal_from_neutral(u[k].cpu().numpy())[oprob.free]
        ur = grid.nodal_from_neutral(ref["u"][k])[oprob.free]
        assert_energy(Kf, ur, ug)
        assert inf["compliance"] == pytest.approx(ref["c"][k], rel=1e-10)


@pytest.mark.parametrize("H", [8, 32])
def test_mixed_solve_with_tensor_core_patches(H):
    """The mixed flexible CG with its FP32 patch solves forced onto the tensor cores (H = 32:
    130-DOF lines, N = 144 per MMA) converges to the same solution as sparse LU, three
    realisations."""
    m = _gpu()
    wl = workloads.small(128, 64, seed=23, kind="voids", H=H, n_eig=6, etas=(0.3, 0.5, 0.7),
                         rmin=2.0, beta=8.0)
    prob = make_problem(m, wl, "mixed", tol=1e-10, patch_kernel="tensor_cores")
    prob.set_design(cuda(wl.rho), wl.rmin, wl.beta, wl.etas, wl.cell)
    prob.build_preconditioner()
    u, infos = prob.solve(cuda(wl.force), -1)
    ref = pipeline.run(wl, "direct", with_grad=False)
    grid, K0, oprob, _ = pipeline.build(wl)
    for k, inf in enumerate(infos):
        assert inf["status"] == 0 and inf["rel_residual"] <= 1e-10
        Kf = oprob.free_matrix(ref["E"][k])
        ug = grid.nodal_from_neutral(u[k].cpu().numpy())[oprob.free]
        ur = grid.nodal_from_neutral(ref["u"][k])[oprob.free]
        assert_energy(Kf, ur, ug)
        assert inf["compliance"] == pytest.approx(ref["c"][k], rel=1e-10)


def test_batch_solve_matches_single_solves_and_oracle():
    """Independent problems of uneven sizes solved concurrently: every instance's whole solve,
    its device-side loop included, runs inside one graph launch for the batch (checked by the
    handles' batch_graph_solves counters); every instance equals its own single solve bit for
    bit (same kernels, fixed reduction order) and the oracle's direct solve.  With per-kernel
    profiling on for one instance the batch takes the per-instance path and gives the same
    results."""
    m = _gpu()
    shapes = [(48, 16, 1), (64, 32, 3), (32, 16, 1), (96, 32, 3), (64, 16, 1)]
    wls = [workloads.small(nx, ny, seed=20 + b, kind="voids", bc="cantilever", H=8, n_eig=4,
                           etas=(0.5,) if ne == 1 else (0.3, 0.5, 0.7), rmin=2.0, beta=8.0)
           for b, (nx, ny, ne) in enumerate(shapes)]
    probs = []
    for wl in wls:
        p = make_problem(m, wl, "mixed", tol=1e-10)
        p.set_design(cuda(wl.rho), wl.rmin, wl.beta, wl.etas, wl.cell)
        probs.append(p)
    m.batch_build_preconditioner(probs)
    fs = [cuda(wl.force) for wl in wls]
    g0 = [p.stats()["batch_graph_solves"] for p in probs]
    us, infos = m.batch_solve(probs, fs)
    assert [p.stats()["batch_graph_solves"] - g for p, g in zip(probs, g0)] == [1] * len(probs)
    us2, infos2 = m.batch_solve(probs, fs)   # a second batch: a new graph, the same results
    probs[1].set_profiling(True)
    us3, infos3 = m.batch_solve(probs, fs)   # profiling on: one launch sequence per instance
    probs[1].set_profiling(False)
    assert [p.stats()["batch_graph_solves"] - g for p, g in zip(probs, g0)] == [2] * len(probs)
    for b, (p, wl) in enumerate(zip(probs, wls)):
        u1, inf1 = p.solve(cuda(wl.force), -1)
        assert torch.equal(u1, us[b]) and torch.equal(u1, us2[b]) and torch.equal(u1, us3[b])
        assert [i["iterations"] for i in inf1] == [i["iterations"] for i in infos[b]]
        assert [i["iterations"] for i in infos2[b]] == [i["iterations"] for i in infos3[b]] == \
            [i["iterations"] for i in infos[b]]
        assert all(i["ms"] > 0.0 for i in infos[b])
        ref = pipeline.run(wl, "direct", with_grad=False)
        for k, inf in enumerate(infos[b]):
            assert inf["status"] == 0 and inf["rel_residual"] <= 1e-10
            assert inf["compliance"] == pytest.approx(ref["c"][k], rel=1e-10)


def test_autograd_gradient_matches_central_differences():
    """torch.autograd through RobustCompliance (hand-written adjoint through SIMP, projection,
    tiling and the filter transpose) against central differences of the robust objective
    (h = 1e-3: the oracle's exact-solve differences agree with its gradient to ~1e-6 there;
    FP64 solves to 1e-12 keep the solver's share below 1e-7)."""
    m = _gpu()
    wl = workloads.small(48, 32, seed=17, kind="voids", cell=(16, 16), H=8, n_eig=6,
                         etas=(0.3, 0.5, 0.7), rmin=2.0, beta=8.0)
    prob = make_problem(m, wl, "fp64", tol=1e-12)
    f = cuda(wl.force)
    rho = cuda(wl.rho).requires_grad_(True)
    obj = m.RobustCompliance.apply(rho, prob, f, wl.rmin, wl.beta, wl.etas, wl.cell, 1.0)
    obj.backward()
    g = rho.grad.cpu().numpy().reshape(-1)
    ref = pipeline.run(wl, "direct")
    assert float(obj.detach()) == pytest.approx(ref["f_robust"], rel=1e-10)
    assert np.linalg.norm(g - ref["dfdrho"].reshape(-1)) <= 1e-7 * np.linalg.norm(g)

    def value(r):
        return float(m.RobustCompliance.apply(cuda(r.reshape(wl.rho.shape)), prob, f, wl.rmin,
                                              wl.beta, wl.etas, wl.cell, 1.0))

    h = 1e-3
    for j in np.random.default_rng(3).choice(g.size, 6, replace=False):
        rp = wl.rho.reshape(-1).copy(); rp[j] += h
        rm = wl.rho.reshape(-1).copy(); rm[j] -= h
        fd = (value(rp) - value(rm)) / (2 * h)
        assert abs(fd - g[j]) <= 1e-5 * max(abs(g[j]), 1e-3 * np.abs(g).max())


def test_periodic_26m_structure_on_a_reduced_copy_against_oracle():
    """The 3200 x 4096 periodic workload's structure (32 x 32 void cell, filter radius 3,
    beta 8, eta in {0.3, 0.5, 0.7}, H = 32, six eigenvectors) on a 192 x 256 copy: the
    mixed-precision batch of three realisations, the robust objective and its design
    gradient against the oracle's direct solves and chain."""
    m = _gpu()
    wl = workloads.make("mbb_c5", 16)
    assert (wl.nelx, wl.nely) == (192, 256)
    prob = make_problem(m, wl, "mixed", tol=1e-10)
    prob.set_design(cuda(wl.rho), wl.rmin, wl.beta, wl.etas, wl.cell)
    prob.build_preconditioner()
    u, infos = prob.solve(cuda(wl.force), -1)
    c, fr, g = prob.compliance_and_sensitivity(1.0)
    ref = pipeline.run(wl, "direct")
    for k, inf in enumerate(infos):
        assert inf["status"] == 0 and inf["rel_residual"] <= 1e-10
    assert np.allclose(c, ref["c"], rtol=1e-10)
    assert fr == pytest.approx(ref["f_robust"], rel=1e-10)
    g = g.cpu().numpy()
    assert np.linalg.norm(g - ref["dfdrho"]) <= 1e-7 * np.linalg.norm(ref["dfdrho"])


def test_injected_sweep_stall_times_out_and_handle_recovers():
    """A grid barrier of the coarse block sweeps that cannot complete (test injection) gives up
    within its bound: the call returns TIMEOUT, nothing faults, and the next call works."""
    m = _gpu()
    wl = workloads.small(96, 48, seed=12, kind="random", H=4, n_eig=4, Emin=1e-3)
    prob = make_problem(m, wl, coarse_solver="blocktri")
    prob.set_design(cuda(wl.rho), wl.rmin, wl.beta, wl.etas, wl.cell)
    prob.build_preconditioner()
    r = torch.from_numpy(np.random.default_rng(5).standard_normal(prob.n_dof)).cuda()
    z_ok = prob.apply_precond(r, m.FP64, 1).cpu().numpy()
    prob.inject(1)
    with pytest.raises(m.MstopoError) as ei:
        prob.apply_precond(r, m.FP64, 1)
    assert ei.value.status == 7   # MSTOPO_TIMEOUT
    z_again = prob.apply_precond(r, m.FP64, 1).cpu().numpy()
    assert np.array_equal(z_ok, z_again)


def test_reused_preconditioner_on_a_new_design():
    """reuse_preconditioner keeps the last build across set_design (basis re-use, Sec. 5.1):
    the solve on the perturbed design still reaches the tolerance and matches sparse LU."""
    m = _gpu()
    wl = workloads.small(64, 32, seed=15, kind="voids", H=8, n_eig=6, etas=(0.3, 0.5, 0.7),
                         rmin=2.0, beta=8.0)
    prob = make_problem(m, wl, "mixed", tol=1e-10, reuse_preconditioner=True)
    prob.set_design(cuda(wl.rho), wl.rmin, wl.beta, wl.etas, wl.cell)
    prob.build_preconditioner()
    prob.solve(cuda(wl.force), -1)
    rho2 = np.clip(wl.rho + 0.05 * np.random.default_rng(1).standard_normal(wl.rho.shape), 0, 1)
    prob.set_design(cuda(rho2), wl.rmin, wl.beta, wl.etas, wl.cell)
    u, infos = prob.solve(cuda(wl.force), -1)
    import copy
    wl2 = copy.copy(wl)
    wl2.rho = rho2
    ref = pipeline.run(wl2, "direct", with_grad=False)
    for k, inf in enumerate(infos):
        assert inf["status"] == 0 and inf["rel_residual"] <= 1e-10
        assert inf["compliance"] == pytest.approx(ref["c"][k], rel=1e-10)


def test_eigenvalue_threshold_basis():
    """lambda_thresh > 0 keeps only eigenvalues below it (Sec. 2.4, lambda_Omega), capped at
    n_eig: the kept count varies over the agglomerates and the solve still matches sparse LU."""
    m = _gpu()
    wl = workloads.small(64, 32, seed=16, kind="voids", H=8, n_eig=8)
    prob = make_problem(m, wl, "fp64", tol=1e-10, lambda_thresh=2e-3)
    prob.set_design(cuda(wl.rho), wl.rmin, wl.beta, wl.etas, wl.cell)
    info = prob.build_preconditioner()
    assert info["n_coarse"] < info["n_agglomerates"] * wl.n_eig
    u, infos = prob.solve(cuda(wl.force), -1)
    ref = pipeline.run(wl, "direct", with_grad=False)
    assert infos[0]["status"] == 0
    assert infos[0]["compliance"] == pytest.approx(ref["c"][0], rel=1e-10)


def test_fp32_matvec_all_realisations_in_one_launch():
    """apply_K_f32(realisation=-1, input_masked) is the flexible CG's launch: bit-identical to
    one call per realisation on inputs that are zero at the Dirichlet DOFs."""
    m = _gpu()
    wl = workloads.small(40, 24, seed=18, kind="random", H=4, etas=(0.3, 0.5, 0.7))
    prob = make_problem(m, wl)
    prob.set_design(cuda(wl.rho), wl.rmin, wl.beta, wl.etas, wl.cell)
    free = torch.from_numpy(~np.asarray(wl.fixed, dtype=bool).reshape(-1)).cuda()
    u = torch.randn(3, prob.n_dof, device="cuda", dtype=torch.float32) * free
    y_all = prob.apply_K_f32(u, -1, input_masked=True)
    for k in range(3):
        assert torch.equal(y_all[k], prob.apply_K_f32(u[k].clone(), k))


def test_invalid_calls_are_rejected():
    m = _gpu()
    wl33 = workloads.small(66, 66, seed=1, kind="solid", H=33)
    with pytest.raises(m.MstopoError):   # H above 32 (the patch solve's row coverage)
        m.Problem(66, 66, wl33.fixed, H=33, n_eig=4)
    wl = workloads.small(32, 16, seed=19, kind="voids", H=8, n_eig=4)
    prob = make_problem(m, wl)
    with pytest.raises(m.MstopoError) as ei:
        prob.solve(cuda(wl.force), -1)
    assert ei.value.status == 8   # NOT_READY
    prob.set_design(cuda(wl.rho), wl.rmin, wl.beta, wl.etas, wl.cell)
    with pytest.raises(m.MstopoError) as ei:
        prob.apply_K_f32(torch.zeros(prob.n_dof, device="cuda"), 3)
    assert ei.value.status == 1   # INVALID_ARG
    with pytest.raises(m.MstopoError):
        prob.inject(9)


@pytest.mark.parametrize("ratio,rebuilds", [(0.5, True), (100.0, False)])
def test_basis_update_rule(ratio, rebuilds):
    """The update rule of Sec. 5.2 (reuse_preconditioner with rebuild_ratio): a solve that needs
    more than ratio x the iterations of the first solve after the last build marks a rebuild,
    which the next all-realisation solve performs first.  Ratio 0.5 triggers on an unchanged
    design (same iteration count), ratio 100 never does; every solve still matches sparse LU."""
    m = _gpu()
    wl = workloads.small(64, 32, seed=21, kind="voids", H=8, n_eig=6, rmin=2.0, beta=8.0)
    prob = make_problem(m, wl, "mixed", tol=1e-10, reuse_preconditioner=True, rebuild_ratio=ratio)
    prob.set_design(cuda(wl.rho), wl.rmin, wl.beta, wl.etas, wl.cell)
    prob.build_preconditioner()
    ref = pipeline.run(wl, "direct", with_grad=False)
    f = cuda(wl.force)
    _, i1 = prob.solve(f, -1)
    st = prob.stats()
    assert st["builds"] == 1 and st["base_iterations"] == i1[0]["iterations"]
    assert st["rebuild_pending"] == 0
    _, i2 = prob.solve(f, -1)
    assert prob.stats()["rebuild_pending"] == (1 if rebuilds else 0)
    _, i3 = prob.solve(f, -1)
    st = prob.stats()
    assert st["builds"] == (2 if rebuilds else 1)
    for inf in i1 + i2 + i3:
        assert inf["status"] == 0
        assert inf["compliance"] == pytest.approx(ref["c"][0], rel=1e-10)


# ---------------------------------------------------------------- the paper's preconditioner
def _free_vec(grid, oprob, v):
    return grid.nodal_from_neutral(np.asarray(v))[oprob.free]


def _neutral(grid, oprob, vf):
    z = np.zeros(grid.n_dof)
    z[oprob.free] = vf
    return grid.nodal_to_neutral(z)


@pytest.mark.parametrize("size,bc", [((28, 12), "mbb"), ((33 * 4, 5 * 4), "cantilever")])
def test_sgs_sweep_matches_oracle(size, bc):
    """One symmetric node-block Gauss-Seidel sweep from zero (colours 0..3, then 3..0;
    apply_precond part 2 of the multiplicative preconditioner) against the oracle's
    colour sweep: FP64 to round-off, FP32 to its unit round-off times the conditioning
    of the 2x2 node blocks."""
    m = _gpu()
    wl = workloads.small(*size, seed=31, kind="voids", bc=bc, H=4, n_eig=4, Emin=1e-3)
    prob = make_problem(m, wl, "mixed", preconditioner="sgs")
    prob.set_design(cuda(wl.rho), wl.rmin, wl.beta, wl.etas, wl.cell)
    prob.build_preconditioner()
    grid, K0, oprob, chain = pipeline.build(wl)
    E = chain.forward(wl.rho)["E"][0]
    K = oprob.free_matrix(E)
    S = smoother.SymmetricGaussSeidel(oprob, K, "colour")
    r = np.random.default_rng(9).standard_normal((wl.nely + 1, wl.nelx + 1, 2))
    rf = _free_vec(grid, oprob, r)
    z_ref = _neutral(grid, oprob, S.sweep(np.zeros_like(rf), rf))
    z = prob.apply_precond(cuda(r), m.FP64, 2).cpu().numpy()
    assert np.linalg.norm(z - z_ref) <= 1e-12 * np.linalg.norm(z_ref)
    z32 = prob.apply_precond(cuda(r), m.MIXED, 2).cpu().numpy()
    assert np.linalg.norm(z32 - z_ref) <= 1e-4 * np.linalg.norm(z_ref)


def test_multiplicative_sgs_operator_matches_oracle():
    """SGS, coarse correction, SGS (Sec. 2.4.2) against the oracle's operator (the coarse
    space within the eigen-solve's tolerance) and symmetric to round-off."""
    m = _gpu()
    wl = workloads.small(64, 32, seed=32, kind="voids", H=8, n_eig=4, Emin=1e-3)
    prob = make_problem(m, wl, "fp64", preconditioner="sgs")
    prob.set_design(cuda(wl.rho), wl.rmin, wl.beta, wl.etas, wl.cell)
    prob.build_preconditioner()
    grid, K0, oprob, chain = pipeline.build(wl)
    E = chain.forward(wl.rho)["E"][0]
    K = oprob.free_matrix(E)
    tl = msfem.TwoLevel(oprob, E, wl.H, wl.n_eig, with_patches=False)
    Mref = smoother.MultiplicativeTwoLevel(K, smoother.SymmetricGaussSeidel(oprob, K, "colour"),
                                           tl.coarse)
    rng = np.random.default_rng(10)
    a = rng.standard_normal((wl.nely + 1, wl.nelx + 1, 2))
    b = rng.standard_normal((wl.nely + 1, wl.nelx + 1, 2))
    fa, fb = _free_vec(grid, oprob, a), _free_vec(grid, oprob, b)
    za = prob.apply_precond(cuda(a), m.FP64, 0).cpu().numpy()
    zb = prob.apply_precond(cuda(b), m.FP64, 0).cpu().numpy()
    z_ref = _neutral(grid, oprob, Mref.apply(fa))
    assert np.linalg.norm(za - z_ref) <= 1e-6 * np.linalg.norm(z_ref)
    ga, gb = _free_vec(grid, oprob, za), _free_vec(grid, oprob, zb)
    assert abs(ga @ fb - fa @ gb) <= 1e-10 * np.linalg.norm(ga) * np.linalg.norm(fb)
    assert ga @ fa > 0.0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("etas", [(0.5,), (0.3, 0.5, 0.7)])
def test_solve_with_multiplicative_sgs(precision, etas):
    """The flexible CG with the paper's multiplicative SGS preconditioner converges to the
    sparse-LU solution of every realisation."""
    m = _gpu()
    wl = workloads.small(96, 48, seed=33, kind="voids", H=8, n_eig=6, etas=etas, rmin=2.0,
                         beta=8.0)
    prob = make_problem(m, wl, precision, tol=1e-10, preconditioner="sgs")
    prob.set_design(cuda(wl.rho), wl.rmin, wl.beta, wl.etas, wl.cell)
    prob.build_preconditioner()
    u, infos = prob.solve(cuda(wl.force), -1)
    ref = pipeline.run(wl, "direct", with_grad=False)
    grid, K0, oprob, _ = pipeline.build(wl)
    for k, inf in enumerate(infos):
        assert inf["status"] == 0 and inf["rel_residual"] <= 1e-10
        Kf = oprob.free_matrix(ref["E"][k])
        ug = grid.nodal_from_neutral(u[k].cpu().numpy())[oprob.free]
        ur = grid.nodal_from_neutral(ref["u"][k])[oprob.free]
        assert_energy(Kf, ur, ug)
        assert inf["compliance"] == pytest.approx(ref["c"][k], rel=1e-10)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_device_side_loop_equals_host_driven_loop(precision):
    """With CUDA graphs the whole flexible-CG loop is one graph launch (a WHILE conditional
    node, an IF node for the FP64 residual replacement, convergence decided on the device);
    without graphs the host drives chunks of iterations.  Same kernels, same decisions: the
    solutions are bitwise equal, three realisations, and the stats show which loop ran."""
    m = _gpu()
    wl = workloads.small(96, 48, seed=13, kind="voids", H=8, n_eig=6, etas=(0.3, 0.5, 0.7),
                         rmin=2.0, beta=8.0)
    out = {}
    for graphs in (True, False):
        prob = make_problem(m, wl, precision, tol=1e-10, graphs=graphs)
        prob.set_design(cuda(wl.rho), wl.rmin, wl.beta, wl.etas, wl.cell)
        prob.build_preconditioner()
        u, infos = prob.solve(cuda(wl.force), -1)
        u2, infos2 = prob.solve(cuda(wl.force), -1)
        assert torch.equal(u, u2)
        out[graphs] = (u, [i["iterations"] for i in infos], [i["rel_residual"] for i in infos])
        assert prob.stats()["device_loop_solves"] == (2 if graphs else 0)
        assert all(i["status"] == 0 and i["rel_residual"] <= 1e-10 for i in infos)
    assert torch.equal(out[True][0], out[False][0])
    assert out[True][1] == out[False][1] and out[True][2] == out[False][2]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("etas", [(0.5,), (0.3, 0.5, 0.7)])
def test_gmres_with_multiplicative_sgs_matches_oracle(precision, etas):
    """GMRES(m), the paper's outer method for its multiplicative preconditioner (Sec. 2.4.2),
    restarted every 20 steps: every realisation converges to the sparse-LU solution, and the
    iteration count is the oracle's GMRES on the same operator (its SGS in the GPU's colour
    order and the same spectral coarse space)."""
    m = _gpu()
    wl = workloads.small(96, 48, seed=33, kind="voids", H=8, n_eig=6, etas=etas, rmin=2.0,
                         beta=8.0)
    prob = make_problem(m, wl, precision, tol=1e-10, preconditioner="sgs", krylov="gmres",
                        gmres_restart=20)
    prob.set_design(cuda(wl.rho), wl.rmin, wl.beta, wl.etas, wl.cell)
    prob.build_preconditioner()
    u, infos = prob.solve(cuda(wl.force), -1)
    u2, _ = prob.solve(cuda(wl.force), -1)
    assert torch.equal(u, u2)   # deterministic reductions
    ref = pipeline.run(wl, "direct", with_grad=False)
    grid, K0, oprob, chain = pipeline.build(wl)
    E = chain.forward(wl.rho)["E"]
    for k, inf in enumerate(infos):
        assert inf["status"] == 0 and inf["rel_residual"] <= 1e-10
        Kf = oprob.free_matrix(ref["E"][k])
        ug = grid.nodal_from_neutral(u[k].cpu().numpy())[oprob.free]
        ur = grid.nodal_from_neutral(ref["u"][k])[oprob.free]
        assert_energy(Kf, ur, ug)
        assert inf["compliance"] == pytest.approx(ref["c"][k], rel=1e-10)
    # the oracle's GMRES with the preconditioner built on each realisation's moduli (the
    # coarse basis from the dilated realisation, as the library builds it)
    k0 = 0
    K = oprob.free_matrix(E[k0])
    tl = msfem.TwoLevel(oprob, E[k0], wl.H, wl.n_eig, with_patches=False)
    Mref = smoother.MultiplicativeTwoLevel(K, smoother.SymmetricGaussSeidel(oprob, K, "colour"),
                                           tl.coarse)
    f = grid.nodal_from_neutral(wl.force)[oprob.free]
    _, it_ref, rel_ref = smoother.gmres(K, f, Mref.apply, tol=1e-10, restart=20, maxit=2000)
    print("GPU", [i["iterations"] for i in infos], "oracle", it_ref, rel_ref)
    assert rel_ref <= 1e-10
    assert abs(infos[k0]["iterations"] - it_ref) <= max(2, 0.05 * it_ref)


def test_autotuned_patch_solves_time_every_configuration_once_per_shape():
    """MSTOPO_EXEC_AUTOTUNE: the first build of a shape times the FP32 patch-solve
    configurations and reports it (patch_tuned 1); a second problem of the same shape keeps
    the choice (2) and builds the same kernel; the solves match sparse LU as with the cost
    model's choice, and the patch solves match the FP64 ones within the FP32 bound of
    whichever kernel was chosen."""
    m = _gpu()
    wl = workloads.small(256, 128, seed=31, kind="voids", H=32, n_eig=4, etas=(0.5,),
                         rmin=2.0, beta=8.0)
    infos = []
    for _ in range(2):
        prob = make_problem(m, wl, "mixed", tol=1e-10, autotune=True)
        prob.set_design(cuda(wl.rho), wl.rmin, wl.beta, wl.etas, wl.cell)
        infos.append(prob.build_preconditioner())
        u, sinfo = prob.solve(cuda(wl.force), -1)
        assert sinfo[0]["status"] == 0 and sinfo[0]["rel_residual"] <= 1e-10
        r = cuda(np.random.default_rng(3).standard_normal((wl.nely + 1, wl.nelx + 1, 2)))
        z64 = prob.apply_precond(r, m.FP64, 2)
        z32 = prob.apply_precond(r, m.MIXED, 2)
        err = (torch.linalg.norm(z32 - z64) / torch.linalg.norm(z64)).item()
        assert err < 1e-5, (infos[-1], err)
        del prob
    a, b = infos
    assert (a["patch_tuned"], b["patch_tuned"]) in ((1, 2), (2, 2))   # (2, 2) if an earlier test timed it
    assert a["patch_kernel"] == b["patch_kernel"] and a["patch_cols"] == b["patch_cols"]
    assert a["patch_cols"] in (4, 8, 16, 128)
    assert (a["patch_kernel"] == 2) == (a["patch_cols"] == 128)
    ref = pipeline.run(wl, "direct", with_grad=False)
    grid, K0, oprob, _ = pipeline.build(wl)
    Kf = oprob.free_matrix(ref["E"][0])
    ug = grid.nodal_from_neutral(u[0].cpu().numpy())[oprob.free]
    ur = grid.nodal_from_neutral(ref["u"][0])[oprob.free]
    assert_energy(Kf, ur, ug)
