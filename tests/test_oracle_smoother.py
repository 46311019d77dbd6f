"""Pins for oracle/smoother.py: the symmetric Gauss-Seidel smoother and the paper's
multiplicative two-level preconditioner (Sec. 2.4.2)."""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import workloads
from oracle import msfem, pipeline, smoother


def setup(nelx=12, nely=8, H=4, seed=0, Emin=1e-3, n_eig=4):
    wl = workloads.small(nelx, nely, seed=seed, kind="voids", H=H, Emin=Emin, n_eig=n_eig)
    grid, K0, prob, chain = pipeline.build(wl)
    E = chain.forward(wl.rho)["E"][0]
    return wl, grid, prob, E, prob.free_matrix(E)


def test_lex_forward_sweep_is_the_textbook_loop():
    """x_i <- (r_i - sum_{j<i} K_ij x_j(new) - sum_{j>i} K_ij x_j(old)) / K_ii, DOF by DOF."""
    wl, grid, prob, E, K = setup(6, 4, H=2)
    S = smoother.SymmetricGaussSeidel(prob, K, "lex")
    rng = np.random.default_rng(1)
    r, x0 = rng.standard_normal(K.shape[0]), rng.standard_normal(K.shape[0])
    Kd = K.toarray()
    x = x0.copy()
    for i in range(len(x)):
        s = r[i] - Kd[i, :i] @ x[:i] - Kd[i, i + 1:] @ x[i + 1:]
        x[i] = s / Kd[i, i]
    assert np.allclose(S.forward(x0, r), x, rtol=1e-12, atol=1e-12)
    # and the backward sweep runs the same loop in reverse order
    x = x0.copy()
    for i in reversed(range(len(x))):
        s = r[i] - Kd[i, :i] @ x[:i] - Kd[i, i + 1:] @ x[i + 1:]
        x[i] = s / Kd[i, i]
    assert np.allclose(S.backward(x0, r), x, rtol=1e-12, atol=1e-12)


def _colour_permutation(grid, prob):
    """Free DOFs in colour order (nodes of colour 0, 1, 2, 3; x before y in a node), with the
    colour and node of every permuted DOF."""
    pos = -np.ones(grid.n_dof, dtype=np.int64)
    pos[prob.free] = np.arange(prob.free.size)
    perm, col, node = [], [], []
    for c in range(4):
        for j in range(c >> 1, grid.nely + 1, 2):
            for i in range(c & 1, grid.nelx + 1, 2):
                n = grid.node(i, j)
                for d in (2 * n, 2 * n + 1):
                    if pos[d] >= 0:
                        perm.append(pos[d]); col.append(c); node.append(n)
    return np.array(perm), np.array(col), np.array(node)


def test_colour_sweep_is_a_block_triangular_solve():
    """The colour-by-colour node-block sweep equals x + P^T (D_b + L_c)^-1 P (r - K x), with
    D_b the node blocks and L_c the couplings to nodes of earlier colours in the permuted
    matrix (a direct sparse solve, not the sweep); no two nodes of a colour are coupled."""
    wl, grid, prob, E, K = setup(10, 6, H=2, seed=3)
    perm, col, node = _colour_permutation(grid, prob)
    Kp = sp.csr_matrix(K)[perm][:, perm].tocoo()
    same_colour_other_node = (col[Kp.row] == col[Kp.col]) & (node[Kp.row] != node[Kp.col])
    assert np.all(Kp.data[same_colour_other_node] == 0.0)
    keep = (col[Kp.row] > col[Kp.col]) | (node[Kp.row] == node[Kp.col])
    Lf = sp.csr_matrix((Kp.data[keep], (Kp.row[keep], Kp.col[keep])), shape=Kp.shape)
    keep_b = (col[Kp.row] < col[Kp.col]) | (node[Kp.row] == node[Kp.col])
    Ub = sp.csr_matrix((Kp.data[keep_b], (Kp.row[keep_b], Kp.col[keep_b])), shape=Kp.shape)
    S = smoother.SymmetricGaussSeidel(prob, K, "colour")
    rng = np.random.default_rng(2)
    r, x0 = rng.standard_normal(K.shape[0]), rng.standard_normal(K.shape[0])
    res = r - K @ x0
    want = x0.copy()
    want[perm] += spla.spsolve(Lf.tocsc(), res[perm])
    assert np.allclose(S.forward(x0, r), want, rtol=1e-11, atol=1e-11)
    res = r - K @ x0
    want = x0.copy()
    want[perm] += spla.spsolve(Ub.tocsc(), res[perm])
    assert np.allclose(S.backward(x0, r), want, rtol=1e-11, atol=1e-11)


def test_sgs_and_multiplicative_operators_are_spd():
    """SGS(0; .) and the multiplicative two-level operator are symmetric and positive
    definite (symmetric smoother before and after the coarse correction)."""
    wl, grid, prob, E, K = setup(16, 8, H=4, seed=5)
    tl = msfem.TwoLevel(prob, E, wl.H, wl.n_eig, with_patches=False)
    rng = np.random.default_rng(4)
    a, b = rng.standard_normal(K.shape[0]), rng.standard_normal(K.shape[0])
    for order in ("lex", "colour"):
        S = smoother.SymmetricGaussSeidel(prob, K, order)
        Sa, Sb = S.sweep(np.zeros_like(a), a), S.sweep(np.zeros_like(b), b)
        assert abs(Sa @ b - a @ Sb) <= 1e-10 * np.linalg.norm(Sa) * np.linalg.norm(b)
        M = smoother.MultiplicativeTwoLevel(K, S, tl.coarse)
        Ma, Mb = M.apply(a), M.apply(b)
        assert abs(Ma @ b - a @ Mb) <= 1e-9 * np.linalg.norm(Ma) * np.linalg.norm(b)
        assert Ma @ a > 0.0 and Mb @ b > 0.0


def test_multiplicative_error_propagation():
    """I - M^-1 K = (I - S K)(I - C K)(I - S K), S = SGS(0; .), C = R_c^T K_c^-1 R_c: the
    three-stage definition, evaluated as a product of its factors."""
    wl, grid, prob, E, K = setup(16, 8, H=4, seed=6)
    tl = msfem.TwoLevel(prob, E, wl.H, wl.n_eig, with_patches=False)
    S = smoother.SymmetricGaussSeidel(prob, K, "colour")
    M = smoother.MultiplicativeTwoLevel(K, S, tl.coarse)
    x = np.random.default_rng(7).standard_normal(K.shape[0])
    Sop = lambda v: S.sweep(np.zeros_like(v), v)
    e = x - Sop(K @ x)
    e = e - tl.coarse(K @ e)
    e = e - Sop(K @ e)
    assert np.allclose(x - M.apply(K @ x), e, rtol=1e-9, atol=1e-9 * np.linalg.norm(x))


def test_pcg_with_multiplicative_preconditioner_matches_direct_solve():
    """PCG with the paper's preconditioner converges to the sparse-LU solution, and in far
    fewer iterations than with the one-level SGS preconditioner (the coarse space at work)."""
    wl, grid, prob, E, K = setup(32, 16, H=8, seed=8, Emin=1e-9, n_eig=4)
    tl = msfem.TwoLevel(prob, E, wl.H, wl.n_eig, with_patches=False)
    f = grid.nodal_from_neutral(wl.force)[prob.free]
    u = spla.splu(K.tocsc()).solve(f)
    S = smoother.SymmetricGaussSeidel(prob, K, "colour")
    M = smoother.MultiplicativeTwoLevel(K, S, tl.coarse)
    x, it, rr = msfem.pcg(K, f, M.apply, tol=1e-10, maxit=2000)
    assert rr <= 1e-10 and msfem.energy_error(K, u, x) < 1e-6
    _, it_one, _ = msfem.pcg(K, f, lambda v: S.sweep(np.zeros_like(v), v), tol=1e-10, maxit=4000)
    assert 2 * it < it_one


def test_gmres_converges_in_as_many_steps_as_distinct_eigenvalues():
    """Unpreconditioned GMRES on a diagonal matrix with 4 distinct eigenvalues: the Krylov
    space holds the solution after exactly 4 steps, not before."""
    vals = np.tile([1.0, 2.0, 3.0, 5.0], 10)
    K = sp.diags(vals).tocsr()
    f = np.random.default_rng(11).standard_normal(vals.size)
    hist = []
    x, it, rr = smoother.gmres(K, f, lambda v: v, tol=1e-12, restart=20, history=hist)
    assert it == 4 and rr <= 1e-12
    assert hist[2] > 1e-6 * np.linalg.norm(f)
    assert np.allclose(x, f / vals, rtol=1e-12, atol=1e-12)


def test_gmres_residual_never_exceeds_pcg_residual():
    """Right-preconditioned GMRES and PCG (x0 = 0, the same SPD preconditioner) search the
    same affine Krylov space; GMRES minimises the 2-norm of the residual over it, so at every
    step its residual is at most PCG's."""
    wl, grid, prob, E, K = setup(16, 8, H=4, seed=12, Emin=1e-3)
    tl = msfem.TwoLevel(prob, E, wl.H, wl.n_eig, with_patches=False)
    M = smoother.MultiplicativeTwoLevel(K, smoother.SymmetricGaussSeidel(prob, K, "colour"),
                                        tl.coarse)
    f = grid.nodal_from_neutral(wl.force)[prob.free]
    hist = []
    smoother.gmres(K, f, M.apply, tol=1e-13, restart=100, maxit=12, history=hist)
    for j in range(1, min(12, len(hist)) + 1):
        xp, itp, _ = msfem.pcg(K, f, M.apply, tol=1e-300, maxit=j)
        assert itp == j
        assert hist[j - 1] <= np.linalg.norm(f - K @ xp) * (1 + 1e-8) + 1e-14 * np.linalg.norm(f)


def test_gmres_with_multiplicative_preconditioner_matches_direct_solve():
    """The paper's solver (GMRES + coarse/SGS multiplicative preconditioner) against sparse
    LU, at contrast 1e9."""
    wl, grid, prob, E, K = setup(32, 16, H=8, seed=13, Emin=1e-9, n_eig=4)
    tl = msfem.TwoLevel(prob, E, wl.H, wl.n_eig, with_patches=False)
    M = smoother.MultiplicativeTwoLevel(K, smoother.SymmetricGaussSeidel(prob, K, "colour"),
                                        tl.coarse)
    f = grid.nodal_from_neutral(wl.force)[prob.free]
    u = spla.splu(K.tocsc()).solve(f)
    x, it, rr = smoother.gmres(K, f, M.apply, tol=1e-10, restart=200, maxit=2000)
    assert rr <= 1e-10 and msfem.energy_error(K, u, x) < 1e-6
    _, it_pcg, _ = msfem.pcg(K, f, M.apply, tol=1e-10, maxit=2000)
    assert it <= it_pcg + 2


def test_colour_order_costs_few_iterations_against_lexicographic():
    """The GPU's colour node-block order against the lexicographic point order read from the
    paper: PCG with either multiplicative preconditioner converges to the same solution, and
    the colour order needs at most 30 % more iterations."""
    wl, grid, prob, E, K = setup(48, 24, H=8, seed=3, Emin=1e-9, n_eig=4)
    tl = msfem.TwoLevel(prob, E, wl.H, wl.n_eig, with_patches=False)
    f = grid.nodal_from_neutral(wl.force)[prob.free]
    u = spla.splu(K.tocsc()).solve(f)
    its = {}
    for order in ("lex", "colour"):
        M = smoother.MultiplicativeTwoLevel(K, smoother.SymmetricGaussSeidel(prob, K, order),
                                            tl.coarse)
        x, its[order], rr = msfem.pcg(K, f, M.apply, tol=1e-10, maxit=2000)
        assert rr <= 1e-10 and msfem.energy_error(K, u, x) < 1e-6
    assert its["colour"] <= 1.3 * its["lex"]
