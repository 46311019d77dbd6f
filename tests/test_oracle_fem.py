"""Pins for oracle/fem.py: closed forms and invariants of the Q4 discretisation (Sec. 2.1)."""
import numpy as np
import pytest

from oracle import fem


def rigid_modes(grid):
    i = np.repeat(np.arange(grid.nelx + 1), grid.nely + 1).astype(float)
    j = np.tile(np.arange(grid.nely + 1), grid.nelx + 1).astype(float)
    tx = np.zeros(grid.n_dof); tx[0::2] = 1
    ty = np.zeros(grid.n_dof); ty[1::2] = 1
    rot = np.zeros(grid.n_dof); rot[0::2] = -j; rot[1::2] = i
    return [tx, ty, rot]


@pytest.mark.parametrize("nu", [0.0, 0.3, 0.45])
def test_K0_hand_integrated_entries(nu):
    """Entries integrated by hand from the bilinear shape functions:
    K0[0,0] = (1/3 + (1-nu)/6)/(1-nu^2),  K0[0,1] = ((nu + (1-nu)/2)/4)/(1-nu^2),
    K0[0,2] = (-1/3 + (1-nu)/12)/(1-nu^2) (x-x coupling of the two bottom nodes),
    K0[0,4] = (-1/6 - (1-nu)/12)/(1-nu^2) (x-x coupling of diagonal nodes)."""
    K0 = fem.element_stiffness(nu)
    s = 1.0 / (1.0 - nu * nu)
    assert K0[0, 0] == pytest.approx((1 / 3 + (1 - nu) / 6) * s, rel=1e-14)
    assert K0[0, 1] == pytest.approx((nu + (1 - nu) / 2) / 4 * s, rel=1e-14)
    assert K0[0, 2] == pytest.approx((-1 / 3 + (1 - nu) / 12) * s, rel=1e-14)
    assert K0[0, 4] == pytest.approx((-1 / 6 - (1 - nu) / 12) * s, rel=1e-14)


def test_K0_symmetric_with_three_rigid_modes():
    K0 = fem.element_stiffness(0.3)
    assert np.abs(K0 - K0.T).max() < 1e-15
    lam = np.linalg.eigvalsh(K0)
    assert np.sum(np.abs(lam) < 1e-13) == 3 and np.all(lam[3:] > 1e-3)
    g = fem.Grid(1, 1)
    for m in rigid_modes(g):
        assert np.abs(K0 @ m[g.edof[0]]).max() < 1e-14


def test_assembled_K_kills_rigid_modes_and_is_spd_with_bcs():
    rng = np.random.default_rng(0)
    g = fem.Grid(7, 5)
    K0 = fem.element_stiffness(0.3)
    E = 10.0 ** rng.uniform(-9, 0, g.n_el)
    K = fem.assemble(g, E, K0)
    nK = abs(K).sum(axis=1).max()
    for m in rigid_modes(g):
        assert np.abs(K @ m).max() <= 1e-13 * nK * max(1.0, np.abs(m).max())
    assert abs(K - K.T).max() == 0.0
    fixed = np.zeros((6, 8, 2), np.uint8); fixed[:, 0, :] = 1
    Kf = fem.Problem(g, K0, fixed).free_matrix(E.reshape(g.nelx, g.nely).T)
    np.linalg.cholesky(Kf.toarray())


def test_patch_test_linear_field_gives_zero_interior_forces():
    g = fem.Grid(6, 4)
    K0 = fem.element_stiffness(0.3)
    K = fem.assemble(g, np.full(g.n_el, 2.0), K0)
    i = np.repeat(np.arange(7), 5).astype(float)
    j = np.tile(np.arange(5), 7).astype(float)
    u = np.zeros(g.n_dof)
    u[0::2] = 0.1 + 0.02 * i - 0.03 * j
    u[1::2] = -0.2 + 0.05 * i + 0.01 * j
    y = K @ u
    interior = (i > 0) & (i < 6) & (j > 0) & (j < 4)
    assert np.abs(y.reshape(-1, 2)[interior]).max() < 1e-14


@pytest.mark.parametrize("nelx,nely,E", [(12, 4, 2.5), (9, 3, 1.0)])
def test_bar_in_tension_compliance_closed_form(nelx, nely, E):
    """L x B plate, u_x = 0 on the left edge, u_y = 0 at the lower-left node, total load P
    spread consistently over the right edge: uniform stress, so Q4 is exact and
    c = P^2 L / (E B) (plane stress, unit thickness)."""
    P = 3.0
    g = fem.Grid(nelx, nely)
    K0 = fem.element_stiffness(0.3)
    fixed = np.zeros((nely + 1, nelx + 1, 2), np.uint8)
    fixed[:, 0, 0] = 1
    fixed[0, 0, 1] = 1
    f = np.zeros((nely + 1, nelx + 1, 2))
    f[:, nelx, 0] = P / nely
    f[0, nelx, 0] = f[nely, nelx, 0] = P / (2 * nely)
    prob = fem.Problem(g, K0, fixed)
    u = prob.solve_direct(np.full((nely, nelx), E), f)
    c = float(np.sum(f * u))
    assert c == pytest.approx(P * P * nelx / (E * nely), rel=1e-12)


def test_dof_count_of_the_largest_example():
    """Sec. 6.1.1: 2560 x 5120 elements carry 26,229,762 displacement DOFs."""
    g = fem.Grid.__new__(fem.Grid)
    g.nelx, g.nely = 2560, 5120
    assert 2 * (g.nelx + 1) * (g.nely + 1) == 26229762
    assert fem.Grid(256, 512).n_dof == 2 * 257 * 513


def test_matvec_matches_assembled_and_constrained_apply():
    rng = np.random.default_rng(1)
    g = fem.Grid(5, 3)
    K0 = fem.element_stiffness(0.3)
    E = rng.uniform(0.1, 1.0, (3, 5))
    fixed = np.zeros((4, 6, 2), np.uint8); fixed[:, 0, 0] = 1; fixed[0, 5, 1] = 1
    prob = fem.Problem(g, K0, fixed)
    u = rng.standard_normal((4, 6, 2))
    y = prob.apply(E, u)
    K = prob.stiffness(E).toarray()
    uo = g.nodal_from_neutral(u); uo[prob.fixed] = 0
    yo = K @ uo; yo[prob.fixed] = 0
    assert np.allclose(g.nodal_from_neutral(y), yo, rtol=0, atol=1e-13)
    # the element loop and the assembled matrix are independent routes to K u


def test_paper_printed_mesh_sizes():
    """Element and DOF counts printed in the paper (tests/golden/paper_mesh_sizes.txt)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_mesh_sizes.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        nelx, nely, nel, ndof = map(int, r[:4])
        g = fem.Grid(min(nelx, 64), min(nely, 32))        # the formula, on a small instance
        assert g.n_dof == 2 * (g.nelx + 1) * (g.nely + 1)
        assert nelx * nely == nel
        assert 2 * (nelx + 1) * (nely + 1) == ndof
