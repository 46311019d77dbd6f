"""Pins for oracle/pde_filter.py: the PDE (Helmholtz) density filter with collapsed-DOF
periodicity and connectivity (Sec. 4.3, 4.5)."""
import numpy as np
import pytest

from oracle import pde_filter as pf


def test_element_matrices_by_gauss_quadrature():
    """int grad N_a . grad N_b and int N_a N_b on the unit square by 2x2 Gauss quadrature
    (exact for these bilinear products)."""
    g = 0.5 + np.array([-1.0, 1.0]) / (2.0 * np.sqrt(3.0))
    corners = ((0, 0), (1, 0), (1, 1), (0, 1))
    K = np.zeros((4, 4))
    M = np.zeros((4, 4))
    for x in g:
        for y in g:
            N = np.array([(x if cx else 1 - x) * (y if cy else 1 - y) for cx, cy in corners])
            dx = np.array([(1 if cx else -1) * (y if cy else 1 - y) for cx, cy in corners])
            dy = np.array([(x if cx else 1 - x) * (1 if cy else -1) for cx, cy in corners])
            K += 0.25 * (np.outer(dx, dx) + np.outer(dy, dy))
            M += 0.25 * np.outer(N, N)
    Kl, Me = pf.element_matrices()
    assert np.allclose(Kl, K, atol=1e-14) and np.allclose(Me, M, atol=1e-14)


FILTERS = {
    "plain": lambda: pf.plain(12, 8, 4.0),
    "periodic": lambda: pf.periodic_cell(16, 12, 5.0),
    "stacked": lambda: pf.stacked_blocks(16, (8, 12, 6), 4.0),
}


@pytest.mark.parametrize("kind", sorted(FILTERS))
def test_constants_are_preserved(kind):
    F = FILTERS[kind]()
    assert np.allclose(F.apply(np.full(F.mesh.n_el, 0.37)), 0.37, atol=1e-13)


@pytest.mark.parametrize("kind", sorted(FILTERS))
def test_filter_operator_is_symmetric(kind):
    """rho_tilde = T^T P K^-1 P^T T rho is symmetric: the sensitivity chain uses the same map."""
    F = FILTERS[kind]()
    rng = np.random.default_rng(1)
    a, b = rng.random(F.mesh.n_el), rng.random(F.mesh.n_el)
    assert abs(F.apply(a) @ b - a @ F.apply(b)) <= 1e-12 * np.linalg.norm(a) * np.linalg.norm(b)


def test_periodic_filter_commutes_with_cyclic_shifts():
    nx, ny = 16, 12
    F = pf.periodic_cell(nx, ny, 5.0)
    rho = np.random.default_rng(2).random((ny, nx))
    shifted = np.roll(rho, (3, 5), axis=(0, 1))
    a = F.apply(rho.ravel()).reshape(ny, nx)
    b = F.apply(shifted.ravel()).reshape(ny, nx)
    assert np.allclose(np.roll(a, (3, 5), axis=(0, 1)), b, atol=1e-13)


def test_cosine_mode_is_damped_like_the_continuum_symbol():
    """On a periodic cell a cosine along x (at element centres) is an eigenvector of the
    discrete filter; its eigenvalue approaches the continuum 1 / (1 + r^2 k^2)."""
    N, rmin = 64, 6.0
    F = pf.periodic_cell(N, 8, rmin)
    ex = np.tile(np.arange(N), 8)
    rho = np.cos(2.0 * np.pi * (ex + 0.5) / N)
    out = F.apply(rho)
    alpha = (out @ rho) / (rho @ rho)
    assert np.allclose(out, alpha * rho, atol=1e-12)
    r = rmin / (2.0 * np.sqrt(3.0))
    assert abs(alpha - 1.0 / (1.0 + (r * 2.0 * np.pi / N) ** 2)) < 5e-3


def test_identical_stacked_blocks_reduce_to_one_periodic_cell():
    """With the same cell design in every block, collapsing all tops and bottoms together
    and each cell's sides gives each block exactly the single periodic cell's filter."""
    nx, ny, B, rmin = 12, 10, 3, 4.0
    rho = np.random.default_rng(3).random(nx * ny)
    one = pf.periodic_cell(nx, ny, rmin).apply(rho)
    many = pf.stacked_blocks(nx, (ny,) * B, rmin).apply(np.tile(rho, B))
    for b in range(B):
        assert np.allclose(many[b * nx * ny:(b + 1) * nx * ny], one, atol=1e-13)


def test_stacked_blocks_couple_across_interfaces():
    """Connectivity: the filtered field of one block depends on the other blocks' designs
    (a change in block 0 reaches block 2 through the shared top/bottom edges)."""
    F = pf.stacked_blocks(12, (8, 8, 8), 4.0)
    n = 12 * 8
    rho = np.random.default_rng(4).random(3 * n)
    d = rho.copy()
    d[:n] += 0.1
    assert np.abs(F.apply(d)[2 * n:] - F.apply(rho)[2 * n:]).max() > 1e-6
