"""Pins for oracle/design.py: the filter, projection, SIMP and the adjoint chain (Sec. 4)."""
import numpy as np
import pytest

import workloads
from oracle import design, pipeline


def brute_filter(rho, rmin, periodic):
    ny, nx = rho.shape
    out = np.zeros_like(rho)
    for y in range(ny):
        for x in range(nx):
            s = w = 0.0
            for yy in range(ny if not periodic else 3 * ny):
                for xx in range(nx if not periodic else 3 * nx):
                    if periodic:
                        d = np.hypot(xx - nx - x, yy - ny - y)
                        val = rho[yy % ny, xx % nx]
                    else:
                        d = np.hypot(xx - x, yy - y)
                        val = rho[yy, xx]
                    wt = max(0.0, rmin - d)
                    s += wt * val
                    w += wt
            out[y, x] = s / w
    return out


@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("rmin", [1.5, 2.0, 3.0])
def test_filter_against_brute_force(periodic, rmin):
    rho = np.random.default_rng(3).random((5, 7))
    H = design.filter_matrix(7, 5, rmin, periodic)
    assert np.allclose((H @ rho.ravel()).reshape(5, 7), brute_filter(rho, rmin, periodic), atol=1e-14)


def test_periodic_filter_is_centre_tile_of_3x3_block():
    """Sec. 4.3: periodic filtering = standard filter applied to a 3x3 block of the cell."""
    rho = np.random.default_rng(4).random((6, 8))
    Hp = design.filter_matrix(8, 6, 2.5, True)
    Hf = design.filter_matrix(24, 18, 2.5, False)
    big = (Hf @ np.tile(rho, (3, 3)).ravel()).reshape(18, 24)
    assert np.allclose((Hp @ rho.ravel()).reshape(6, 8), big[6:12, 8:16], atol=1e-14)


@pytest.mark.parametrize("periodic", [False, True])
def test_filter_preserves_constants(periodic):
    H = design.filter_matrix(9, 4, 3.0, periodic)
    assert np.allclose(H @ np.full(36, 0.37), 0.37, atol=1e-15)


def test_projection_endpoints_limit_and_derivative():
    for beta in (1.0, 8.0, 64.0):
        for eta in (0.3, 0.5, 0.7):
            assert design.heaviside(0.0, beta, eta) == pytest.approx(0.0, abs=1e-15)
            assert design.heaviside(1.0, beta, eta) == pytest.approx(1.0, abs=1e-15)
            x = np.linspace(0.05, 0.95, 7)
            h = 1e-6
            fd = (design.heaviside(x + h, beta, eta) - design.heaviside(x - h, beta, eta)) / (2 * h)
            assert np.allclose(design.heaviside_deriv(x, beta, eta), fd, rtol=1e-6, atol=1e-8)
    x = np.linspace(0, 1, 11)
    assert np.allclose(design.heaviside(x, 1e-5, 0.5), x, atol=1e-9)


def test_robust_combine_gradient():
    c = np.array([1.3, 2.1, 0.7])
    f, w = design.robust_combine(c)
    assert f == pytest.approx(c.mean() + np.sqrt(np.mean((c - c.mean()) ** 2)), rel=1e-15)
    for k in range(3):
        d = np.zeros(3); d[k] = 1e-6
        fd = (design.robust_combine(c + d)[0] - design.robust_combine(c - d)[0]) / 2e-6
        assert w[k] == pytest.approx(fd, rel=1e-7)


def _objective(wl, rho):
    wl2 = workloads.Workload(**{**wl.__dict__, "rho": rho})
    return pipeline.run(wl2, "direct", with_grad=False)["f_robust"]


@pytest.mark.parametrize("cell", [None, (4, 4)])
@pytest.mark.parametrize("etas", [(0.5,), (0.3, 0.5, 0.7)])
def test_design_gradient_against_central_differences(cell, etas):
    """Self-adjoint sensitivity (Sec. 4.2) chained through SIMP, projection, tiling and the
    filter, and the robust combination (Sec. 4.4), against central differences."""
    wl = workloads.small(8, 4, seed=5, kind="random", cell=cell, etas=etas, rmin=1.6, beta=3.0)
    wl.Emin = 1e-3
    rho = 0.2 + 0.6 * wl.rho
    wl.rho = rho
    g = pipeline.run(wl, "direct")["dfdrho"]
    rng = np.random.default_rng(0)
    idx = rng.choice(rho.size, 6, replace=False)
    for i in idx:
        h = 1e-5
        rp = rho.copy().ravel(); rp[i] += h
        rm = rho.copy().ravel(); rm[i] -= h
        fd = (_objective(wl, rp.reshape(rho.shape)) - _objective(wl, rm.reshape(rho.shape))) / (2 * h)
        assert g.ravel()[i] == pytest.approx(fd, rel=1e-6, abs=1e-9 * np.abs(g).max())
