"""The PDE (Helmholtz) density filter with collapsed degrees of freedom on the GPU (Sec. 4.3,
4.5) against the oracle's sparse-LU filter on the same domains."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import pde_filter as pf  # noqa: E402

CASES = [("plain", 20, [12], 2.5), ("periodic_cell", 16, [16], 3.0),
         ("stacked_blocks", 12, [6, 10, 8], 2.0), ("periodic_cell", 32, [24], 1.5)]


def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1411_3923_gb300 as m
    return m


def _oracle(domain, nx, ny, rmin):
    if domain == "plain":
        return pf.plain(nx, ny[0], rmin)
    if domain == "periodic_cell":
        return pf.periodic_cell(nx, ny[0], rmin)
    return pf.stacked_blocks(nx, ny, rmin)


@pytest.mark.parametrize("domain,nx,ny,rmin", CASES)
def test_pde_filter_matches_oracle(domain, nx, ny, rmin):
    m = _gpu()
    ref = _oracle(domain, nx, ny, rmin)
    f = m.PDEFilter(domain, nx, ny, rmin, tol=1e-13)
    assert f.n_el == ref.mesh.n_el
    assert f.n_unknowns == ref.P.shape[1]          # the same identification
    rng = np.random.default_rng(7)
    rho = rng.random(ref.mesh.n_el)
    out = f.apply(torch.from_numpy(rho).cuda()).cpu().numpy()
    exp = ref.apply(rho)
    print(domain, "CG iterations", f.iterations, "residual", f.rel_residual)
    assert f.rel_residual <= 1e-13
    assert np.abs(out - exp).max() <= 1e-11 * np.abs(exp).max()
    out2 = f.apply(torch.from_numpy(rho).cuda()).cpu().numpy()
    assert np.array_equal(out, out2)               # fixed-order sums
    f.close()


@pytest.mark.parametrize("domain,nx,ny,rmin", CASES[1:3])
def test_pde_filter_is_symmetric_and_preserves_constants(domain, nx, ny, rmin):
    """<F a, b> = <a, F b> (the sensitivity chain applies F unchanged) and F 1 = 1 (the mass
    term reproduces constants under natural boundary conditions)."""
    m = _gpu()
    f = m.PDEFilter(domain, nx, ny, rmin, tol=1e-13)
    rng = np.random.default_rng(8)
    a, b = rng.random(f.n_el), rng.random(f.n_el)
    fa = f.apply(torch.from_numpy(a).cuda()).cpu().numpy()
    fb = f.apply(torch.from_numpy(b).cuda()).cpu().numpy()
    assert abs(fa @ b - a @ fb) <= 1e-12 * abs(fa @ b)
    one = f.apply(torch.ones(f.n_el, dtype=torch.float64, device="cuda")).cpu().numpy()
    assert np.abs(one - 1.0).max() <= 1e-11
    f.close()
