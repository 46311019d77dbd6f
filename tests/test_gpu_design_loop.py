"""The design loop on the GPU (Sec. 4.4, 4.5): the expected-volume constraint, the method of
moving asymptotes and the continuation schedule, against oracle/optimise.py."""
import copy

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import workloads  # noqa: E402
from oracle import optimise  # noqa: E402


def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1411_3923_gb300 as m
    return m


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _problem(m, wl, tol=1e-11):
    return m.Problem(wl.nelx, wl.nely, wl.fixed, nu=wl.nu, E0=wl.E0, Emin=wl.Emin,
                     penal=wl.penal, H=wl.H, n_eig=wl.n_eig, precision="fp64", tol=tol,
                     max_iter=5000)


@pytest.mark.parametrize("cell,etas", [(None, (0.5,)), ((8, 4), (0.3, 0.5, 0.7))])
def test_volume_constraint_and_gradient_match_oracle(cell, etas):
    m = _gpu()
    wl = workloads.small(32, 16, seed=41, kind="random", H=8, n_eig=4, etas=etas, cell=cell,
                         rmin=2.0, beta=4.0)
    prob = _problem(m, wl)
    prob.set_design(cuda(wl.rho), wl.rmin, wl.beta, wl.etas, wl.cell)
    g, dg = prob.volume(0.4)
    _, _, g_ref, dg_ref, _ = optimise.robust_objective_and_volume(wl, wl.rho, 0.4)
    assert g == pytest.approx(g_ref, rel=1e-13, abs=1e-15)
    dg = dg.cpu().numpy().reshape(np.shape(dg_ref))
    assert np.abs(dg - dg_ref).max() <= 1e-13 * np.abs(dg_ref).max()


def test_mma_steps_match_oracle():
    """Five consecutive steps on the same seeded (f, df, g, dg) sequence: the asymptote
    updates from the third step on and the dual's multiplier follow the oracle."""
    m = _gpu()
    n = 3000
    rng = np.random.default_rng(3)
    x = rng.uniform(0.2, 0.8, n)
    ref = optimise.MMA(n, 0.0, 1.0, s0=0.25)
    gpu = m.MMA(n, 0.0, 1.0, s0=0.25)
    xg = cuda(x)
    for k in range(5):
        df = rng.standard_normal(n) - 0.3
        dg = np.abs(rng.standard_normal(n)) / n + 1e-4
        g = 0.05 if k % 2 == 0 else -0.02
        x_ref = ref.step(x, 1.0, df, g, dg)
        xg = gpu.step(xg, 1.0, cuda(df), g, cuda(dg))
        diff = np.abs(xg.cpu().numpy() - x_ref).max()
        print("step", k, "max |x - x_ref|", diff, "lam", gpu.lam)
        assert diff <= 1e-12
        x = x_ref
        xg = cuda(x)    # the next step from the oracle's iterate (isolates each step)


@pytest.mark.parametrize("etas", [(0.5,), (0.3, 0.5, 0.7)])
def test_optimise_matches_oracle(etas):
    """Two continuation stages (penal 3, beta 1 then 2) of robust compliance minimisation
    under the expected-volume constraint: the objective history and the final design follow
    the oracle (direct solves), the GPU solving each state to a true residual of 1e-11."""
    m = _gpu()
    wl = workloads.small(48, 24, seed=42, kind="random", H=8, n_eig=4, etas=etas, rmin=2.0,
                         beta=1.0)
    wl.rho = np.full((wl.nely, wl.nelx), 0.5)
    stages = [(3.0, 1.0, 3), (3.0, 2.0, 3)]
    hist_ref = []
    rho_ref = optimise.optimise(copy.copy(wl), 0.5, stages, kappa=1.0, rel_change=1e-9,
                                history=hist_ref)
    prob = _problem(m, wl)
    prob.set_design(cuda(wl.rho), wl.rmin, wl.beta, wl.etas, wl.cell)
    rho, hist = prob.optimise(cuda(wl.rho), cuda(wl.force), stages, 0.5, kappa=1.0,
                              rel_change=1e-9)
    assert len(hist) == len(hist_ref)
    for h, r in zip(hist, hist_ref):
        print(h["stage"], h["iteration"], h["f"], r["f"], h["g"], r["g"])
        assert h["f"] == pytest.approx(r["f"], rel=1e-7)
        assert h["g"] == pytest.approx(r["g"], rel=1e-7, abs=1e-9)
    assert np.abs(rho.cpu().numpy().reshape(rho_ref.shape) - rho_ref).max() <= 1e-6


def test_robust_verification_matches_oracle():
    """Compliance of one design over seven thresholds spread on [0.3, 0.7] (Sec. 4.4): two
    batches of realisations on the GPU against one direct solve per threshold."""
    m = _gpu()
    wl = workloads.small(48, 24, seed=43, kind="voids", H=8, n_eig=4, etas=(0.5,), rmin=2.0,
                         beta=8.0)
    etas = np.linspace(0.3, 0.7, 7)
    prob = _problem(m, wl)
    prob.set_design(cuda(wl.rho), wl.rmin, wl.beta, wl.etas, wl.cell)
    c = prob.robust_verification(cuda(wl.rho), cuda(wl.force), etas)
    c_ref = optimise.robust_verification(wl, wl.rho, etas)
    print(c, c_ref)
    assert np.allclose(c, c_ref, rtol=1e-10, atol=0.0)
    assert np.all(np.diff(c) > 0.0)    # thinner (eroded) designs are more compliant
