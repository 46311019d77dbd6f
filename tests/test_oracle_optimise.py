"""Pins for oracle/optimise.py: MMA (Svanberg 1987, one constraint) and the design loop of
Sec. 4.4-4.5."""
import numpy as np
import pytest

import workloads
from oracle import optimise


def test_mma_reaches_the_optimum_of_a_separable_convex_problem():
    """min sum c_j / x_j  s.t. mean(x) <= V, 0.01 <= x <= 1: the optimum (Lagrange condition
    c_j / x_j^2 = const) is x_j = n V sqrt(c_j) / sum_k sqrt(c_k)."""
    rng = np.random.default_rng(1)
    n, V = 20, 0.3
    c = rng.uniform(1.0, 4.0, n)
    x_opt = n * V * np.sqrt(c) / np.sqrt(c).sum()
    assert x_opt.max() < 1.0
    mma = optimise.MMA(n, 0.01, 1.0, s0=0.2)
    x = np.full(n, V)
    for _ in range(100):
        f, df = np.sum(c / x), -c / x ** 2
        g, dg = x.mean() / V - 1.0, np.full(n, 1.0 / (n * V))
        x = mma.step(x, f, df, g, dg)
    assert np.allclose(x, x_opt, rtol=1e-6)
    assert x.mean() <= V * (1 + 1e-9)


def test_mma_approximation_matches_value_and_gradient():
    """f~ built at x equals f(x) and has gradient df there (central differences)."""
    rng = np.random.default_rng(2)
    n = 7
    x = rng.uniform(0.2, 0.8, n)
    low, upp = x - 0.3, x + 0.4
    df = rng.standard_normal(n)
    p, q = optimise.MMA.coefficients(x, low, upp, df)
    assert optimise.MMA.approx(x, x, low, upp, 2.5, p, q) == pytest.approx(2.5, abs=1e-14)
    h = 1e-6
    for j in range(n):
        e = np.zeros(n)
        e[j] = h
        d = (optimise.MMA.approx(x + e, x, low, upp, 2.5, p, q)
             - optimise.MMA.approx(x - e, x, low, upp, 2.5, p, q)) / (2 * h)
        assert d == pytest.approx(df[j], rel=1e-6, abs=1e-8)


@pytest.mark.parametrize("cell", [None, (8, 4)])
def test_volume_constraint_gradient_by_central_differences(cell):
    """g = E[mean(rho_bar)] / v_f - 1 through the projection and filter (three
    realisations), against central differences on seeded design variables."""
    wl = workloads.small(16, 8, seed=3, kind="random", etas=(0.3, 0.5, 0.7), rmin=1.5,
                         beta=4.0, cell=cell)
    rho = wl.rho.copy()
    _, _, g, dg, _ = optimise.robust_objective_and_volume(wl, rho, 0.4)
    rng = np.random.default_rng(4)
    h = 1e-6
    for idx in rng.choice(rho.size, 5, replace=False):
        e = np.zeros(rho.size)
        e[idx] = h
        gp = optimise.robust_objective_and_volume(wl, rho + e.reshape(rho.shape), 0.4)[2]
        gm = optimise.robust_objective_and_volume(wl, rho - e.reshape(rho.shape), 0.4)[2]
        assert (gp - gm) / (2 * h) == pytest.approx(dg.ravel()[idx], rel=1e-5, abs=1e-10)


def test_design_loop_lowers_the_robust_compliance_within_the_volume():
    """Two continuation stages (p 1.5 then 3, beta 4) on a 24x8 MBB beam, three
    realisations: the topology forms in the first stage (the robust compliance falls more
    than threefold), the penalised second stage still lowers it, and the expected-volume
    constraint ends active (satisfied, within 5 %)."""
    wl = workloads.small(24, 8, seed=5, kind="solid", etas=(0.3, 0.5, 0.7), rmin=1.5,
                         beta=4.0, Emin=1e-6)
    wl.rho = np.full_like(wl.rho, 0.5)
    hist = []
    rho = optimise.optimise(wl, 0.5, [(1.5, 4.0, 25), (3.0, 4.0, 25)], history=hist)
    assert rho.min() >= 0.0 and rho.max() <= 1.0
    f1 = [h["f"] for h in hist if h["penal"] == 1.5]
    f2 = [h["f"] for h in hist if h["penal"] == 3.0]
    assert f1[-1] < f1[0] / 3.0
    assert f2[-1] < 0.97 * f2[0]
    assert -0.05 <= hist[-1]["g"] <= 1e-3


def test_robust_verification_compliance_rises_with_the_threshold():
    """A higher threshold eta erodes the projected design pointwise, so the stiffness falls
    in the Loewner order and the compliance f^T K^-1 f rises: monotone over eta in [0.3, 0.7]."""
    wl = workloads.small(24, 8, seed=6, kind="random", rmin=1.5, beta=4.0, Emin=1e-6)
    etas = np.linspace(0.3, 0.7, 21)
    c = optimise.robust_verification(wl, wl.rho, etas)
    assert np.all(np.diff(c) > 0.0)
