"""Oracle, part 6: the design loop around the hot path (Sec. 4.4, 4.5): robust compliance
minimisation under a constraint on the expected volume, solved with the method of moving
asymptotes and a continuation schedule on the SIMP exponent and beta.

TEST INFRASTRUCTURE ONLY -- plain FP64 NumPy.

Problem (Sec. 4.4):
    minimise   f(rho) = E[c] + kappa sqrt(Var[c])          over the realisations eta_k
    subject to g(rho) = E[rho_bar^T v] / (v_f e^T v) - 1 <= 0,   0 <= rho <= 1

MMA (Svanberg 1987), one constraint, restated from the published method:
  - moving asymptotes L_j < x_j < U_j; in the first two iterations at x -/+ s0 (x_max - x_min)
    with s0 = 0.5 / (1 + beta) (the paper's initial asymptote size, no external move limits);
    afterwards moved by 0.7 when x_j oscillates, by 1.2 when it moves monotonically
    (distance kept within [0.01, 10] (x_max - x_min) as a safeguard);
  - convex separable approximations of f_i (i = 0 objective, 1 constraint) at x^k:
        f~_i(x) = f_i(x^k) + sum_j p_ij (1/(U_j - x_j) - 1/(U_j - x_j^k))
                           + q_ij (1/(x_j - L_j) - 1/(x_j^k - L_j)),
        p_ij = (U_j - x_j^k)^2 max(df_i/dx_j, 0),  q_ij = (x_j^k - L_j)^2 max(-df_i/dx_j, 0);
    they match f_i and its gradient at x^k;
  - the subproblem min f~_0 s.t. f~_1 <= 0 on alpha <= x <= beta (alpha = max(x_min,
    0.9 L + 0.1 x^k), beta = min(x_max, 0.9 U + 0.1 x^k)) through its dual: for a multiplier
    lam >= 0 each x_j(lam) minimises (P_j/(U_j - x) + Q_j/(x - L_j)), P = p_0 + lam p_1,
    Q = q_0 + lam q_1, i.e. x_j = (L_j sqrt(P_j) + U_j sqrt(Q_j)) / (sqrt(P_j) + sqrt(Q_j))
    clipped to [alpha_j, beta_j]; lam is the root of f~_1(x(lam)) = 0 (decreasing in lam),
    found by bisection, or 0 when f~_1(x(0)) <= 0.
"""
from __future__ import annotations

import numpy as np

from . import pipeline


class MMA:
    """State of the moving asymptotes for one design vector."""

    def __init__(self, n: int, xmin=0.0, xmax=1.0, s0: float = 0.5, asydecr: float = 0.7,
                 asyincr: float = 1.2):
        self.xmin = np.full(n, float(xmin)) if np.isscalar(xmin) else np.asarray(xmin, float)
        self.xmax = np.full(n, float(xmax)) if np.isscalar(xmax) else np.asarray(xmax, float)
        self.s0, self.asydecr, self.asyincr = s0, asydecr, asyincr
        self.k = 0
        self.xold1 = self.xold2 = None
        self.low = self.upp = None

    def asymptotes(self, x: np.ndarray):
        span = self.xmax - self.xmin
        if self.k < 2:
            low, upp = x - self.s0 * span, x + self.s0 * span
        else:
            s = (x - self.xold1) * (self.xold1 - self.xold2)
            gam = np.where(s < 0, self.asydecr, np.where(s > 0, self.asyincr, 1.0))
            low = x - gam * (self.xold1 - self.low)
            upp = x + gam * (self.upp - self.xold1)
            low = np.clip(low, x - 10.0 * span, x - 0.01 * span)
            upp = np.clip(upp, x + 0.01 * span, x + 10.0 * span)
        return low, upp

    @staticmethod
    def coefficients(x, low, upp, df):
        p = (upp - x) ** 2 * np.maximum(df, 0.0)
        q = (x - low) ** 2 * np.maximum(-df, 0.0)
        return p, q

    @staticmethod
    def approx(xt, x, low, upp, fval, p, q):
        """f~(xt) of the approximation built at x."""
        return fval + np.sum(p * (1.0 / (upp - xt) - 1.0 / (upp - x))
                             + q * (1.0 / (xt - low) - 1.0 / (x - low)))

    def step(self, x, f0, df0, g, dg):
        """One MMA iteration: returns the next design."""
        x = np.asarray(x, float)
        low, upp = self.asymptotes(x)
        alpha = np.maximum(self.xmin, 0.9 * low + 0.1 * x)
        beta = np.minimum(self.xmax, 0.9 * upp + 0.1 * x)
        p0, q0 = self.coefficients(x, low, upp, df0)
        p1, q1 = self.coefficients(x, low, upp, dg)

        def x_of(lam):
            P, Q = np.sqrt(p0 + lam * p1), np.sqrt(q0 + lam * q1)
            with np.errstate(divide="ignore", invalid="ignore"):
                xs = np.where(P + Q > 0, (low * P + upp * Q) / (P + Q), x)
            return np.clip(xs, alpha, beta)

        def g_of(lam):
            return self.approx(x_of(lam), x, low, upp, g, p1, q1)

        lam = 0.0
        if g_of(0.0) > 0.0:
            hi = 1.0
            while g_of(hi) > 0.0 and hi < 1e40:
                hi *= 10.0
            lo = 0.0
            for _ in range(200):
                mid = 0.5 * (lo + hi)
                if g_of(mid) > 0.0:
                    lo = mid
                else:
                    hi = mid
                if hi - lo <= 1e-14 * max(hi, 1e-300):
                    break
            lam = hi
        xnew = x_of(lam)
        self.xold2, self.xold1 = self.xold1, x.copy()
        self.low, self.upp = low, upp
        self.k += 1
        return xnew


def robust_objective_and_volume(wl, rho: np.ndarray, volfrac: float, kappa: float = 1.0):
    """f, df/drho (direct state solves), g, dg/drho for the problem of Sec. 4.4, at rho."""
    import copy
    wl = copy.copy(wl)
    wl.rho = np.asarray(rho, float)
    out = pipeline.run(wl, "direct", kappa=kappa)
    _, _, _, chain = pipeline.build(wl)
    n_eta = len(wl.etas)
    # expected projected volume over the design mesh (every element has unit volume)
    n_el = wl.nelx * wl.nely
    vol = np.mean([chain.to_mesh(rb).sum() for rb in out["rho_bar"]]) / n_el
    g = vol / volfrac - 1.0
    dv = [np.full((wl.nely, wl.nelx), 1.0 / (n_el * volfrac))] * n_eta
    dg = chain.backward(rho, dv, np.full(n_eta, 1.0 / n_eta))
    return out["f_robust"], out["dfdrho"], g, dg, out["c"]


def optimise(wl, volfrac: float, stages, kappa: float = 1.0, rel_change: float = 1e-3,
             history: list | None = None):
    """The continuation schedule of Sec. 4.5: ``stages`` is a list of (penal, beta, max
    iterations); a stage ends after its iterations or when the objective's relative change
    falls below rel_change.  The asymptotes restart with 0.5 / (1 + beta) at every stage.
    Returns the final design (design-domain layout)."""
    import copy
    rho = np.asarray(wl.rho, float).copy()
    for penal, beta, iters in stages:
        w = copy.copy(wl)
        w.penal, w.beta = penal, beta
        mma = MMA(rho.size, 0.0, 1.0, s0=0.5 / (1.0 + beta))
        f_prev = None
        for _ in range(iters):
            f, df, g, dg, c = robust_objective_and_volume(w, rho, volfrac, kappa)
            if history is not None:
                history.append({"penal": penal, "beta": beta, "f": f, "g": g, "c": c})
            if f_prev is not None and abs(f - f_prev) <= rel_change * abs(f_prev):
                break
            f_prev = f
            rho = mma.step(rho.ravel(), f, df.ravel(), g, dg.ravel()).reshape(rho.shape)
    return rho


def robust_verification(wl, rho: np.ndarray, etas) -> np.ndarray:
    """Compliance of one design over many thresholds (Sec. 4.4 verifies final designs on
    uniformly distributed eta in [0.3, 0.7]); direct state solves, one realisation each."""
    import copy
    out = []
    for eta in etas:
        w = copy.copy(wl)
        w.rho, w.etas = np.asarray(rho, float), (float(eta),)
        out.append(pipeline.run(w, "direct", with_grad=False)["c"][0])
    return np.array(out)
