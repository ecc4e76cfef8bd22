"""The oracle's Newton direction (Algorithm 1) against the Newton system it solves (CPU only).

Sec. 4.3: Algorithm 1 solves (J_k + mu_k I)[dw] = -R(w_k), with J_k a generalized Jacobian of
R (Eq. 4.2).  Where Z = X - Phi*(gamma) - lambda1 I has no eigenvalue near 0, R is differentiable
and J_k[dw] is its directional derivative.  Central differences of the oracle's own residual()
give that derivative without any of Algorithm 1's algebra (the Schur reduction, T_k, Psi), so a
wrong sign, weight or block in that algebra fails this test.  One point has an X with an
antisymmetric part.  R sees it (X enters r2 directly) and the projection onto S^l_+ does not;
a T_k that acted on the raw argument missed this.
"""
import numpy as np
import pytest

from oracle import kot_oracle as ko
from paper_2310_14087_gb300 import workloads as wl


def _point(seed, antisym):
    p = wl.paper_regime(seed=seed, d=2, n=120, l=40)
    F = ko.build_features(p.X, p.Y, p.Xf, p.Yf, p.sigma, p.lambda1, p.lambda2)
    r = ko.ssn_solve(F, 0.0, ko.Options(max_iter=4))
    X = r.X
    if antisym:
        A = np.random.default_rng(seed).standard_normal(X.shape)
        X = X + antisym * np.linalg.norm(X) * (A - A.T) / np.linalg.norm(A - A.T)
    return F, r.gamma, X


def _system_residual(F, gamma, X, mu):
    res = ko.residual(F, gamma, X)
    sig = res.eig.sig
    assert np.min(np.abs(sig)) > 1e-3 * np.max(np.abs(sig))   # differentiable with room to spare
    d = ko.newton_direction(F, res, mu, ko.Options(), cg_tol_abs=1e-13)
    s = np.linalg.norm(d.dgamma) + np.linalg.norm(d.dX)
    h = 1e-6 / s
    rp = ko.residual(F, gamma + h * d.dgamma, X + h * d.dX)
    rm = ko.residual(F, gamma - h * d.dgamma, X - h * d.dX)
    J1 = (rp.r1 - rm.r1) / (2 * h)
    J2 = (rp.r2 - rm.r2) / (2 * h)
    e1 = J1 + mu * d.dgamma + res.r1
    e2 = J2 + mu * d.dX + res.r2
    return np.linalg.norm(e1), np.linalg.norm(e2), np.linalg.norm(res.r1), np.linalg.norm(res.r2)


@pytest.mark.parametrize("seed,antisym,mu", [(0, 0.0, 1e-1), (4, 0.0, 1e-2), (5, 0.0, 1e-3),
                                              (0, 1e-3, 1e-2), (4, 1e-4, 1e-3)])
def test_direction_solves_the_regularised_newton_system(seed, antisym, mu):
    F, gamma, X = _point(seed, antisym)
    e1, e2, n1, n2 = _system_residual(F, gamma, X, mu)
    scale = n1 + n2
    assert e1 <= 1e-6 * scale
    assert e2 <= 1e-6 * scale
