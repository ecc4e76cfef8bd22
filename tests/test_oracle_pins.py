"""Pins of the oracle against facts fixed by the paper and by mathematics (CPU only).

Each test checks the oracle against something other than itself: a hand-worked example,
a library routine computing the same quantity another way, a closed form, an invariant,
a finite difference, the explicit Kronecker-form matrices of Lemma 4.4, or an independent
interior-point solve.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.spatial.distance

from oracle import kot_oracle as ko
from tests import independent as ind
from paper_2310_14087_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_sym(rng, l, scale=1.0):
    A = rng.standard_normal((l, l))
    return scale * (A + A.T) / 2


def _small_features(seed=0, l=6, n=30, d=2, sigma=0.3, lambda1=0.05, lambda2=0.2):
    p = wl.paper_regime(seed=seed, d=d, n=n, l=l, sigma2=sigma * sigma)
    return ko.build_features(p.X, p.Y, p.Xf, p.Yf, p.sigma, lambda1, lambda2)


# ---------------------------------------------------------------- features (Sec. 3)
def test_kernel_bandwidth_convention():
    # reading: k(a,b) = exp(-||a-b||^2/(2 sigma^2)); at distance sigma the value is e^{-1/2}
    a = np.array([[0.0, 0.0, 0.0]])
    b = np.array([[0.0, 0.7, 0.0]])
    assert ko.gaussian_kernel(a, b, 0.7)[0, 0] == pytest.approx(math.exp(-0.5), rel=1e-15)
    assert ko.gaussian_kernel(a, a, 0.3)[0, 0] == 1.0


def test_sqdist_matches_scipy():
    rng = np.random.default_rng(1)
    A, B = rng.standard_normal((17, 5)), rng.standard_normal((9, 5))
    ref = scipy.spatial.distance.cdist(A, B, "sqeuclidean")
    np.testing.assert_allclose(ko.sqdist(A, B), ref, rtol=1e-13, atol=1e-13)


def test_hand_worked_features():
    g = json.load(open(os.path.join(GOLDEN, "hand_features.json")))
    i = g["inputs"]
    F = ko.build_features(np.array(i["X"]), np.array(i["Y"]), np.array(i["Xf"]),
                          np.array(i["Yf"]), i["sigma"], i["lambda1"], i["lambda2"])
    for key in ("w_mu", "w_nu", "Q", "c", "z", "K"):
        np.testing.assert_allclose(getattr(F, key), np.array(g[key]), rtol=1e-15, atol=1e-15)
    assert F.q2 == pytest.approx(g["q2"], rel=1e-15)


def test_embedding_two_point_closed_form():
    # ||w||^2 = (1/n^2) sum_ij k(s_i, s_j) = (2 + 2 k(a,b))/4 for two samples
    a, b = np.array([0.1, 0.2]), np.array([0.4, -0.3])
    S = np.stack([a, b])
    kab = math.exp(-np.sum((a - b) ** 2) / (2 * 0.5 ** 2))
    assert ko.embedding_sqnorm(S, 0.5) == pytest.approx((2 + 2 * kab) / 4, rel=1e-14)
    # mean embedding of identical samples is the kernel at that sample
    P = np.array([[1.0, 1.0], [0.0, 0.5]])
    S2 = np.stack([a, a, a])
    expect = [math.exp(-np.sum((a - p) ** 2) / (2 * 0.5 ** 2)) for p in P]
    np.testing.assert_allclose(ko.kernel_mean_embedding(S2, P, 0.5), expect, rtol=1e-14)


def test_features_translation_and_scale_invariance():
    p = wl.paper_regime(seed=4, d=3, n=40, l=9, sigma2=0.05)
    F0 = ko.build_features(p.X, p.Y, p.Xf, p.Yf, p.sigma, 0.1, 0.3)
    t = np.array([0.3, -2.0, 5.0])
    F1 = ko.build_features(p.X + t, p.Y + t, p.Xf + t, p.Yf + t, p.sigma, 0.1, 0.3)
    s = 3.5
    F2 = ko.build_features(s * p.X, s * p.Y, s * p.Xf, s * p.Yf, s * p.sigma, 0.1, 0.3)
    for F in (F1, F2):
        for key in ("Q", "K", "w_mu", "w_nu"):
            np.testing.assert_allclose(getattr(F, key), getattr(F0, key), rtol=1e-11, atol=1e-13)
        assert F.q2 == pytest.approx(F0.q2, rel=1e-12)
    np.testing.assert_allclose(F1.z, F0.z, rtol=1e-11, atol=1e-12)   # c depends on xf - yf only


def test_cholesky_factor_properties():
    F = _small_features(l=12, sigma=0.5)
    assert np.allclose(np.tril(F.R, -1), 0.0)
    assert np.all(np.diag(F.R) > 0)
    np.testing.assert_allclose(F.R.T @ F.R, F.K + F.eps * np.eye(F.l), rtol=1e-12, atol=1e-13)
    assert F.eps == pytest.approx(1e-10 * np.max(np.diag(F.K)))
    # the factor agrees with scipy's upper Cholesky of the same matrix
    np.testing.assert_allclose(F.R, scipy.linalg.cholesky(F.K + F.eps * np.eye(F.l), lower=False),
                               rtol=1e-12, atol=1e-13)


def test_cholesky_jitter_escalates_then_fails():
    K = np.array([[1.0, 1.0], [1.0, 1.0]]) - 1e-9 * np.eye(2)   # slightly indefinite
    R, eps = ko.cholesky_upper_jittered(K, 1e-10, 1e-6)
    assert eps == pytest.approx(1e-8)                         # 1e-10, 1e-9 fail; 1e-8 works
    with pytest.raises(np.linalg.LinAlgError):
        ko.cholesky_upper_jittered(-np.eye(2), 1e-10, 1e-6)


# ---------------------------------------------------------------- operators (Sec. 4.1)
def test_phi_adjoint_and_basis():
    rng = np.random.default_rng(2)
    F = _small_features(l=7)
    X = _rand_sym(rng, F.l)
    g = rng.standard_normal(F.l)
    assert ko.phi(F.R, X) @ g == pytest.approx(np.sum(X * ko.phi_star(F.R, g)), rel=1e-12)
    for i in range(F.l):
        e = np.zeros(F.l); e[i] = 1.0
        np.testing.assert_allclose(ko.phi_star(F.R, e), np.outer(F.R[:, i], F.R[:, i]), atol=1e-15)
    # Phi(I)_i = ||Phi_i||^2 = (K + eps I)_ii
    np.testing.assert_allclose(ko.phi(F.R, np.eye(F.l)), np.diag(F.K) + F.eps, rtol=1e-13)


# ---------------------------------------------------------------- projection (Eq. (4.4))
def test_projection_matches_matrix_absolute_value():
    rng = np.random.default_rng(3)
    Z = _rand_sym(rng, 9)
    absZ = np.real(scipy.linalg.sqrtm(Z @ Z))
    np.testing.assert_allclose(ko.proj_psd(Z), (Z + absZ) / 2, atol=1e-10)
    P = ko.proj_psd(Z)
    N = Z - P
    assert np.linalg.eigvalsh(P).min() > -1e-12            # PSD
    assert np.linalg.eigvalsh(N).max() < 1e-12             # remainder NSD
    assert abs(np.sum(P * N)) < 1e-10                      # Moreau orthogonality
    np.testing.assert_allclose(ko.proj_psd(P), P, atol=1e-12)


def test_jacobian_of_projection_is_directional_derivative():
    # Daleckii-Krein: at Z without zero eigenvalues M(Z)[S] is the derivative of Pi_{S+}
    rng = np.random.default_rng(4)
    l = 6
    Pq, _ = np.linalg.qr(rng.standard_normal((l, l)))
    sig = np.array([-2.0, -0.7, -0.1, 0.3, 1.1, 2.5])
    Z = Pq @ np.diag(sig) @ Pq.T
    S = _rand_sym(rng, l)
    h = 1e-6
    fd = (ko.proj_psd(Z + h * S) - ko.proj_psd(Z - h * S)) / (2 * h)
    np.testing.assert_allclose(ko.jacobian_proj_apply(ko.eig_sym(Z), S), fd, atol=1e-8)


def test_T_equals_kronecker_form_and_schur_identities():
    rng = np.random.default_rng(5)
    l = 4
    Z = _rand_sym(rng, l)
    e = ko.eig_sym(Z)
    assert 0 < e.alpha.sum() < l
    mu = 0.37
    W, D, Tk = ind.kron_operators(e.P, e.sig, mu)
    S = _rand_sym(rng, l)
    np.testing.assert_allclose(ko.t_apply(e, ko.psi_matrix(e.sig, mu), S),
                               ind.unvec(Tk @ ind.vec(S), l), atol=1e-12)
    n2 = l * l
    # Lemma 4.4 proof: D^{-1} = (I + T)/(mu + 1) and D^{-1} W = T
    np.testing.assert_allclose(np.linalg.inv(D), (np.eye(n2) + Tk) / (mu + 1), atol=1e-12)
    np.testing.assert_allclose(np.linalg.solve(D, W), Tk, atol=1e-12)


@pytest.mark.parametrize("n_pos", [1, 3, 6])
def test_T_cost_reduced_forms_equal_dense(n_pos):
    # Sec. 4.3: G + G^T with U = P_a^T S (|alpha| small) and the complement form (|alpha| large)
    rng = np.random.default_rng(6 + n_pos)
    l = 8
    Pq, _ = np.linalg.qr(rng.standard_normal((l, l)))
    sig = np.sort(rng.uniform(0.1, 2.0, l))
    sig[: l - n_pos] *= -1
    sig = np.sort(sig)
    e = ko.Eig(P=Pq, sig=sig)
    mu = 0.05
    S = _rand_sym(rng, l)
    Psi = ko.psi_matrix(sig, mu)
    dense = ko.t_apply(e, Psi, S)
    a = sig > 0
    Pa, Pb = Pq[:, a], Pq[:, ~a]
    xi = Psi[np.ix_(a, ~a)]
    U = Pa.T @ S
    G = Pa @ ((1 / (2 * mu)) * (U @ Pa) @ Pa.T + (xi * (U @ Pb)) @ Pb.T)
    np.testing.assert_allclose(G + G.T, dense, atol=1e-10)
    comp = S / mu - Pq @ ((1 / mu - Psi) * (Pq.T @ S @ Pq)) @ Pq.T
    np.testing.assert_allclose(comp, dense, atol=1e-9)


# ---------------------------------------------------------------- Newton step (Alg. 1)
def _point(F, rng):
    A = rng.standard_normal((F.l, F.l))
    return rng.standard_normal(F.l), A @ A.T / F.l


def test_residual_jacobian_matches_finite_differences():
    rng = np.random.default_rng(7)
    F = _small_features(l=6)
    g, X = _point(F, rng)
    res = ko.residual(F, g, X)
    dg, dX = rng.standard_normal(F.l), _rand_sym(rng, F.l)
    h = 1e-6
    rp, rm = ko.residual(F, g + h * dg, X + h * dX), ko.residual(F, g - h * dg, X - h * dX)
    J1 = F.Q @ dg / (2 * F.lambda2) - ko.phi(F.R, dX)
    J2 = dX - ko.jacobian_proj_apply(res.eig, dX - ko.phi_star(F.R, dg))
    np.testing.assert_allclose(J1, (rp.r1 - rm.r1) / (2 * h), atol=1e-6)
    np.testing.assert_allclose(J2, (rp.r2 - rm.r2) / (2 * h), atol=1e-6)


@pytest.mark.parametrize("mu", [1e-3, 0.2, 3.0])
def test_algorithm1_equals_dense_newton_system(mu):
    rng = np.random.default_rng(8)
    F = _small_features(l=5)
    g, X = _point(F, rng)
    res = ko.residual(F, g, X)
    d = ko.newton_direction(F, res, mu, ko.Options(), cg_tol_abs=1e-12)
    dg, dX = ind.dense_newton(F.Q, F.R, F.lambda2, res.eig.P, res.eig.sig, mu, res.r1, res.r2)
    np.testing.assert_allclose(d.dgamma, dg, rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(d.dX, dX, rtol=1e-8, atol=1e-10)


@pytest.mark.parametrize("mu", [0.05, 1.0])
def test_sqmr_direction_equals_dense_newton_system(mu):
    # the symmetric QMR option (Sec. 4.3 names CG or symmetric QMR) solves the same Schur system:
    # run to a tight tolerance it must give the direction of the dense (l + l^2) Newton solve, and
    # the true residual it carries must equal a1 - H x recomputed
    F = _small_features(l=5)
    rng = np.random.default_rng(4)
    g, X = _point(F, rng)
    res = ko.residual(F, g, 0.05 * X)
    dg, dX = ind.dense_newton(F.Q, F.R, F.lambda2, res.eig.P, res.eig.sig, mu, res.r1, res.r2)
    d = ko.newton_direction(F, res, mu, ko.Options(schur_solver=1), cg_tol_abs=1e-13)
    np.testing.assert_allclose(d.dgamma, dg, atol=1e-9 * max(1.0, np.abs(dg).max()))
    np.testing.assert_allclose(d.dX, dX, atol=1e-9 * max(1.0, np.abs(dX).max()))
    # inexact: the carried residual is the true residual of the returned iterate
    d = ko.newton_direction(F, res, mu, ko.Options(schur_solver=1, cg_max_iter=3), cg_tol_abs=1e-30)
    Psi = ko.psi_matrix(res.eig.sig, mu)
    T = lambda S: ko.t_apply(res.eig, Psi, S)
    a1 = -res.r1 - ko.phi(F.R, res.r2 + T(res.r2)) / (mu + 1.0)
    H = F.Q @ d.dgamma / (2 * F.lambda2) + mu * d.dgamma + ko.phi(F.R, T(ko.phi_star(F.R, d.dgamma)))
    assert d.cg_res == pytest.approx(np.linalg.norm(a1 - H), rel=1e-8)


def test_inexact_cg_residual_is_full_system_residual():
    rng = np.random.default_rng(9)
    F = _small_features(l=6)
    g, X = _point(F, rng)
    res = ko.residual(F, g, X)
    mu = 0.1
    opt = ko.Options(cg_max_iter=2)
    d = ko.newton_direction(F, res, mu, opt)
    M = lambda S: ko.jacobian_proj_apply(res.eig, S)
    e1 = F.Q @ d.dgamma / (2 * F.lambda2) - ko.phi(F.R, d.dX) + mu * d.dgamma + res.r1
    e2 = d.dX - M(d.dX - ko.phi_star(F.R, d.dgamma)) + mu * d.dX + res.r2
    assert np.linalg.norm(e2) < 1e-10 * max(1.0, np.linalg.norm(res.r2))
    assert np.linalg.norm(e1) == pytest.approx(d.cg_res, rel=1e-6)


# ---------------------------------------------------------------- Algorithm 2, closed forms
def _features_direct(Q, z, R, lambda1, lambda2, q2=1.0):
    l = Q.shape[0]
    return ko.Features(Q=Q, z=z, q2=q2, K=R.T @ R, R=R, w_mu=np.zeros(l), w_nu=np.zeros(l),
                       c=np.zeros(l), eps=0.0, lambda1=lambda1, lambda2=lambda2)


@pytest.mark.parametrize("z1", [0.3, -0.5])
def test_l1_closed_form(z1):
    # l = 1: min a g^2 - b g s.t. g R11^2 + lambda1 >= 0, a = Q11/(4 l2), b = z1/(2 l2)
    Q, R, lam1, lam2 = np.array([[1.7]]), np.array([[0.8]]), 0.05, 0.1
    F = _features_direct(Q, np.array([z1]), R, lam1, lam2)
    r = ko.ssn_solve(F, 1e-10, ko.Options(max_iter=400))
    a, b = Q[0, 0] / (4 * lam2), z1 / (2 * lam2)
    assert r.converged
    assert r.gamma[0] == pytest.approx(max(b / (2 * a), -lam1 / R[0, 0] ** 2), abs=1e-9)


def test_separable_closed_form():
    # Q = q I, R = I: each coordinate is an l = 1 problem, gamma_i = max(z_i/q, -lambda1)
    rng = np.random.default_rng(10)
    l, q, lam1, lam2 = 12, 2.0, 0.05, 0.1
    z = rng.uniform(-0.5, 0.5, l)
    F = _features_direct(q * np.eye(l), z, np.eye(l), lam1, lam2)
    r = ko.ssn_solve(F, 1e-10, ko.Options(max_iter=400))
    assert r.converged
    np.testing.assert_allclose(r.gamma, np.maximum(z / q, -lam1), atol=1e-9)
    # X from r1 = 0: X_ii = (q gamma_i - z_i)/(2 lambda2), zero off the diagonal
    np.testing.assert_allclose(np.diag(r.X), (q * r.gamma - z) / (2 * lam2), atol=1e-8)


def test_inactive_constraint_closed_form():
    # if lambda1 > -lambda_min(Phi*(Q^{-1} z)) the constraint is slack: gamma = Q^{-1} z, X = 0
    F0 = _small_features(l=6)
    g_free = np.linalg.solve(F0.Q, F0.z)
    lam1 = 1.5 * max(1e-3, -np.linalg.eigvalsh(ko.phi_star(F0.R, g_free)).min())
    F = _features_direct(F0.Q, F0.z, F0.R, lam1, F0.lambda2)
    r = ko.ssn_solve(F, 1e-11, ko.Options(max_iter=100))
    assert r.converged
    np.testing.assert_allclose(r.gamma, g_free, rtol=1e-8, atol=1e-10)
    assert np.abs(r.X).max() < 1e-9


@pytest.mark.parametrize("seed,l", [(0, 4), (0, 8), (1, 10), (3, 8)])
def test_matches_independent_interior_point(seed, l):
    F = _small_features(seed=seed, l=l, sigma=0.35)
    r = ko.ssn_solve(F, 1e-10, ko.Options(max_iter=500))
    assert r.converged
    g, _ = ind.ipm_solve(F.Q, F.z, F.q2, F.R, F.lambda1, F.lambda2)
    f_ipm = ko.objective(F, g)
    assert r.objective == pytest.approx(f_ipm, rel=1e-8, abs=1e-10)
    np.testing.assert_allclose(r.gamma, g, rtol=1e-4, atol=1e-5)


def test_kkt_invariants_at_solution():
    # Prop. 4.1 and its proof: R(w) = 0 iff X >= 0, S = Phi*(gamma) + lambda1 I >= 0,
    # <X, S> = 0 and r1 = 0; at ||R(w)|| <= tol each holds up to O(tol)
    tol = 1e-6
    p = wl.paper_regime(seed=2, d=2, n=100, l=50)
    F = ko.build_features(p.X, p.Y, p.Xf, p.Yf, p.sigma, p.lambda1, p.lambda2)
    r = ko.ssn_solve(F, tol, ko.Options())
    assert r.converged
    S = ko.phi_star(F.R, r.gamma) + F.lambda1 * np.eye(F.l)
    scale = 1.0 + np.linalg.norm(r.X) + np.linalg.norm(S)
    assert np.linalg.eigvalsh(r.X).min() > -tol
    assert np.linalg.eigvalsh(S).min() > -tol
    assert abs(np.sum(r.X * S)) < 10 * tol * scale
    r1 = (F.Q @ r.gamma - F.z) / (2 * F.lambda2) - ko.phi(F.R, r.X)
    assert np.linalg.norm(r1) <= tol


def test_primal_dual_gap_closes_at_solution():
    # Lagrangian of Eq. (3.3) with multiplier X for the PSD constraint: minimising over gamma
    # (Q > 0) gives the dual function g(X) = q^2/(4 l2) - l1 tr X - b^T Q^-1 b/(4 l2),
    # b = z + 2 l2 Phi(X); weak duality f(gamma) >= g(X) holds for every X >= 0, and at a
    # solution (R(w) = 0) the gap f - g = <X, Phi*(gamma) + l1 I> closes (strong duality)
    F = _small_features(seed=0, l=8, sigma=0.35)
    r = ko.ssn_solve(F, 1e-10, ko.Options(max_iter=500))
    assert r.converged

    def g_dual(X):
        b = F.z + 2 * F.lambda2 * ko.phi(F.R, X)
        return F.q2 / (4 * F.lambda2) - F.lambda1 * np.trace(X) - b @ np.linalg.solve(F.Q, b) / (4 * F.lambda2)

    f = ko.objective(F, r.gamma)
    assert f - g_dual(r.X) == pytest.approx(0.0, abs=1e-8 * max(1.0, abs(f)))
    # weak duality at other PSD points (the dual function lies below the primal optimum)
    rng = np.random.default_rng(3)
    for _ in range(5):
        A = rng.standard_normal((F.l, F.l))
        assert g_dual(0.1 * A @ A.T) <= f + 1e-10


def test_golden_algorithm_constants():
    g = json.load(open(os.path.join(GOLDEN, "algorithm_constants.json")))
    o = ko.Options()
    for key in ("alpha1", "alpha2", "beta0", "beta1", "beta2", "cg_max_iter"):
        assert getattr(o, key) == g[key], key


def test_eg_operator_is_the_lagrangian_gradient():
    # F(gamma, X) = (grad_gamma L, -grad_X L) for the min-max objective L of Eq. (4.1):
    # L = gamma^T Q gamma/(4 lambda2) - gamma^T z/(2 lambda2) + q^2/(4 lambda2)
    #     - <X, Phi*(gamma) + lambda1 I>.
    # Central differences of L along random directions give both blocks of F.
    rng = np.random.default_rng(12)
    F = _small_features(l=7)

    def L(g, X):
        S = (F.R * g[None, :]) @ F.R.T + F.lambda1 * np.eye(F.l)
        return (g @ F.Q @ g / (4 * F.lambda2) - g @ F.z / (2 * F.lambda2) + F.q2 / (4 * F.lambda2)
                - np.sum(X * S))

    g, X = _point(F, rng)
    Fg, FX = ko.eg_operator(F, g, X)
    h = 1e-6
    for _ in range(3):
        dg, dX = rng.standard_normal(F.l), _rand_sym(rng, F.l)
        dLg = (L(g + h * dg, X) - L(g - h * dg, X)) / (2 * h)
        dLX = (L(g, X + h * dX) - L(g, X - h * dX)) / (2 * h)
        assert Fg @ dg == pytest.approx(dLg, rel=1e-7, abs=1e-9)
        assert -np.sum(FX * dX) == pytest.approx(dLX, rel=1e-7, abs=1e-9)


def test_eg_step_size_bounds_operator_norm():
    # eta = 1/L must not exceed 1/||linear part||; compute that norm by dense SVD
    F = _small_features(l=5)
    A = np.stack([np.kron(F.R[:, i], F.R[:, i]) for i in range(F.l)])
    l2 = F.l * F.l
    M = np.block([[F.Q / (2 * F.lambda2), -A], [A.T, np.zeros((l2, l2))]])
    assert ko.eg_lipschitz(F) >= np.linalg.norm(M, 2) * (1 - 1e-12)


def test_eg_is_monotone_descent_of_residual_on_average():
    # pure EG (Appendix F) converges, slowly, on a small problem
    F = _small_features(l=5)
    r0 = ko.residual(F, np.zeros(F.l), np.zeros((F.l, F.l))).norm
    r = ko.eg_solve(F, 1e-12, 400)
    assert r.residual < 0.5 * r0


def test_eg_step_l1_is_scalar_projected_extragradient():
    # l = 1 (R = [r], Q = [q]): the min-max operator is F(g, x) = ((q g - z)/(2 l2) - r^2 x,
    # r^2 g + l1) on R x [0, inf), so one Korpelevich step is scalar projected gradient twice
    q, r, z, l1, l2, eta = 1.7, 0.8, 0.3, 0.05, 0.1, 0.07
    F = _features_direct(np.array([[q]]), np.array([z]), np.array([[r]]), l1, l2)
    g0, x0 = -0.4, 0.9
    Fg = lambda g, x: (q * g - z) / (2 * l2) - r * r * x
    Fx = lambda g, x: r * r * g + l1
    gh, xh = g0 - eta * Fg(g0, x0), max(0.0, x0 - eta * Fx(g0, x0))
    g1, x1 = g0 - eta * Fg(gh, xh), max(0.0, x0 - eta * Fx(gh, xh))
    gn, Xn = ko.eg_step(F, np.array([g0]), np.array([[x0]]), eta)
    assert gn[0] == pytest.approx(g1, rel=1e-14)
    assert Xn[0, 0] == pytest.approx(x1, rel=1e-14)


def test_eg_step_fixes_a_solution():
    # a solution w* of the variational inequality of Eq. (4.1) (R(w*) = 0) is a fixed point of
    # the projected extragradient map for every step size
    F = _small_features(l=6)
    r = ko.ssn_solve(F, 1e-12, ko.Options(max_iter=500))
    assert r.converged
    for eta in (1e-3, 0.5 / ko.eg_lipschitz(F)):
        g1, X1 = ko.eg_step(F, r.gamma, r.X, eta)
        np.testing.assert_allclose(g1, r.gamma, atol=1e-9)
        np.testing.assert_allclose(X1, r.X, atol=1e-9)


def test_rejected_steps_reach_the_same_optimum():
    # Algorithm 2's acceptance test: with theta0 = 1e4 the first Newton steps are short and the
    # extragradient iterate wins several times; without the safeguard every Newton step is taken.
    # The optimum is unique (the objective is strongly convex in gamma), so all three runs must
    # agree on it to the accuracy a residual of 1e-6 gives (runs stopped at 1e-6 differ from the
    # optimum by up to ~2e-5 in f on these problems), and the counts must add up.
    p = wl.paper_regime(seed=2, d=2, n=100, l=50)
    F = ko.build_features(p.X, p.Y, p.Xf, p.Yf, p.sigma, p.lambda1, p.lambda2)
    base = ko.ssn_solve(F, 1e-6)
    slow = ko.ssn_solve(F, 1e-6, ko.Options(theta0=1e4))
    plain = ko.ssn_solve(F, 1e-6, ko.Options(use_eg=False))
    assert base.converged and slow.converged and plain.converged
    assert slow.eg_taken >= 1 and slow.ssn_accepted + slow.eg_taken == slow.iters
    assert plain.eg_taken == 0 and plain.ssn_accepted == plain.iters
    for r in (slow, plain):
        assert r.objective == pytest.approx(base.objective, rel=1e-4)
        np.testing.assert_allclose(r.gamma, base.gamma, atol=1e-3 * np.abs(base.gamma).max())


def test_potentials_reproduce_the_estimator():
    # <u, w_mu>_H = (1/n) sum_j u(x_j) (reproducing property), so averaging the potentials over
    # the samples must give OT-hat = q^2/(2 l2) - sum_i gamma_i (w_mu(xf_i) + w_nu(yf_i))/(2 l2)
    # as the paper prints it (Sec. 3), for any gamma
    p = wl.paper_regime(seed=4, d=3, n=40, l=12)
    F = ko.build_features(p.X, p.Y, p.Xf, p.Yf, p.sigma, p.lambda1, p.lambda2)
    gamma = np.random.default_rng(3).standard_normal(F.l)
    u, _, _ = ko.potential(p.X, p.Xf, gamma, p.sigma, p.lambda2, p.X)
    v, _, _ = ko.potential(p.Y, p.Yf, gamma, p.sigma, p.lambda2, p.Y)
    assert u.mean() + v.mean() == pytest.approx(ko.ot_estimate(F, gamma), rel=1e-12)


def test_potential_gradient_and_map():
    p = wl.paper_regime(seed=5, d=4, n=30, l=10)
    gamma = np.random.default_rng(1).standard_normal(p.l)
    P = np.random.default_rng(2).uniform(0.0, 1.0, (7, 4))
    u, grad, T = ko.potential(p.X, p.Xf, gamma, p.sigma, p.lambda2, P)
    h = 1e-6
    for k in range(4):
        e = np.zeros(4); e[k] = h
        up, _, _ = ko.potential(p.X, p.Xf, gamma, p.sigma, p.lambda2, P + e)
        um, _, _ = ko.potential(p.X, p.Xf, gamma, p.sigma, p.lambda2, P - e)
        np.testing.assert_allclose(grad[:, k], (up - um) / (2 * h), rtol=1e-6, atol=1e-6 * np.abs(grad).max())
    np.testing.assert_allclose(T, P - grad, rtol=0, atol=0)
    # gamma = 0: u is the kernel mean embedding of mu-hat over 2 lambda2
    u0, _, _ = ko.potential(p.X, p.Xf, np.zeros(p.l), p.sigma, p.lambda2, P)
    emb = np.exp(-scipy.spatial.distance.cdist(P, p.X, "sqeuclidean") / (2 * p.sigma ** 2)).mean(axis=1)
    np.testing.assert_allclose(u0, emb / (2 * p.lambda2), rtol=1e-13)


def test_estimator_near_closed_form_gaussian_w2():
    # loose statistical sanity check (not a parity gate): for mu = N(0, I_2), nu = N((1,1),
    # diag(0.5, 2)) the estimator targets W2^2/2 = (|m1 - m2|^2 + tr(S1 + S2 - 2 (S2^1/2 S1
    # S2^1/2)^1/2))/2 = (2 + (1 - sqrt .5)^2 + (1 - sqrt 2)^2)/2 = 1.1287; with the paper's
    # lambda2 = 1/sqrt(n) (Sec. 3 remark) at n = 100, l = 50 the estimate at the optimum (taken
    # from the independent interior-point solve) lands within a factor 1.5 of it
    half_w2 = 0.5 * (2.0 + (1 - math.sqrt(0.5)) ** 2 + (1 - math.sqrt(2.0)) ** 2)
    p = wl.gaussian_pair(n=100, l=50, lambda2=0.1, lambda1=1e-3)
    F = ko.build_features(p.X, p.Y, p.Xf, p.Yf, p.sigma, p.lambda1, p.lambda2)
    g, _ = ind.ipm_solve(F.Q, F.z, F.q2, F.R, F.lambda1, F.lambda2)
    est = ko.ot_estimate(F, g)
    assert half_w2 / 1.5 < est < 1.5 * half_w2


# ---------------------------------------------------------------- planted mistakes
def test_planted_mistakes_are_caught(monkeypatch):
    """Each mutation reproduces a plausible slip; the pin named beside it must reject it."""
    F = _small_features(l=5)
    rng = np.random.default_rng(11)
    g, X = _point(F, rng)
    X = 0.05 * X
    res = ko.residual(F, g, X)
    assert 0 < res.eig.alpha.sum() < F.l          # both blocks of Omega are present
    mu = 0.2
    good = ko.newton_direction(F, res, mu, ko.Options(), cg_tol_abs=1e-12)
    dg, dX = ind.dense_newton(F.Q, F.R, F.lambda2, res.eig.P, res.eig.sig, mu, res.r1, res.r2)
    assert np.allclose(good.dgamma, dg, atol=1e-9)

    # eta_ij = sig_j/(sig_i - sig_j) instead of sig_i/(sig_i - sig_j)
    orig = ko.omega_matrix

    def bad_omega(sig):
        Om = orig(sig)
        a = sig > 0
        for i in np.where(a)[0]:
            for j in np.where(~a)[0]:
                Om[i, j] = Om[j, i] = -sig[j] / (sig[i] - sig[j])
        return Om
    monkeypatch.setattr(ko, "omega_matrix", bad_omega)
    bad = ko.newton_direction(F, res, mu, ko.Options(), cg_tol_abs=1e-12)
    assert not np.allclose(bad.dgamma, dg, atol=1e-6)
    monkeypatch.setattr(ko, "omega_matrix", orig)

    # transposed Cholesky factor in Phi* (R^T diag R instead of R diag R^T)
    monkeypatch.setattr(ko, "phi_star", lambda R, gam: (R.T * gam[None, :]) @ R)
    e = np.zeros(F.l); e[2] = 1.0
    assert not np.allclose(ko.phi_star(F.R, e), np.outer(F.R[:, 2], F.R[:, 2]), atol=1e-12)
