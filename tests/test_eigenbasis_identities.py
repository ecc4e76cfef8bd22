"""Identities behind the eigenbasis form of Algorithm 1 that the CUDA path computes (CPU only).

With Z = P diag(sig) P^T (alpha-bar = {sig <= 0} first), Cb = P^T R and Psi of Sec. 4.3, the CUDA
path applies the Schur operator of the Newton system as
    Phi(T[Phi*(p)]) = 2 diag(Cb_alpha^T W Cb),  W = alpha rows of Psi o (Cb diag(p) Cb^T) with the
    alpha x alpha block halved,
carries T[Phi*(x)] = P (W-full) P^T through W, measures ||at2 - T[Phi*(x)]||_F in the eigenbasis,
and forms the right-hand side and the direction there:
    A2 = P^T at2 P = -(1 + Psi) o (P^T r2 P)/(mu + 1),  a1 = -r1 + diag(Cb^T A2 Cb),
    dX = P (A2 - P^T T[Phi*(x)] P) P^T.
Each is checked here against the oracle's own phi_star / t_apply / phi on random data, including
the degenerate splits alpha = {} and alpha-bar = {} (a wrong halving, weight or sign fails).
"""
import numpy as np
import pytest

from oracle import kot_oracle as ko

SPLITS = [(7, 3), (9, 6), (8, 0), (8, 8), (12, 1), (12, 11)]


def _problem(seed, l, npos):
    rng = np.random.default_rng(seed)
    R = np.triu(rng.standard_normal((l, l)))
    P, _ = np.linalg.qr(rng.standard_normal((l, l)))
    sig = np.concatenate([-rng.random(l - npos) - 0.1, rng.random(npos) + 0.1])
    return rng, R, P, sig


def _row_weights(sig, nb, mu):
    """Weights of the alpha rows (G + G^T form): 1/(2 mu) on alpha columns, xi on alpha-bar."""
    l = sig.size
    Wt = np.empty((l - nb, l))
    for r in range(l - nb):
        i = nb + r
        for j in range(l):
            if j >= nb:
                Wt[r, j] = 0.5 / mu
            else:
                eta = sig[i] / (sig[i] - sig[j])
                Wt[r, j] = eta / (mu + 1.0 - eta)
    return Wt


def _full_from_rows(W, nb, l):
    """P^T T P from its alpha rows W (alpha x alpha halved)."""
    F = np.zeros((l, l))
    F[nb:, :nb] = W[:, :nb]
    F[:nb, nb:] = W[:, :nb].T
    F[nb:, nb:] = 2.0 * W[:, nb:]
    return F


@pytest.mark.parametrize("l,npos", SPLITS)
def test_operator_in_eigenbasis(l, npos):
    mu = 0.37
    rng, R, P, sig = _problem(3 + l + npos, l, npos)
    e = ko.Eig(P=P, sig=sig)
    Psi = ko.psi_matrix(sig, mu)
    nb = l - npos
    p = rng.standard_normal(l)
    T_ref = ko.t_apply(e, Psi, ko.phi_star(R, p))
    H_ref = ko.phi(R, T_ref)
    Cb = P.T @ R
    W = ((Cb[nb:] * p[None, :]) @ Cb.T) * _row_weights(sig, nb, mu)
    H = 2.0 * np.sum(Cb[nb:] * (W @ Cb), axis=0)
    scale = max(1.0, np.max(np.abs(H_ref)))
    assert np.max(np.abs(H - H_ref)) <= 1e-12 * scale
    T = P @ _full_from_rows(W, nb, l) @ P.T
    assert np.max(np.abs(T - T_ref)) <= 1e-12 * max(1.0, np.max(np.abs(T_ref)))
    # the G + G^T reconstruction the direction used before it moved to P D P^T
    G = P[:, nb:] @ W @ P.T
    assert np.max(np.abs(G + G.T - T_ref)) <= 1e-12 * max(1.0, np.max(np.abs(T_ref)))


@pytest.mark.parametrize("l,npos", SPLITS)
def test_stopping_norm_in_eigenbasis(l, npos):
    mu = 0.37
    rng, R, P, sig = _problem(11 + l + npos, l, npos)
    e = ko.Eig(P=P, sig=sig)
    Psi = ko.psi_matrix(sig, mu)
    nb = l - npos
    x = rng.standard_normal(l)
    at2 = rng.standard_normal((l, l))
    at2 = at2 + at2.T
    ref = np.sum((at2 - ko.t_apply(e, Psi, ko.phi_star(R, x))) ** 2)
    Cb = P.T @ R
    Wx = ((Cb[nb:] * x[None, :]) @ Cb.T) * _row_weights(sig, nb, mu)
    A2 = P.T @ at2 @ P
    cbb = np.sum(A2[:nb, :nb] ** 2)
    j = np.arange(l)
    w = np.where(j < nb, 2.0, 1.0)
    c = np.where(j < nb, 1.0, 2.0)
    got = cbb + np.sum(w[None, :] * (A2[nb:] - c[None, :] * Wx) ** 2)
    assert abs(got - ref) <= 1e-12 * ref


@pytest.mark.parametrize("l,npos", SPLITS)
def test_rhs_and_direction_in_eigenbasis(l, npos):
    mu = 0.29
    rng, R, P, sig = _problem(23 + l + npos, l, npos)
    e = ko.Eig(P=P, sig=sig)
    Psi = ko.psi_matrix(sig, mu)
    nb = l - npos
    r1 = rng.standard_normal(l)
    r2 = rng.standard_normal((l, l))
    r2 = r2 + r2.T

    def T(S):
        return ko.t_apply(e, Psi, S)

    a1_ref = -r1 - ko.phi(R, r2 + T(r2)) / (mu + 1.0)
    at2_ref = (-r2 + T(-r2)) / (mu + 1.0)
    Cb = P.T @ R
    A2 = -(1.0 + Psi) * (P.T @ r2 @ P) / (mu + 1.0)
    assert np.max(np.abs(P @ A2 @ P.T - at2_ref)) <= 1e-12 * np.max(np.abs(at2_ref))
    a1 = -r1 + np.sum(Cb * (A2 @ Cb), axis=0)
    assert np.max(np.abs(a1 - a1_ref)) <= 1e-12 * max(1.0, np.max(np.abs(a1_ref)))
    x = rng.standard_normal(l)
    Wx = ((Cb[nb:] * x[None, :]) @ Cb.T) * _row_weights(sig, nb, mu)
    dX = P @ (A2 - _full_from_rows(Wx, nb, l)) @ P.T
    dX_ref = at2_ref - T(ko.phi_star(R, x))
    assert np.max(np.abs(dX - dX_ref)) <= 1e-12 * max(1.0, np.max(np.abs(dX_ref)))


# ---- complement form (|alpha| > |alpha-bar|, Sec. 4.3, last paragraph) -------------------------
# With Psi' = E/mu - Psi (zero on alpha x alpha), Psi o V = V/mu - Psi' o V, and for orthogonal P
# diag(Cb^T V Cb) = (Kt o Kt) p with Kt = R^T R, V = Cb diag(p) Cb^T.  So
#     Phi(T[Phi*(p)]) = (Kt o Kt) p / mu - 2 diag(Cb_abar^T W' Cb),
# W' = alpha-bar rows of Psi' o V with the alpha-bar x alpha-bar block halved, i.e. the rows
# U = Cb_abar diag(p) Cb^T weighted by 1/(2 mu) on alpha-bar columns and 1/mu - xi on alpha.
# The CUDA path carries U for x (unweighted) and measures the stopping norm by the expansion
#     ||A2 - Psi o Vx||^2 = ||A2||^2 + 4 <A2_abar, W'> + sum_j w'_j W'^2
#                           - (2/mu) (x . Phi(at2) + 2 <W', U>) + x^T (Kt o Kt) x / mu^2,
# w'_j = 4 on alpha-bar columns and 2 on alpha columns; dX = P (A2 - Psi o Vx) P^T.

def _comp_row_weights(sig, nb, mu):
    """Weights of the alpha-bar rows (complement form): 1/(2 mu) on alpha-bar columns, 1/mu - xi on
    alpha columns."""
    l = sig.size
    Wt = np.empty((nb, l))
    for r in range(nb):
        for j in range(l):
            if j < nb:
                Wt[r, j] = 0.5 / mu
            else:
                eta = sig[j] / (sig[j] - sig[r])
                Wt[r, j] = 1.0 / mu - eta / (mu + 1.0 - eta)
    return Wt


@pytest.mark.parametrize("l,npos", SPLITS)
def test_complement_operator_in_eigenbasis(l, npos):
    mu = 0.37
    rng, R, P, sig = _problem(5 + l + npos, l, npos)
    e = ko.Eig(P=P, sig=sig)
    Psi = ko.psi_matrix(sig, mu)
    nb = l - npos
    p = rng.standard_normal(l)
    H_ref = ko.phi(R, ko.t_apply(e, Psi, ko.phi_star(R, p)))
    Cb = P.T @ R
    Kt = R.T @ R
    U = (Cb[:nb] * p[None, :]) @ Cb.T
    Wc = U * _comp_row_weights(sig, nb, mu)
    H = (Kt * Kt) @ p / mu - 2.0 * np.sum(Cb[:nb] * (Wc @ Cb), axis=0)
    assert np.max(np.abs(H - H_ref)) <= 1e-12 * max(1.0, np.max(np.abs(H_ref)))


@pytest.mark.parametrize("l,npos", SPLITS)
def test_complement_stopping_norm_in_eigenbasis(l, npos):
    mu = 0.37
    rng, R, P, sig = _problem(13 + l + npos, l, npos)
    e = ko.Eig(P=P, sig=sig)
    Psi = ko.psi_matrix(sig, mu)
    nb = l - npos
    x = rng.standard_normal(l)
    at2 = rng.standard_normal((l, l))
    at2 = at2 + at2.T
    ref = np.sum((at2 - ko.t_apply(e, Psi, ko.phi_star(R, x))) ** 2)
    Cb = P.T @ R
    Kt = R.T @ R
    A2 = P.T @ at2 @ P
    phi_at2 = np.sum(Cb * (A2 @ Cb), axis=0)             # Phi(at2) = diag(Cb^T A2 Cb)
    assert np.allclose(phi_at2, ko.phi(R, at2), rtol=1e-12, atol=1e-12)
    U = (Cb[:nb] * x[None, :]) @ Cb.T
    Wc = U * _comp_row_weights(sig, nb, mu)
    wp = np.where(np.arange(l) < nb, 4.0, 2.0)
    got = (np.sum(A2 ** 2) + 4.0 * np.sum(A2[:nb] * Wc) + np.sum(wp[None, :] * Wc ** 2)
           - (2.0 / mu) * (x @ phi_at2 + 2.0 * np.sum(Wc * U)) + x @ (Kt * Kt) @ x / mu ** 2)
    assert abs(got - ref) <= 1e-11 * max(ref, np.sum(A2 ** 2))


@pytest.mark.parametrize("l,npos", SPLITS)
def test_complement_direction_in_eigenbasis(l, npos):
    mu = 0.29
    rng, R, P, sig = _problem(29 + l + npos, l, npos)
    e = ko.Eig(P=P, sig=sig)
    Psi = ko.psi_matrix(sig, mu)
    r2 = rng.standard_normal((l, l))
    r2 = r2 + r2.T
    at2_ref = (-r2 + ko.t_apply(e, Psi, -r2)) / (mu + 1.0)
    Cb = P.T @ R
    A2 = -(1.0 + Psi) * (P.T @ r2 @ P) / (mu + 1.0)
    x = rng.standard_normal(l)
    Vx = (Cb * x[None, :]) @ Cb.T
    dX = P @ (A2 - Psi * Vx) @ P.T
    dX_ref = at2_ref - ko.t_apply(e, Psi, ko.phi_star(R, x))
    assert np.max(np.abs(dX - dX_ref)) <= 1e-12 * max(1.0, np.max(np.abs(dX_ref)))
