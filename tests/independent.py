"""Independent checkers used to pin the oracle (test infrastructure).

Nothing here shares code with the oracle's solver: a log-barrier interior-point method for
the dual SDP (Eq. (3.3)), the explicit Kronecker-form matrices of Lemma 4.4 and a dense
solve of the (l + l^2) Newton system.
"""
from __future__ import annotations

import numpy as np


def ipm_solve(Q, z, q2, R, lambda1, lambda2, t_end=1e-13):
    """Damped-Newton log-barrier method for
        min  gamma^T Q gamma/(4 l2) - gamma^T z/(2 l2) + q2/(4 l2)
        s.t. R diag(gamma) R^T + lambda1 I >= 0.
    Returns (gamma, X) with X = t S^{-1} the barrier's dual estimate; the duality gap of the
    central point is l * t."""
    l = Q.shape[0]

    def f(g):
        return g @ Q @ g / (4 * lambda2) - g @ z / (2 * lambda2) + q2 / (4 * lambda2)

    def barrier(g, t):
        S = (R * g[None, :]) @ R.T + lambda1 * np.eye(l)
        try:
            C = np.linalg.cholesky(S)
        except np.linalg.LinAlgError:
            return np.inf
        return f(g) - 2.0 * t * np.sum(np.log(np.diag(C)))

    g = np.zeros(l)
    t = 1.0
    while True:
        for _ in range(200):
            S = (R * g[None, :]) @ R.T + lambda1 * np.eye(l)
            Si = np.linalg.inv(S)
            M = R.T @ Si @ R
            grad = (Q @ g - z) / (2 * lambda2) - t * np.diag(M)
            H = Q / (2 * lambda2) + t * M * M
            step = -np.linalg.solve(H, grad)
            dec = -grad @ step
            if dec < 1e-22:
                break
            s, f0 = 1.0, barrier(g, t)
            while barrier(g + s * step, t) > f0 - 0.25 * s * dec and s > 1e-30:
                s *= 0.5
            g = g + s * step
        if t <= t_end:
            S = (R * g[None, :]) @ R.T + lambda1 * np.eye(l)
            return g, t * np.linalg.inv(S)
        t *= 0.25


def kron_operators(P, sig, mu):
    """Explicit l^2 x l^2 matrices of Lemma 4.4 with column-major vec (vec(A S B) =
    (B^T kron A) vec(S)): P~ = P kron P, Gamma = diag(vec Omega), W = P~ Gamma P~^T,
    D = P~((mu+1)I - Gamma)P~^T, T = P~ L P~^T with L_ii = Gamma_ii/(mu+1-Gamma_ii).
    Omega is built here entry by entry from its definition in Sec. 4.2."""
    l = sig.shape[0]
    Om = np.zeros((l, l))
    for i in range(l):
        for j in range(l):
            if sig[i] > 0 and sig[j] > 0:
                Om[i, j] = 1.0
            elif sig[i] > 0 and sig[j] <= 0:
                Om[i, j] = sig[i] / (sig[i] - sig[j])
            elif sig[j] > 0 and sig[i] <= 0:
                Om[i, j] = sig[j] / (sig[j] - sig[i])
    Pt = np.kron(P, P)
    gam = Om.flatten(order="F")
    W = Pt @ np.diag(gam) @ Pt.T
    D = Pt @ np.diag(mu + 1.0 - gam) @ Pt.T
    T = Pt @ np.diag(gam / (mu + 1.0 - gam)) @ Pt.T
    return W, D, T


def vec(A):
    return A.flatten(order="F")


def unvec(v, l):
    return v.reshape((l, l), order="F")


def dense_newton(Q, R, lambda2, P, sig, mu, r1, r2):
    """Solve (J + mu I) dw = -r with the explicit block matrix of Lemma 4.4's proof,
    J + mu I = [[Q/(2 l2) + mu I, -A], [W A^T, D]], A_i = (Phi_i kron Phi_i)^T."""
    l = Q.shape[0]
    A = np.stack([np.kron(R[:, i], R[:, i]) for i in range(l)])  # l x l^2
    W, D, _ = kron_operators(P, sig, mu)
    top = np.hstack([Q / (2 * lambda2) + mu * np.eye(l), -A])
    bot = np.hstack([W @ A.T, D])
    J = np.vstack([top, bot])
    rhs = -np.concatenate([r1, vec(r2)])
    sol = np.linalg.solve(J, rhs)
    return sol[:l], unvec(sol[l:], l)
