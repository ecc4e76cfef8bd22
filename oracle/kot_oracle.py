"""Oracle for the kernel-based OT semismooth Newton method (Lin, Cuturi & Jordan,
"A Specialized Semismooth Newton Method for Kernel-Based Optimal Transport").

TEST INFRASTRUCTURE ONLY. This module is a plain, slow, FP64 NumPy restatement of the
paper's method, written to be checked against the paper by eye. Only the test suite,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import it. The
CUDA library never calls it and it never calls the CUDA library.

Notation follows the paper with the sample/filling-point clash resolved as:
  n  = number of samples drawn from each measure (the paper's n_sample),
  l  = number of filling points (the paper's n),
  d  = dimension of x and of y.

Readings of points the paper leaves open (each is also an option here):
  * kernel: Gaussian k(a,b) = exp(-||a-b||^2 / (2 sigma^2)), one sigma for k_X, k_Y, k_XY
    (Sec. 5 gives only a Gaussian bandwidth);
  * q^2 = ||w_mu||^2 + ||w_nu||^2, both squared (the printed definition after Eq. (3.2)
    drops the square on the nu term, the displayed formulas below it square both);
  * Cholesky jitter: K + eps*I with eps = jitter * max_i K_ii, multiplied by 10 on failure
    up to jitter_max;
  * EG step size eta = 1/L with L = max row-sum(|Q|)/(2 lambda2) + sqrt(max row-sum(Kt o Kt)),
    Kt = R^T R (an upper bound of the Lipschitz constant of the min-max operator);
  * tau = 0.1, kappa = 1 for the inexact-Newton test (Eq. (4.3));
  * theta_0 = 1, theta_min = 1e-6, theta_max = 1e6; alpha1, alpha2, beta0..2 from Sec. 5;
  * ||dw||^2 in the theta rule = (||dgamma||_2 + ||dX||_F)^2 (the norm below Eq. (4.3));
  * w_0 = v_0 = (0, 0); the EG sequence v is never reset to w;
  * R is printed on R^l x R^{l x l}, but the projection onto S^l_+ (symmetric PSD matrices)
    of a general matrix is that of its symmetric part, so the generalized Jacobian M(Z) of
    Sec. 4.2, and with it T_k of Sec. 4.3, acts on the symmetric part of its argument.  (Applied
    to the raw argument, rounding-level asymmetry of X grows by about 1/mu per Newton step.)

Functions whose result is pinned only by properties (no closed form or printed value) say so
in their docstring.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


# ----------------------------------------------------------------------------------------
# Options (Sec. 5 constants and the readings listed in the module docstring)
# ----------------------------------------------------------------------------------------
@dataclass
class Options:
    max_iter: int = 200
    cg_max_iter: int = 20          # Sec. 4.4 remark: CG capped at 20 iterations
    tau: float = 0.1               # Eq. (4.3): 0 < tau < 1 (value not given)
    kappa: float = 1.0             # Eq. (4.3): kappa (value not given)
    alpha1: float = 1e-6           # Sec. 5
    alpha2: float = 1.0            # Sec. 5
    beta0: float = 0.5             # Sec. 5
    beta1: float = 1.2             # Sec. 5
    beta2: float = 5.0             # Sec. 5
    theta0: float = 1.0
    theta_min: float = 1e-6
    theta_max: float = 1e6
    eg_step: float = 0.0           # <= 0: 1/L (see module docstring)
    jitter: float = 1e-10
    jitter_max: float = 1e-6
    use_eg: bool = True            # Algorithm 2 safeguard on/off
    record_history: bool = False
    schur_solver: int = 0          # 0: CG, 1: symmetric QMR (Sec. 4.3 names both)


# ----------------------------------------------------------------------------------------
# Feature assembly (Sec. 3, the definitions of Q, z, q^2, K, R after Eq. (3.2))
# ----------------------------------------------------------------------------------------
def sqdist(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Pairwise squared Euclidean distances ||a_i - b_j||^2 by explicit differences."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    out = np.empty((A.shape[0], B.shape[0]))
    step = max(1, int(2e7 // max(1, B.shape[0] * A.shape[1])))
    for s in range(0, A.shape[0], step):
        diff = A[s:s + step, None, :] - B[None, :, :]
        out[s:s + step] = np.sum(diff * diff, axis=2)
    return out


def gaussian_kernel(A: np.ndarray, B: np.ndarray, sigma: float) -> np.ndarray:
    """k(a, b) = exp(-||a - b||^2 / (2 sigma^2)) for all pairs (reading of Sec. 5)."""
    return np.exp(-sqdist(A, B) / (2.0 * sigma * sigma))


@dataclass
class Features:
    """Problem data of the dual SDP (Eq. (3.3))."""
    Q: np.ndarray        # l x l, Q_ij = k_X(xf_i, xf_j) + k_Y(yf_i, yf_j)
    z: np.ndarray        # l, z_i = w_mu(xf_i) + w_nu(yf_i) - lambda2 ||xf_i - yf_i||^2
    q2: float            # ||w_mu||^2 + ||w_nu||^2
    K: np.ndarray        # l x l Gram of k_XY on the filling pairs
    R: np.ndarray        # l x l upper triangular, R^T R = K + eps I; Phi_i = R[:, i]
    w_mu: np.ndarray     # l, kernel mean embedding of mu-hat at xf_i
    w_nu: np.ndarray     # l, kernel mean embedding of nu-hat at yf_i
    c: np.ndarray        # l, ||xf_i - yf_i||^2
    eps: float           # jitter actually added to K before the Cholesky
    lambda1: float
    lambda2: float

    @property
    def l(self) -> int:
        return self.Q.shape[0]


def kernel_mean_embedding(S: np.ndarray, P: np.ndarray, sigma: float) -> np.ndarray:
    """w(p_i) = (1/n) sum_j k(s_j, p_i) (Sec. 3, displayed formulas for w_mu, w_nu)."""
    return gaussian_kernel(P, S, sigma).mean(axis=1)


def embedding_sqnorm(S: np.ndarray, sigma: float) -> float:
    """||w||^2 = (1/n^2) sum_{i,j} k(s_i, s_j) (Sec. 3, displayed formulas)."""
    n = S.shape[0]
    total = 0.0
    step = 512
    for a in range(0, n, step):
        total += float(gaussian_kernel(S[a:a + step], S, sigma).sum())
    return total / (n * n)


def cholesky_upper_jittered(K: np.ndarray, jitter: float, jitter_max: float):
    """Upper R with R^T R = K + eps I (Sec. 3: R is the Cholesky factor of K).

    eps = jitter * max_i K_ii, multiplied by 10 until the factorisation succeeds or
    eps exceeds jitter_max * max_i K_ii (then raises LinAlgError)."""
    scale = float(np.max(np.diag(K)))
    rel = jitter
    while True:
        eps = rel * scale
        try:
            L = np.linalg.cholesky(K + eps * np.eye(K.shape[0]))
            return L.T.copy(), eps
        except np.linalg.LinAlgError:
            rel *= 10.0
            if not rel > 0.0 or rel > jitter_max * (1 + 1e-12):
                raise


def build_features(X, Y, Xf, Yf, sigma, lambda1, lambda2, opt: Options | None = None) -> Features:
    """Assemble Q, z, q^2, K and R from samples and filling points (Sec. 3)."""
    opt = opt or Options()
    X = np.asarray(X, np.float64); Y = np.asarray(Y, np.float64)
    Xf = np.asarray(Xf, np.float64); Yf = np.asarray(Yf, np.float64)
    w_mu = kernel_mean_embedding(X, Xf, sigma)
    w_nu = kernel_mean_embedding(Y, Yf, sigma)
    q2 = embedding_sqnorm(X, sigma) + embedding_sqnorm(Y, sigma)
    Q = gaussian_kernel(Xf, Xf, sigma) + gaussian_kernel(Yf, Yf, sigma)
    c = np.sum((Xf - Yf) ** 2, axis=1)
    z = w_mu + w_nu - lambda2 * c
    F = np.concatenate([Xf, Yf], axis=1)
    K = gaussian_kernel(F, F, sigma)
    R, eps = cholesky_upper_jittered(K, opt.jitter, opt.jitter_max)
    return Features(Q=Q, z=z, q2=q2, K=K, R=R, w_mu=w_mu, w_nu=w_nu, c=c, eps=eps,
                    lambda1=float(lambda1), lambda2=float(lambda2))


# ----------------------------------------------------------------------------------------
# Operators (Sec. 4.1)
# ----------------------------------------------------------------------------------------
def phi_star(R: np.ndarray, gamma: np.ndarray) -> np.ndarray:
    """Phi*(gamma) = sum_i gamma_i Phi_i Phi_i^T = R diag(gamma) R^T (Sec. 4.1)."""
    return (R * gamma[None, :]) @ R.T


def phi(R: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Phi(X)_i = <X, Phi_i Phi_i^T> = (R^T X R)_ii (Sec. 4.1)."""
    return np.sum(R * (X @ R), axis=0)


def objective(F: Features, gamma: np.ndarray) -> float:
    """Dual objective of Eq. (3.3)."""
    lam2 = F.lambda2
    return float(gamma @ F.Q @ gamma / (4 * lam2) - gamma @ F.z / (2 * lam2) + F.q2 / (4 * lam2))


def ot_estimate(F: Features, gamma: np.ndarray) -> float:
    """OT-hat = q^2/(2 lambda2) - (1/(2 lambda2)) sum_i gamma_i (w_mu(xf_i) + w_nu(yf_i)) (Sec. 3)."""
    return float(F.q2 / (2 * F.lambda2) - gamma @ (F.w_mu + F.w_nu) / (2 * F.lambda2))


def sym(A: np.ndarray) -> np.ndarray:
    return 0.5 * (A + A.T)


@dataclass
class Eig:
    """Spectral decomposition Z = P diag(sig) P^T with alpha = {sig > 0} (Eq. (4.4))."""
    P: np.ndarray
    sig: np.ndarray

    @property
    def alpha(self) -> np.ndarray:
        return self.sig > 0.0


def eig_sym(Z: np.ndarray) -> Eig:
    sig, P = np.linalg.eigh(sym(Z))
    return Eig(P=P, sig=sig)


def proj_psd_from_eig(e: Eig) -> np.ndarray:
    """Pi_{S+}(Z) = P_alpha Sigma_alpha P_alpha^T (Eq. (4.4))."""
    a = e.alpha
    Pa = e.P[:, a]
    return (Pa * e.sig[a][None, :]) @ Pa.T


def proj_psd(Z: np.ndarray) -> np.ndarray:
    return proj_psd_from_eig(eig_sym(Z))


@dataclass
class Residual:
    """Natural residual R(w) = (r1, r2) of Eq. (4.2) and the pieces it was built from."""
    r1: np.ndarray
    r2: np.ndarray
    eig: Eig          # spectral decomposition of Z = X - (Phi*(gamma) + lambda1 I)
    proj: np.ndarray  # Pi_{S+}(Z)

    @property
    def norm(self) -> float:
        """||w|| = ||gamma||_2 + ||X||_F (the norm defined below Eq. (4.3))."""
        return float(np.linalg.norm(self.r1) + np.linalg.norm(self.r2))


def residual(F: Features, gamma: np.ndarray, X: np.ndarray) -> Residual:
    """R(w) for w = (gamma, X), Eq. (4.2)."""
    l = F.l
    S = phi_star(F.R, gamma) + F.lambda1 * np.eye(l)
    Z = sym(X - S)
    e = eig_sym(Z)
    Pi = proj_psd_from_eig(e)
    r1 = (F.Q @ gamma - F.z) / (2 * F.lambda2) - phi(F.R, X)
    r2 = X - Pi
    return Residual(r1=r1, r2=r2, eig=e, proj=Pi)


def pair_norm(a: np.ndarray, A: np.ndarray) -> float:
    return float(np.linalg.norm(a) + np.linalg.norm(A))


def pair_inner(a: np.ndarray, A: np.ndarray, b: np.ndarray, B: np.ndarray) -> float:
    return float(a @ b + np.sum(A * B))


# ----------------------------------------------------------------------------------------
# Generalised Jacobian of the projection and the operator T_k (Sec. 4.2, 4.3)
# ----------------------------------------------------------------------------------------
def omega_matrix(sig: np.ndarray) -> np.ndarray:
    """Omega of M(Z): ones on alpha x alpha, eta_ij = sig_i/(sig_i - sig_j) on alpha x
    alpha-bar (and its transpose), zero on alpha-bar x alpha-bar (Sec. 4.2)."""
    a = sig > 0
    l = sig.shape[0]
    Om = np.zeros((l, l))
    Om[np.ix_(a, a)] = 1.0
    ia = np.where(a)[0]
    ib = np.where(~a)[0]
    for i in ia:
        for j in ib:
            eta = sig[i] / (sig[i] - sig[j])
            Om[i, j] = eta
            Om[j, i] = eta
    return Om


def jacobian_proj_apply(e: Eig, S: np.ndarray) -> np.ndarray:
    """M(Z)[S] = P (Omega o (P^T S P)) P^T (Sec. 4.2)."""
    Om = omega_matrix(e.sig)
    return e.P @ (Om * (e.P.T @ S @ e.P)) @ e.P.T


def psi_matrix(sig: np.ndarray, mu: float) -> np.ndarray:
    """Psi_k: 1/mu on alpha x alpha, xi_ij = eta_ij/(mu + 1 - eta_ij) on alpha x alpha-bar
    and its transpose, zero on alpha-bar x alpha-bar (Sec. 4.3, the display defining Psi_k).
    Entry-wise this is Omega_ij/(mu + 1 - Omega_ij), the diagonal of L_k in Lemma 4.4."""
    Om = omega_matrix(sig)
    return Om / (mu + 1.0 - Om)


def t_apply(e: Eig, Psi: np.ndarray, S: np.ndarray) -> np.ndarray:
    """T_k[S] = P (Psi o (P^T sym(S) P)) P^T (Sec. 4.3), the operator form of T_k = P~ L_k P~^T.

    sym(S): M(Z) is the generalized Jacobian of the projection onto S^l_+, which sees only the
    symmetric part of a matrix (see the module docstring)."""
    return e.P @ (Psi * (e.P.T @ sym(S) @ e.P)) @ e.P.T


# ----------------------------------------------------------------------------------------
# Newton direction: Algorithm 1 with CG on the Schur-reduced system (Sec. 4.3)
# ----------------------------------------------------------------------------------------
@dataclass
class Direction:
    dgamma: np.ndarray
    dX: np.ndarray
    cg_iters: int
    cg_res: float
    stop_margin: float = math.inf   # min over CG stop tests of | ||e|| - threshold | / threshold


def newton_direction(F: Features, res: Residual, mu: float, opt: Options,
                     cg_tol_abs: float | None = None) -> Direction:
    """Algorithm 1. Solves (J_k + mu_k I)[dw] = -r_k inexactly (Eq. (4.3)).

    a1 = -r1 - Phi(r2 + T[r2])/(mu+1), a2 = -r2;
    (Q/(2 lambda2) + mu I + Phi T Phi*) at1 = a1 by CG (or symmetric QMR) from 0;
    at2 = (a2 + T[a2])/(mu+1);  dgamma = at1,  dX = at2 - T[Phi*(at1)].

    The full-system residual of an inexact at1 equals the CG residual (the second block row
    of the Schur form is solved exactly, Lemma 4.4), so CG stops when
    ||e||_2 <= tau * min(1, kappa * ||r_k|| * ||dw||) with dw implied by the current iterate,
    or after cg_max_iter iterations. ``cg_tol_abs`` replaces that test by ||e|| <= cg_tol_abs
    (used by tests that want a nearly exact direction)."""
    R, Q, lam2 = F.R, F.Q, F.lambda2
    Psi = psi_matrix(res.eig.sig, mu)

    def T(S):
        return t_apply(res.eig, Psi, S)

    r1, r2 = res.r1, res.r2
    rnorm = res.norm
    a1 = -r1 - phi(R, r2 + T(r2)) / (mu + 1.0)
    a2 = -r2
    at2 = (a2 + T(a2)) / (mu + 1.0)

    def schur_matvec(v):
        TPv = T(phi_star(R, v))
        return Q @ v / (2 * lam2) + mu * v + phi(R, TPv), TPv

    x = np.zeros_like(a1)
    TPx = np.zeros_like(at2)        # T[Phi*(x)], kept alongside x
    e = a1.copy()                   # residual a1 - H x
    p = e.copy()
    ee = float(e @ e)
    it = 0

    margin = [math.inf]

    def stop(x, TPx, ee):
        enorm = math.sqrt(ee)
        if cg_tol_abs is not None:
            return enorm <= cg_tol_abs
        dw = pair_norm(x, at2 - TPx)
        thr = opt.tau * min(1.0, opt.kappa * rnorm * dw)
        if thr > 0:
            margin[0] = min(margin[0], abs(enorm - thr) / thr)
        return enorm <= thr

    cap = opt.cg_max_iter if cg_tol_abs is None else 10 * x.size + 50
    if opt.schur_solver == 0:
        while not stop(x, TPx, ee) and it < cap:
            Hp, TPp = schur_matvec(p)
            pHp = float(p @ Hp)
            if pHp <= 0.0:
                break
            a = ee / pHp
            x = x + a * p
            TPx = TPx + a * TPp
            e = e - a * Hp
            ee_new = float(e @ e)
            p = e + (ee_new / ee) * p
            ee = ee_new
            it += 1
    else:
        # Symmetric QMR without preconditioning (Freund and Nachtigal): the Lanczos/CG residual
        # rl drives the recurrences, the iterate x moves along the smoothed direction d, and the
        # true residual e = a1 - H x and T[Phi*(x)] are updated through H d and T[Phi*(d)].
        rl = e.copy()
        q = rl.copy()
        tau_q = math.sqrt(float(rl @ rl))
        theta = 0.0
        rho = float(rl @ rl)
        d = np.zeros_like(x)
        Hd = np.zeros_like(x)
        TPd = np.zeros_like(TPx)
        while not stop(x, TPx, ee) and it < cap:
            t, TPq = schur_matvec(q)
            sig = float(q @ t)
            if sig <= 0.0 or tau_q == 0.0:
                break
            a = rho / sig
            rl = rl - a * t
            theta_old = theta
            theta = math.sqrt(float(rl @ rl)) / tau_q
            c2 = 1.0 / (1.0 + theta * theta)
            tau_q = tau_q * theta * math.sqrt(c2)
            d = (c2 * theta_old * theta_old) * d + (c2 * a) * q
            Hd = (c2 * theta_old * theta_old) * Hd + (c2 * a) * t
            TPd = (c2 * theta_old * theta_old) * TPd + (c2 * a) * TPq
            x = x + d
            TPx = TPx + TPd
            e = e - Hd
            ee = float(e @ e)
            rho_old = rho
            rho = float(rl @ rl)
            q = rl + (rho / rho_old) * q
            it += 1
    return Direction(dgamma=x, dX=at2 - TPx, cg_iters=it, cg_res=math.sqrt(ee),
                     stop_margin=margin[0])


# ----------------------------------------------------------------------------------------
# Potentials and transport map from the dual solution
# ----------------------------------------------------------------------------------------
def potential(S: np.ndarray, Sf: np.ndarray, gamma: np.ndarray, sigma: float, lambda2: float,
              P: np.ndarray):
    """Empirical Kantorovich potential of one side and its gradient at the points P (m x d).

    Stationarity of the Lagrangian of Eq. (3.2) in u gives
        u(x) = (w_mu(x) - sum_i gamma_i k(xf_i, x)) / (2 lambda2),  w_mu(x) = (1/n) sum_j k(x_j, x),
    (the same with Y, yf for v); with k(a, x) = exp(-||a - x||^2 / (2 sigma^2)),
        grad u(x) = (1/(2 lambda2)) sum_a c_a k(a, x) (a - x) / sigma^2,
    c_a = 1/n for the samples a = x_j and -gamma_i for the filling points a = xf_i.  The map
    estimate for the cost ||x - y||^2 / 2 is T(x) = x - grad u(x) (the displacement of Figs. 1,
    4 and 7).  Returns (u (m), grad (m x d), T (m x d)).  Pinned by the estimator identity
    <u, w_mu> + <v, w_nu> = OT-hat (Sec. 3), by finite differences and by gamma = 0."""
    n = S.shape[0]
    A = np.vstack([S, Sf])                                   # sources a
    c = np.concatenate([np.full(n, 1.0 / n), -np.asarray(gamma, dtype=np.float64)])
    Kx = gaussian_kernel(P, A, sigma)                        # m x (n + l)
    W = Kx * c[None, :]
    u = W.sum(axis=1) / (2.0 * lambda2)
    grad = (W @ A - W.sum(axis=1)[:, None] * P) / (2.0 * lambda2 * sigma * sigma)
    return u, grad, P - grad


# ----------------------------------------------------------------------------------------
# Extragradient on the min-max problem Eq. (4.1), used as the safeguard of Algorithm 2
# ----------------------------------------------------------------------------------------
def eg_lipschitz(F: Features) -> float:
    """L = max_i sum_j |Q_ij| / (2 lambda2) + sqrt(max_i sum_j (Kt_ij)^2), Kt = R^T R.

    The min-max operator is affine with linear part [[Q/(2 lambda2), -A], [A^T, 0]]; its norm
    is at most ||Q||/(2 lambda2) + ||A|| and ||A||^2 = ||A A^T|| = ||Kt o Kt||; each spectral
    norm is bounded by the maximum absolute row sum."""
    Kt = F.R.T @ F.R
    return float(np.max(np.sum(np.abs(F.Q), axis=1)) / (2 * F.lambda2)
                 + math.sqrt(np.max(np.sum(Kt * Kt, axis=1))))


def eg_operator(F: Features, gamma: np.ndarray, X: np.ndarray):
    """F(gamma, X) = (grad_gamma L, -grad_X L) of the min-max Lagrangian L of Eq. (4.1):
    ((Q gamma - z)/(2 lambda2) - Phi(X),  Phi*(gamma) + lambda1 I)."""
    g = (F.Q @ gamma - F.z) / (2 * F.lambda2) - phi(F.R, X)
    G = phi_star(F.R, gamma) + F.lambda1 * np.eye(F.l)
    return g, G


def eg_step(F: Features, gamma: np.ndarray, X: np.ndarray, eta: float):
    """One projected extragradient step on R^l x S^l_+ (Korpelevich)."""
    g, G = eg_operator(F, gamma, X)
    gh = gamma - eta * g
    Xh = proj_psd(X - eta * G)
    g2, G2 = eg_operator(F, gh, Xh)
    return gamma - eta * g2, proj_psd(X - eta * G2)


# ----------------------------------------------------------------------------------------
# Algorithm 2
# ----------------------------------------------------------------------------------------
@dataclass
class Result:
    gamma: np.ndarray
    X: np.ndarray
    residual: float
    r1_norm: float
    r2_norm: float
    objective: float
    ot_hat: float
    iters: int
    ssn_accepted: int
    eg_taken: int
    cg_total: int
    converged: bool
    history: list = field(default_factory=list)


def ssn_solve(F: Features, tol: float, opt: Options | None = None,
              gamma0: np.ndarray | None = None, X0: np.ndarray | None = None) -> Result:
    """Algorithm 2: EG safeguard + regularised SSN step + adaptive theta + acceptance test.

    Per iteration k: v_{k+1} = EG(v_k); mu_k = theta_k ||R(w_k)||; dw_k from Algorithm 1 at
    w_k; theta_{k+1} from rho_k = -<R(w_k + dw_k), dw_k> (Sec. 4.3 rule);
    w_{k+1} = w_k + dw_k if ||R(w_k + dw_k)|| <= ||R(v_{k+1})||, else v_{k+1}.
    Stops when ||R(w_k)|| <= tol or after max_iter iterations."""
    opt = opt or Options()
    l = F.l
    gamma = np.zeros(l) if gamma0 is None else np.array(gamma0, dtype=np.float64)
    X = np.zeros((l, l)) if X0 is None else np.array(X0, dtype=np.float64)
    vg, vX = gamma.copy(), X.copy()
    theta = opt.theta0
    eta = opt.eg_step if opt.eg_step > 0 else 1.0 / eg_lipschitz(F)
    res = residual(F, gamma, X)
    it = ssn_acc = eg_tk = cg_tot = 0
    hist = []
    while res.norm > tol and it < opt.max_iter:
        if opt.use_eg:
            vg, vX = eg_step(F, vg, vX, eta)
            res_v = residual(F, vg, vX)
        mu = theta * res.norm
        # relative distance of Z(w_k)'s spectrum from 0: how far the alpha split used by this
        # step is from a rounding-level sign decision (recorded for the parity tests)
        sig = res.eig.sig
        split_margin = float(np.min(np.abs(sig)) / max(np.max(np.abs(sig)), 1e-300))
        dirn = newton_direction(F, res, mu, opt)
        cg_tot += dirn.cg_iters
        tg, tX = gamma + dirn.dgamma, X + dirn.dX
        res_t = residual(F, tg, tX)
        dwn = pair_norm(dirn.dgamma, dirn.dX)
        rho = -pair_inner(res_t.r1, res_t.r2, dirn.dgamma, dirn.dX)
        ratio = rho / (dwn * dwn) if dwn > 0 else math.inf
        theta_margin = min(abs(ratio - opt.alpha1) / opt.alpha1, abs(ratio - opt.alpha2) / opt.alpha2)
        accept_margin = (abs(res_t.norm - res_v.norm) / res_v.norm) if opt.use_eg else math.inf
        if rho >= opt.alpha2 * dwn * dwn:
            theta = max(opt.theta_min, opt.beta0 * theta)
        elif rho >= opt.alpha1 * dwn * dwn:
            theta = opt.beta1 * theta
        else:
            theta = min(opt.theta_max, opt.beta2 * theta)
        if (not opt.use_eg) or res_t.norm <= res_v.norm:
            gamma, X, res = tg, tX, res_t
            ssn_acc += 1
        else:
            gamma, X, res = vg.copy(), vX.copy(), res_v
            eg_tk += 1
        it += 1
        if opt.record_history:
            # (||R(w_{k+1})||, mu_k, CG steps, theta_{k+1}, relative margins of the decisions
            #  taken in iteration k: alpha split, CG stop tests, theta rule, acceptance)
            hist.append((res.norm, mu, dirn.cg_iters, theta, split_margin, dirn.stop_margin,
                         theta_margin, accept_margin))
    return Result(gamma=gamma, X=X, residual=res.norm, r1_norm=float(np.linalg.norm(res.r1)),
                  r2_norm=float(np.linalg.norm(res.r2)), objective=objective(F, gamma),
                  ot_hat=ot_estimate(F, gamma), iters=it, ssn_accepted=ssn_acc, eg_taken=eg_tk,
                  cg_total=cg_tot, converged=res.norm <= tol, history=hist)


def eg_solve(F: Features, tol: float, max_iter: int, eta: float | None = None,
             gamma0=None, X0=None) -> Result:
    """Pure extragradient on Eq. (4.1) (the comparison method of Appendix F)."""
    l = F.l
    g = np.zeros(l) if gamma0 is None else np.array(gamma0, dtype=np.float64)
    X = np.zeros((l, l)) if X0 is None else np.array(X0, dtype=np.float64)
    eta = eta if eta is not None else 1.0 / eg_lipschitz(F)
    res = residual(F, g, X)
    it = 0
    while res.norm > tol and it < max_iter:
        g, X = eg_step(F, g, X, eta)
        res = residual(F, g, X)
        it += 1
    return Result(gamma=g, X=X, residual=res.norm, r1_norm=float(np.linalg.norm(res.r1)),
                  r2_norm=float(np.linalg.norm(res.r2)), objective=objective(F, g),
                  ot_hat=ot_estimate(F, g), iters=it, ssn_accepted=0, eg_taken=it,
                  cg_total=0, converged=res.norm <= tol)
