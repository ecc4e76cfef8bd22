"""Seeded synthetic workloads for the kernel-based OT solver.

This module draws samples, filling points and the problem parameters (bandwidth, lambda1,
lambda2, tolerance) with NumPy's PCG64 generator. It holds none of the solver's arithmetic:
the oracle and the CUDA library both receive what it returns, so the same bytes reach both.

Shapes follow the paper's workloads (Sec. 5 and Appendix F): samples X, Y of size n x d from
two Gaussian (mixture) measures, and l filling pairs (xf_j, yf_j) in the product space. The
single-cell 4i data of Sec. 5 are not available, so ``feature_like`` stands in for their shape
(48-dimensional features, a few hundred filling points) at a larger size.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Problem:
    name: str
    X: np.ndarray        # n x d samples of mu
    Y: np.ndarray        # n x d samples of nu
    Xf: np.ndarray       # l x d filling points, x half
    Yf: np.ndarray       # l x d filling points, y half
    sigma: float
    lambda1: float
    lambda2: float
    tol: float = 1e-6

    @property
    def n(self) -> int:
        return self.X.shape[0]

    @property
    def d(self) -> int:
        return self.X.shape[1]

    @property
    def l(self) -> int:
        return self.Xf.shape[0]


def median_distance(P: np.ndarray, max_points: int = 1000) -> float:
    """Median pairwise Euclidean distance of (a fixed prefix of at most max_points of) P."""
    P = P[:max_points]
    G = P @ P.T
    sq = np.diag(G)[:, None] + np.diag(G)[None, :] - 2.0 * G
    iu = np.triu_indices(P.shape[0], 1)
    return float(np.sqrt(np.median(np.maximum(sq[iu], 0.0))))


def gaussian_pair(seed: int = 0, n: int = 100, l: int = 50, sigma: float = 1.0,
                  lambda1: float = 1e-3, lambda2: float | None = None) -> Problem:
    """mu = N(0, I_2), nu = N((1,1), diag(0.5, 2)); filling points uniform on [-3,3]^4.

    Draw order: X, Y, filling points. lambda2 defaults to 1/n."""
    rng = np.random.default_rng(seed)
    d = 2
    X = rng.standard_normal((n, d))
    Y = np.array([1.0, 1.0]) + rng.standard_normal((n, d)) * np.sqrt(np.array([0.5, 2.0]))
    Fp = rng.uniform(-3.0, 3.0, size=(l, 2 * d))
    return Problem("gaussian_pair_d2", X, Y, Fp[:, :d].copy(), Fp[:, d:].copy(), sigma,
                   lambda1, 1.0 / n if lambda2 is None else lambda2)


def wishart_pair(seed: int = 1, d: int = 5, n: int = 1000, l: int = 300,
                 lambda1: float = 1e-4, lambda2: float | None = None) -> Problem:
    """mu, nu Gaussians with means uniform in [-1,1]^d and Wishart(d, I) covariances G G^T;
    filling points uniform on the per-coordinate bounding box of the pooled samples;
    sigma = median pairwise distance of the pooled samples; lambda2 defaults to 1/n."""
    rng = np.random.default_rng(seed)
    m1 = rng.uniform(-1, 1, d)
    m2 = rng.uniform(-1, 1, d)
    G1 = rng.standard_normal((d, d))
    G2 = rng.standard_normal((d, d))
    X = m1 + rng.standard_normal((n, d)) @ G1.T
    Y = m2 + rng.standard_normal((n, d)) @ G2.T
    pooled = np.concatenate([X, Y])
    lo, hi = pooled.min(axis=0), pooled.max(axis=0)
    Xf = rng.uniform(lo, hi, size=(l, d))
    Yf = rng.uniform(lo, hi, size=(l, d))
    sigma = median_distance(pooled)
    return Problem(f"wishart_pair_d{d}", X, Y, Xf, Yf, sigma, lambda1,
                   1.0 / n if lambda2 is None else lambda2)


def _product_filling(rng, X, Y, l):
    """l filling pairs (x_a, y_b) with (a, b) drawn without replacement from [n] x [n]."""
    n = X.shape[0]
    idx = rng.choice(n * n, size=l, replace=False)
    a, b = idx // n, idx % n
    return X[a].copy(), Y[b].copy()


def mixture_rotation(seed: int = 2, d: int = 10, n: int = 2000, l: int = 1024,
                     lambda1: float = 1e-4, lambda2: float | None = None) -> Problem:
    """mu: 4-component equal-weight Gaussian mixture, means uniform in [-2,2]^d, cov 0.25 I;
    nu: fresh mu-draws mapped by y = O x + b, O Haar-orthogonal, b ~ N(0, 0.25 I);
    filling pairs from the product of the samples; sigma = median distance; lambda2 = 1/n."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-2, 2, size=(4, d))

    def draw(m):
        comp = rng.integers(0, 4, size=m)
        return means[comp] + 0.5 * rng.standard_normal((m, d))

    X = draw(n)
    A = rng.standard_normal((d, d))
    O, Rq = np.linalg.qr(A)
    O = O * np.sign(np.diag(Rq))[None, :]
    b = 0.5 * rng.standard_normal(d)
    Y = draw(n) @ O.T + b
    Xf, Yf = _product_filling(rng, X, Y, l)
    sigma = median_distance(np.concatenate([X, Y]))
    return Problem(f"mixture_rotation_d{d}", X, Y, Xf, Yf, sigma, lambda1,
                   1.0 / n if lambda2 is None else lambda2)


def feature_like(seed: int = 3, d: int = 64, n: int = 4000, l: int = 2048,
                 lambda1: float = 1e-4, boot: int = 0) -> Problem:
    """Stand-in for L2-normalised cell features: mu a 10-cluster mixture (centres random unit
    vectors, std 0.1), nu draws around centres perturbed by N(0, 0.05^2 I); both normalised.
    ``boot`` > 0 returns bootstrap resample number ``boot`` of (X, Y) with the filling points
    of resample 0 kept fixed."""
    rng = np.random.default_rng(seed)
    C = rng.standard_normal((10, d))
    C /= np.linalg.norm(C, axis=1, keepdims=True)
    Cn = C + 0.05 * rng.standard_normal((10, d))

    def draw(centres, m):
        comp = rng.integers(0, 10, size=m)
        P = centres[comp] + 0.1 * rng.standard_normal((m, d))
        return P / np.linalg.norm(P, axis=1, keepdims=True)

    X = draw(C, n)
    Y = draw(Cn, n)
    Xf, Yf = _product_filling(rng, X, Y, l)
    sigma = median_distance(np.concatenate([X, Y]))
    if boot > 0:
        brng = np.random.default_rng(seed * 1000 + boot)
        X = X[brng.integers(0, n, size=n)]
        Y = Y[brng.integers(0, n, size=n)]
    return Problem(f"feature_like_d{d}", X, Y, Xf, Yf, sigma, lambda1, 1.0 / n)


def uneven_batch(count: int = 256, base_seed: int = 1000, l_max: int = 512) -> list[Problem]:
    """Uneven batch: d ~ U{2..20}, n ~ U[200, 2000], l ~ U[32, l_max]; mu = N(0, I_d),
    nu = N(1_d, diag(0.5, 2, 0.5, ...)); filling uniform on [-3,3]^{2d};
    sigma = s * median distance with s cycling over {0.5, 1, 2}; lambda1 = 1e-3, lambda2 = 1/n."""
    out = []
    for b in range(count):
        rng = np.random.default_rng(base_seed + b)
        d = int(rng.integers(2, 21))
        n = int(rng.integers(200, 2001))
        l = int(rng.integers(32, l_max + 1))
        var = np.where(np.arange(d) % 2 == 0, 0.5, 2.0)
        X = rng.standard_normal((n, d))
        Y = 1.0 + rng.standard_normal((n, d)) * np.sqrt(var)
        Fp = rng.uniform(-3, 3, size=(l, 2 * d))
        s = (0.5, 1.0, 2.0)[b % 3]
        sigma = s * median_distance(np.concatenate([X, Y]))
        out.append(Problem(f"uneven_{b}", X, Y, Fp[:, :d].copy(), Fp[:, d:].copy(), sigma,
                           1e-3, 1.0 / n))
    return out


def paper_regime(seed: int = 0, d: int = 5, n: int = 1000, l: int = 300,
                 sigma2: float = 0.005, name: str | None = None) -> Problem:
    """The synthetic regime of Sec. 5: mu a mixture of 3 and nu a mixture of 5 d-dimensional
    Gaussians, filling points uniform on the unit cube [0,1]^{2d}, bandwidth sigma^2 = 0.005,
    lambda1 = 1/l and lambda2 = 1/sqrt(n). Component means are uniform in [0.2, 0.8]^d with
    standard deviation 0.08 and equal weights (the paper does not print them)."""
    rng = np.random.default_rng(seed)

    def mixture(k, m):
        means = rng.uniform(0.2, 0.8, size=(k, d))
        comp = rng.integers(0, k, size=m)
        return means[comp] + 0.08 * rng.standard_normal((m, d))

    X = mixture(3, n)
    Y = mixture(5, n)
    Fp = rng.uniform(0.0, 1.0, size=(l, 2 * d))
    return Problem(name or f"paper_regime_d{d}_n{n}_l{l}", X, Y, Fp[:, :d].copy(),
                   Fp[:, d:].copy(), float(np.sqrt(sigma2)), 1.0 / l, 1.0 / np.sqrt(n))


def paper_regime_batch(count: int = 256, base_seed: int = 5000, l_max: int = 512) -> list[Problem]:
    """Uneven batch in the Sec. 5 regime with the size ranges of the batched configuration:
    d ~ U{2..20}, n ~ U[200, 2000], l ~ U[32, l_max]; problem b is paper_regime(seed base+b)."""
    out = []
    for b in range(count):
        rng = np.random.default_rng(base_seed + b)
        d = int(rng.integers(2, 21))
        n = int(rng.integers(200, 2001))
        l = int(rng.integers(32, l_max + 1))
        out.append(paper_regime(seed=base_seed + b, d=d, n=n, l=l, name=f"paper_batch_{b}"))
    return out


def by_name(name: str) -> Problem:
    """Named workloads: 'd2_n100_l50', 'd5_n1000_l300', 'd10_n2000_l1024', 'd64_n4000_l2048'."""
    table = {
        "d2_n100_l50": gaussian_pair,
        "d5_n1000_l300": wishart_pair,
        "d10_n2000_l1024": mixture_rotation,
        "d64_n4000_l2048": feature_like,
    }
    return table[name]()


def bootstrap_resamples(p: Problem, count: int, seed: int):
    """`count` bootstrap resamples of the samples of p, drawn with replacement (X and Y
    independently, each of size n), the filling points kept: the bootstrap setting in which Q, K
    and R are shared.  Returns (Xs, Ys), each count x n x d."""
    rng = np.random.default_rng(seed)
    n = p.n
    ix = rng.integers(0, n, size=(count, n))
    iy = rng.integers(0, n, size=(count, n))
    return np.ascontiguousarray(p.X[ix]), np.ascontiguousarray(p.Y[iy])


def clustered_symmetric(l: int, seed: int, clusters: int = 6, width: float = 1e-9) -> np.ndarray:
    """Symmetric l x l matrix whose eigenvalues sit half in a few tight clusters of both signs
    (width `width`) and half spread over [-1, 1], in a random orthogonal basis: the kind of
    spectrum the matrices Z = X - Phi*(gamma) - lambda1 I of an SSN solve have (many gaps below
    1e-6 ||Z||, eigenvalues on both sides of zero)."""
    rng = np.random.default_rng(seed)
    centers = rng.uniform(-1.0, 1.0, clusters)
    lam = np.where(rng.random(l) < 0.5, centers[rng.integers(0, clusters, l)]
                   + width * rng.standard_normal(l), rng.uniform(-1.0, 1.0, l))
    Qm, _ = np.linalg.qr(rng.standard_normal((l, l)))
    Z = (Qm * lam) @ Qm.T
    return 0.5 * (Z + Z.T)


def separated_symmetric(l: int, seed: int) -> np.ndarray:
    """Symmetric l x l matrix with eigenvalues about 2/l apart over [-1, 1] in a random orthogonal
    basis: no clusters, the easy case of a cold eigen-decomposition."""
    rng = np.random.default_rng(seed)
    lam = -1.0 + 2.0 * (np.arange(l) + 0.25 * rng.random(l)) / l
    Qm, _ = np.linalg.qr(rng.standard_normal((l, l)))
    Z = (Qm * lam) @ Qm.T
    return 0.5 * (Z + Z.T)
