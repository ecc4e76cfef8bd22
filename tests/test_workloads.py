"""The seeded input recipes (paper_2310_14087_gb300/workloads.py) against the properties their
docstrings state: the shapes and regimes of the paper's Sec. 5 experiments and the spectra of the
eigensolver benchmarks.  CPU only."""
import numpy as np

from paper_2310_14087_gb300 import workloads as wl


def test_paper_regime_shapes_and_constants():
    # Sec. 5: sigma^2 = 0.005, lambda1 = 1/l, lambda2 = 1/sqrt(n), filling points uniform on [0,1]^2d
    p = wl.paper_regime(seed=3, d=5, n=200, l=40)
    assert p.X.shape == (200, 5) and p.Y.shape == (200, 5)
    assert p.Xf.shape == (40, 5) and p.Yf.shape == (40, 5)
    assert abs(p.sigma ** 2 - 0.005) < 1e-15
    assert p.Xf.min() >= 0.0 and p.Xf.max() <= 1.0 and p.Yf.min() >= 0.0 and p.Yf.max() <= 1.0
    assert abs(p.lambda1 - 1.0 / 40) < 1e-15 and abs(p.lambda2 - 1.0 / np.sqrt(200)) < 1e-15
    q = wl.paper_regime(seed=3, d=5, n=200, l=40)
    assert np.array_equal(p.X, q.X) and np.array_equal(p.Yf, q.Yf)   # seeded


def test_uneven_batch_ranges():
    probs = wl.paper_regime_batch(count=24, base_seed=11)
    assert len(probs) == 24
    for p in probs:
        assert 2 <= p.d <= 20 and 200 <= p.n <= 2000 and 32 <= p.l <= 512


def test_separated_spectrum():
    l = 64
    Z = wl.separated_symmetric(l, seed=5)
    assert np.array_equal(Z, Z.T)
    lam = np.linalg.eigvalsh(Z)
    gaps = np.diff(lam)
    assert lam.min() > -1.0 - 1e-12 and lam.max() < 1.0 + 1e-12
    assert gaps.min() > 1.0 / l and gaps.max() < 3.0 / l


def test_clustered_spectrum():
    l = 200
    Z = wl.clustered_symmetric(l, seed=7, clusters=6, width=1e-9)
    assert np.array_equal(Z, Z.T)
    lam = np.linalg.eigvalsh(Z)
    # about half the eigenvalues sit in clusters: many gaps below 1e-7
    assert np.sum(np.diff(lam) < 1e-7) > l // 4
    assert np.abs(lam).max() <= 1.0 + 1e-9
