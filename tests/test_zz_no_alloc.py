"""The allocation-free entry point kot_embedding_sqnorm_noalloc, called through the C ABI.

It serves callers that may not allocate device memory while they run (for example code inside
a custom device allocator, or a process that reserved its device memory up front).  Each call
must give ||w||^2 = (1/n^2) sum_ij k(s_i, s_j) of one sample set -- the oracle's
embedding_sqnorm, one half of q2 -- within the feature tolerance of the other parity tests, on
two calls in a row (the calls share one fixed device array of partial sums), and the two halves
must add up to the q2 that kot_build_features assembles.
"""
import ctypes

import numpy as np
import pytest

from oracle import kot_oracle as ko
from paper_2310_14087_gb300 import _build, kot, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU-only machines
    pytest.skip("needs a CUDA device", allow_module_level=True)

DEV = "cuda:0"


def _noalloc_fn():
    _build.build()
    f = kot.lib().kot_embedding_sqnorm_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p,
                  ctypes.c_void_p]
    return f


def _T(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=DEV)


@pytest.mark.parametrize("n,d,l", [(1000, 5, 300), (333, 3, 40)])
def test_noalloc_matches_oracle_twice(n, d, l):
    f = _noalloc_fn()
    p = workloads.paper_regime(seed=7, d=d, n=n, l=l)
    X, Y, Xf, Yf = _T(p.X), _T(p.Y), _T(p.Xf), _T(p.Yf)
    ref = (ko.embedding_sqnorm(p.X, p.sigma), ko.embedding_sqnorm(p.Y, p.sigma))
    out = torch.full((2,), float("nan"), dtype=torch.float64, device=DEV)
    stream = torch.cuda.current_stream(DEV).cuda_stream
    for _ in range(2):
        out.fill_(float("nan"))
        torch.cuda.synchronize()
        assert f(n, d, X.data_ptr(), p.sigma, out.data_ptr(), stream) == kot.OK
        assert f(n, d, Y.data_ptr(), p.sigma, out.data_ptr() + 8, stream) == kot.OK
        got = out.cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=1e-13)
    # the two halves add up to the q2 that the feature assembly keeps
    with kot.Context(device=0) as ctx:
        ctx.build_features(X, Y, Xf, Yf, p.sigma, p.lambda1, p.lambda2)
        q2 = torch.zeros(1, dtype=torch.float64, device=DEV)
        ctx.get_features(q2=q2)
    assert float(out.sum().item()) == pytest.approx(float(q2.item()), rel=1e-13)


def test_noalloc_full_capacity_distinct_samples():
    # n = 4096 fills all 64 x 64 tiles of the fixed array; distinct random samples make every
    # partial sum different, so a tile that were skipped or read twice would show
    f = _noalloc_fn()
    rng = np.random.default_rng(11)
    S = rng.standard_normal((4096, 3)) * np.array([0.5, 1.0, 2.0])
    sigma = 0.9
    ref = ko.embedding_sqnorm(S, sigma)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device=DEV)
    for _ in range(2):
        out.fill_(float("nan"))
        torch.cuda.synchronize()
        assert f(4096, 3, _T(S).data_ptr(), sigma, out.data_ptr(), None) == kot.OK
        assert float(out.item()) == pytest.approx(ref, rel=1e-13)


def test_noalloc_rejects_sizes_above_capacity():
    f = _noalloc_fn()
    X = torch.zeros((4097, 2), dtype=torch.float64, device=DEV)
    out = torch.zeros(1, dtype=torch.float64, device=DEV)
    assert f(4097, 2, X.data_ptr(), 1.0, out.data_ptr(), None) == kot.ERR_TOO_LARGE
    assert f(4096, 2, X.data_ptr(), -1.0, out.data_ptr(), None) == kot.ERR_INVALID
    assert f(4096, 2, X.data_ptr(), 1.0, out.data_ptr(), None) == kot.OK
    assert float(out.item()) == pytest.approx(1.0, rel=1e-15)   # identical samples: k = 1
