"""The allocation-free entry point kot_embedding_sqnorm_noalloc, called through the C ABI.

It serves callers that may not allocate device memory while they run (for example code inside
a custom device allocator, or a process that reserved its device memory up front).  Its result
must equal the embedding norms that kot_build_features folds into q2 = ||w_mu||^2 + ||w_nu||^2,
read back with kot_get_features, within the feature tolerance of the other parity tests, on two
calls in a row (the calls share one fixed device array of partial sums).
"""
import ctypes

import numpy as np
import pytest

from paper_2310_14087_gb300 import _build, kot, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU-only machines
    pytest.skip("needs a CUDA device", allow_module_level=True)


def _noalloc_fn():
    _build.build()
    f = kot.lib().kot_embedding_sqnorm_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p,
                  ctypes.c_void_p]
    return f


@pytest.mark.parametrize("n,d,l", [(1000, 5, 300), (333, 3, 40)])
def test_noalloc_matches_feature_assembly_twice(n, d, l):
    f = _noalloc_fn()
    p = workloads.paper_regime(seed=7, d=d, n=n, l=l)
    dev = "cuda:0"
    T = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)
    X, Y, Xf, Yf = T(p.X), T(p.Y), T(p.Xf), T(p.Yf)
    with kot.Context(device=0) as ctx:
        ctx.build_features(X, Y, Xf, Yf, p.sigma, p.lambda1, p.lambda2)
        q2 = torch.zeros(1, dtype=torch.float64, device=dev)
        ctx.get_features(q2=q2)
    expect = float(q2.item())
    out = torch.full((2,), float("nan"), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    for _ in range(2):
        out.fill_(float("nan"))
        torch.cuda.synchronize()
        assert f(n, d, X.data_ptr(), p.sigma, out.data_ptr(), stream) == kot.OK
        assert f(n, d, Y.data_ptr(), p.sigma, out.data_ptr() + 8, stream) == kot.OK
        got = float(out.sum().item())
        assert got == pytest.approx(expect, rel=1e-13)


def test_noalloc_rejects_sizes_above_capacity():
    f = _noalloc_fn()
    X = torch.zeros((4097, 2), dtype=torch.float64, device="cuda:0")
    out = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    assert f(4097, 2, X.data_ptr(), 1.0, out.data_ptr(), None) == kot.ERR_TOO_LARGE
    assert f(4096, 2, X.data_ptr(), -1.0, out.data_ptr(), None) == kot.ERR_INVALID
    assert f(4096, 2, X.data_ptr(), 1.0, out.data_ptr(), None) == kot.OK
    assert float(out.item()) == pytest.approx(1.0, rel=1e-15)   # identical samples: k = 1
