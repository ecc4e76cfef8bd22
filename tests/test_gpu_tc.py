"""Tensor-core (tcgen05) dense product kot_dense_product against FP64 references.

With one BF16 piece the kernel must reproduce the product of the BF16-rounded inputs up to the
FP32 accumulation error (|err| <= K * 2^-23 * (|A_b| |B_b|^T) element-wise); any mistake in the
TMA tiling, the swizzle or the MMA descriptors breaks that bound by orders of magnitude.  With
three pieces the product must match the FP64 product to about FP32 accuracy.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU-only machines
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2310_14087_gb300 import kot  # noqa: E402

DEV = "cuda:0"


def bf16_round(x):
    return torch.as_tensor(x).to(torch.float32).to(torch.bfloat16).to(torch.float64).numpy()


def op(X, trans):
    return X.T if trans else X


SHAPES = [(128, 128, 64, 0, 0), (300, 300, 300, 0, 1), (1, 7, 5, 0, 0), (257, 130, 513, 1, 0),
          (64, 300, 97, 1, 1), (129, 257, 1000, 0, 1)]


@pytest.mark.parametrize("M,N,K,ta,tb", SHAPES)
def test_one_piece_equals_bf16_product(M, N, K, ta, tb):
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = rng.standard_normal((K, M) if ta else (M, K))
    B = rng.standard_normal((K, N) if tb else (N, K))
    lda, ldb = A.shape[1], B.shape[1]
    ctx = kot.Context(device=0)
    Cm = torch.zeros((M, N), dtype=torch.float64, device=DEV)
    ctx.dense_product(M, N, K, 1.0, torch.as_tensor(A, device=DEV), lda, ta,
                      torch.as_tensor(B, device=DEV), ldb, tb, 0.0, Cm, N, pieces=1)
    Ab, Bb = op(bf16_round(A), ta), op(bf16_round(B), tb)
    ref = Ab @ Bb.T
    bound = K * 2.0 ** -23 * (np.abs(Ab) @ np.abs(Bb).T) + 1e-300
    err = np.abs(Cm.cpu().numpy() - ref)
    assert np.all(err <= bound), float((err / bound).max())


@pytest.mark.parametrize("M,N,K,ta,tb", SHAPES)
def test_three_pieces_match_fp64(M, N, K, ta, tb):
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal((K, M) if ta else (M, K))
    B = rng.standard_normal((K, N) if tb else (N, K))
    lda, ldb = A.shape[1], B.shape[1]
    ctx = kot.Context(device=0)
    C0 = rng.standard_normal((M, N))
    Cm = torch.as_tensor(C0.copy(), device=DEV)
    ctx.dense_product(M, N, K, 0.5, torch.as_tensor(A, device=DEV), lda, ta,
                      torch.as_tensor(B, device=DEV), ldb, tb, -2.0, Cm, N, pieces=3)
    ref = 0.5 * (op(A, ta) @ op(B, tb).T) - 2.0 * C0
    scale = 0.5 * (np.abs(op(A, ta)) @ np.abs(op(B, tb)).T) + 2.0 * np.abs(C0)
    err = np.abs(Cm.cpu().numpy() - ref)
    assert np.all(err <= 4e-6 * scale * np.sqrt(K / 64 + 1)), float((err / scale).max())


FP64_SHAPES = SHAPES + [(300, 300, 300, 1, 0), (22, 300, 300, 1, 0), (300, 300, 22, 0, 0),
                        (16, 16, 1, 0, 1), (513, 511, 1025, 0, 0)]


@pytest.mark.parametrize("M,N,K,ta,tb", FP64_SHAPES)
def test_fp64_product(M, N, K, ta, tb):
    # pieces = 0: the FP64 stream-K GEMM; error within the classical dot-product bound
    # |err| <= (K + 2) u (|A||B| + |beta C|) with u = 2^-53
    rng = np.random.default_rng(3 * M + 5 * N + 7 * K)
    A = rng.standard_normal((K, M) if ta else (M, K))
    B = rng.standard_normal((K, N) if tb else (N, K))
    lda, ldb = A.shape[1], B.shape[1]
    ctx = kot.Context(device=0)
    C0 = rng.standard_normal((M, N))
    Cm = torch.as_tensor(C0.copy(), device=DEV)
    ctx.dense_product(M, N, K, 1.5, torch.as_tensor(A, device=DEV), lda, ta,
                      torch.as_tensor(B, device=DEV), ldb, tb, -0.5, Cm, N, pieces=0)
    Al, Bl = op(A, ta), op(B, tb)
    ref = 1.5 * (Al @ Bl.T) - 0.5 * C0
    bound = (K + 2) * 2.0 ** -53 * (1.5 * np.abs(Al) @ np.abs(Bl).T + 0.5 * np.abs(C0)) * 2 + 1e-300
    err = np.abs(Cm.cpu().numpy() - ref)
    assert np.all(err <= bound), float((err / bound).max())


def test_fp64_product_is_deterministic():
    rng = np.random.default_rng(0)
    M = N = K = 300
    A = torch.as_tensor(rng.standard_normal((M, K)), device=DEV)
    B = torch.as_tensor(rng.standard_normal((N, K)), device=DEV)
    ctx = kot.Context(device=0)
    outs = []
    for _ in range(3):
        Cm = torch.zeros((M, N), dtype=torch.float64, device=DEV)
        ctx.dense_product(M, N, K, 1.0, A, K, 0, B, K, 0, 0.0, Cm, N, pieces=0)
        outs.append(Cm.cpu().numpy())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
