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
                        (16, 16, 1, 0, 1), (513, 511, 1025, 0, 0),
                        # K <= 64 with op(B) given as N x K rows: the one-pass short-K kernel
                        # (ragged 32 x 32 tiles, K = 1 and K = 64), and K = 65 just past it
                        (300, 300, 18, 0, 0), (33, 65, 64, 0, 0), (257, 31, 63, 0, 0),
                        (1, 700, 40, 0, 0), (700, 1, 1, 0, 0), (97, 97, 65, 0, 0)]


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


# ---------------------------------------------------------------- FP64 emulation (pieces = -s)
# Every row of op(A) / op(B) is cut into s fixed-point BF16 slices relative to its largest
# magnitude; slice products of level < s are summed exactly in FP32 and combined in float-float.
# Bound per element (slicing error 2^-(8s) of the row maximum per value, dropped levels, and the
# float-float combination, ~2^-47 of the partial sums):
#   |err| <= (2^(6 - 8 s) + 2^-44) K max_k|A(r,k)| max_k|B(c,k)| + FP64 rounding of the beta term.
EMU_SHAPES = [(300, 300, 300, 0, 1, 6), (300, 300, 300, 1, 0, 6), (1, 7, 5, 0, 0, 6),
              (257, 130, 513, 1, 0, 6), (64, 300, 97, 1, 1, 7), (513, 511, 1025, 0, 0, 6),
              (16, 16, 1, 0, 1, 3), (1024, 1024, 1024, 0, 0, 6), (129, 257, 2100, 0, 1, 8),
              (300, 22, 300, 1, 1, 4),
              # 128 x 128 output tiles (M, N >= 512), ragged edges and both transposes
              (600, 700, 900, 1, 0, 6), (1000, 513, 300, 0, 1, 3), (520, 1030, 64, 1, 1, 7)]


@pytest.mark.parametrize("M,N,K,ta,tb,s", EMU_SHAPES)
def test_emulated_fp64_product(M, N, K, ta, tb, s):
    rng = np.random.default_rng(11 * M + 13 * N + K + s)
    A = rng.standard_normal((K, M) if ta else (M, K))
    B = rng.standard_normal((K, N) if tb else (N, K))
    # rows of very different magnitude (the slicing is relative to each row's maximum)
    A *= np.exp2(rng.integers(-30, 30, size=(1, M) if ta else (M, 1)))
    lda, ldb = A.shape[1], B.shape[1]
    ctx = kot.Context(device=0)
    C0 = rng.standard_normal((M, N))
    Cm = torch.as_tensor(C0.copy(), device=DEV)
    ctx.dense_product(M, N, K, -0.75, torch.as_tensor(A, device=DEV), lda, ta,
                      torch.as_tensor(B, device=DEV), ldb, tb, 0.5, Cm, N, pieces=-s)
    Al, Bl = op(A, ta), op(B, tb)
    ref = -0.75 * (Al @ Bl.T) + 0.5 * C0
    amax, bmax = np.abs(Al).max(axis=1), np.abs(Bl).max(axis=1)
    bound = ((2.0 ** (6 - 8 * s) + 2.0 ** -44) * K * 0.75 * np.outer(amax, bmax)
             + 4 * 2.0 ** -53 * (np.abs(ref) + 0.5 * np.abs(C0)) + 1e-300)
    err = np.abs(Cm.cpu().numpy() - ref)
    assert np.all(err <= bound), float((err / bound).max())


def test_emulated_fp64_integers_are_exact():
    # integer operands of 16 bits: two slices hold them exactly and every partial sum is an exact
    # FP32 integer (groups of <= 512 products), so the product must equal the exact integer one;
    # K = 2000 forces several accumulation groups per level and uneven tile edges
    rng = np.random.default_rng(5)
    M, N, K = 200, 190, 2000
    A = rng.integers(-30000, 30001, size=(M, K)).astype(np.float64)
    B = rng.integers(-30000, 30001, size=(N, K)).astype(np.float64)
    ctx = kot.Context(device=0)
    Cm = torch.zeros((M, N), dtype=torch.float64, device=DEV)
    ctx.dense_product(M, N, K, 1.0, torch.as_tensor(A, device=DEV), K, 0,
                      torch.as_tensor(B, device=DEV), K, 0, 0.0, Cm, N, pieces=-6)
    ref = A.astype(np.int64) @ B.astype(np.int64).T          # exact (|.| < 2^53)
    np.testing.assert_array_equal(Cm.cpu().numpy(), ref.astype(np.float64))


def test_emulated_fp64_rejects_bad_slices():
    ctx = kot.Context(device=0)
    x = torch.zeros((4, 4), dtype=torch.float64, device=DEV)
    for bad in (-1, -2, -9, 4):
        with pytest.raises(kot.KotError) as e:
            ctx.dense_product(4, 4, 4, 1.0, x, 4, 0, x, 4, 0, 0.0, x, 4, pieces=bad)
        assert e.value.status == kot.ERR_INVALID


def test_autotune_records_valid_choices():
    # the autotuner picks a split count per slice count and a Jacobi CTA count for the size
    # bucket; products and decompositions afterwards still meet their accuracy bounds
    ctx = kot.Context(device=0)
    s3, s6, ctas, w3, w6, threads = ctx.autotune(97)
    assert threads in (256, 512, 1024)
    assert s3 in (1, 2, 3, 4, 6, 8, 12, 16) and s6 in (1, 2, 3, 4, 6, 8, 12, 16)
    assert w3 in (64, 128) and w6 in (64, 128)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert ctas in (sms // 4, sms // 2, sms)
    rng = np.random.default_rng(1)
    M = N = K = 97
    A, B = rng.standard_normal((M, K)), rng.standard_normal((N, K))
    Cm = torch.zeros((M, N), dtype=torch.float64, device=DEV)
    ctx.dense_product(M, N, K, 1.0, torch.as_tensor(A, device=DEV), K, 0, torch.as_tensor(B, device=DEV),
                      K, 0, 0.0, Cm, N, pieces=-6)
    bound = (2.0 ** -42 + 2.0 ** -44) * K * np.outer(np.abs(A).max(1), np.abs(B).max(1))
    assert np.all(np.abs(Cm.cpu().numpy() - A @ B.T) <= bound)
    Zs = rng.standard_normal((M, M))
    Zs = Zs + Zs.T
    P, sig = torch.zeros((M, M), dtype=torch.float64, device=DEV), torch.zeros(M, dtype=torch.float64, device=DEV)
    ctx.eig_sym(M, torch.as_tensor(Zs, device=DEV), None, P, sig)
    np.testing.assert_allclose(sig.cpu().numpy(), np.linalg.eigvalsh(Zs), atol=1e-12 * np.abs(Zs).max() * M)
    with pytest.raises(kot.KotError) as e:
        ctx.autotune(0)
    assert e.value.status == kot.ERR_INVALID


def test_bounded_wait_gives_up_with_a_status():
    # failure detection without a fault: a kernel waits on an mbarrier nothing completes, with the
    # bounded poll of the tensor-core pipelines; it gives up (here after ~10^5 polls), the call
    # returns KOT_ERR_TIMEOUT, and the context keeps working
    ctx = kot.Context(device=0)
    assert ctx.wait_probe(100000) == kot.ERR_TIMEOUT
    assert "probe" in ctx.last_error()
    x = torch.ones((8, 8), dtype=torch.float64, device=DEV)
    c = torch.zeros((8, 8), dtype=torch.float64, device=DEV)
    ctx.dense_product(8, 8, 8, 1.0, x, 8, 0, x, 8, 0, 0.0, c, 8, pieces=-6)
    assert torch.all(c == 8.0)
    assert ctx.wait_probe(0) == kot.ERR_INVALID
