"""Symmetric eigen-decomposition kot_eig_sym (the decomposition behind the PSD projection of
Eq. (4.4) and the Omega weights of Sec. 4.2) against the oracle's eigendecomposition.

Both paths are covered: Jacobi sweeps from the identity (no warm basis) and refinement of a
warm basis (the eigenbasis of a nearby matrix, as the SSN iteration hands in), including the
fall-back from a refinement that cannot converge (a basis far from the answer, or exactly
repeated eigenvalues) to Jacobi sweeps.  Every result must be an FP64-accurate decomposition:
eigenvalues within 1e-13 ||Z|| of the oracle's, eigen-residual ||Z P - P diag(sig)||_F and
||P^T P - I||_max at FP64 rounding level, and the projection Pi_{S+}(Z) within 1e-13 ||Z||.
"""
import numpy as np
import pytest

from oracle import kot_oracle as ko
from paper_2310_14087_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU-only machines
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2310_14087_gb300 import kot  # noqa: E402

DEV = "cuda:0"


def clustered_symmetric(l, seed, clusters=6, width=1e-9):
    """Clustered spectrum of both signs in a random orthogonal basis (workloads.clustered_symmetric)."""
    return wl.clustered_symmetric(l, seed, clusters, width)


def separated_symmetric(l, seed):
    """Symmetric l x l matrix with eigenvalues about 2/l apart in a random orthogonal basis."""
    return wl.separated_symmetric(l, seed)


def run_eig(ctx, Z, warm=None):
    l = Z.shape[0]
    P = torch.zeros((l, l), dtype=torch.float64, device=DEV)
    sig = torch.zeros(l, dtype=torch.float64, device=DEV)
    info = ctx.eig_sym(l, torch.as_tensor(Z, device=DEV),
                       None if warm is None else torch.as_tensor(warm, device=DEV), P, sig)
    return P.cpu().numpy(), sig.cpu().numpy(), info


def check_decomposition(Z, P, sig):
    ref = ko.eig_sym(Z)
    nz = max(np.abs(ref.sig).max(), 1e-300)
    l = Z.shape[0]
    # FP64 accuracy of an orthogonal similarity of an l x l matrix: the backward error of a
    # decomposition built from rotations (or Householder steps, for the oracle's LAPACK) grows like
    # l u ||Z||; u l = 1e-16 l, with the 1e-13 floor of the smaller sizes
    tol = max(1e-13, 1e-16 * l)
    assert np.all(np.diff(sig) >= 0)
    assert np.abs(sig - ref.sig).max() <= tol * nz
    assert np.linalg.norm(Z @ P - P * sig[None, :]) <= tol * nz * np.sqrt(l)
    assert np.abs(P.T @ P - np.eye(l)).max() <= tol
    proj = (P * np.maximum(sig, 0.0)) @ P.T
    assert np.abs(proj - ko.proj_psd_from_eig(ref)).max() <= tol * nz


@pytest.mark.parametrize("l", [1, 2, 37, 64, 129, 160, 300, 512, 1024, 2048])
def test_cold_start_jacobi(l):
    # random eigenbasis: from l = 37 up the refinement from the identity gives up at once and
    # Jacobi sweeps decompose; at l = 1 (already diagonal) and l = 2 the refinement may finish
    Z = clustered_symmetric(l, seed=l)
    ctx = kot.Context(device=0)
    P, sig, (sweeps, refine) = run_eig(ctx, Z)
    if l >= 37:
        assert refine == 0 and sweeps > 0
    else:
        assert (refine > 0 and sweeps == 0) or (refine == 0 and sweeps > 0)
    check_decomposition(Z, P, sig)


@pytest.mark.parametrize("l", [37, 100, 160, 161])
def test_cold_start_small_l_uses_the_shared_memory_fp32_basis(l):
    # separated spectrum in a random basis: up to l = 160 the shared-memory FP32 Jacobi supplies a
    # basis that the FP64 refinement finishes (no FP64 sweep); above it the cooperative sweeps run
    Z = separated_symmetric(l, seed=7 * l)
    ctx = kot.Context(device=0)
    P, sig, (sweeps, refine) = run_eig(ctx, Z)
    if l <= 160:
        assert sweeps == 0 and 1 <= refine <= 5
    else:
        assert refine == 0 and sweeps > 0
    check_decomposition(Z, P, sig)


@pytest.mark.parametrize("l,delta", [(50, 1e-3), (300, 1e-4), (513, 1e-5)])
def test_cold_start_nearly_diagonal_refines_from_identity(l, delta):
    # separated diagonal plus a small symmetric perturbation (|E| ~ delta / gap << 1): without a
    # warm basis the refinement starts from the identity and needs no Jacobi sweep
    rng = np.random.default_rng(5 * l)
    d = np.linspace(-1.0, 1.0, l)[rng.permutation(l)]
    Dm = rng.standard_normal((l, l))
    Z = np.diag(d) + delta * 0.5 * (Dm + Dm.T) / np.sqrt(l)
    ctx = kot.Context(device=0)
    P, sig, (sweeps, refine) = run_eig(ctx, Z)
    assert sweeps == 0 and 1 <= refine <= 5
    check_decomposition(Z, P, sig)


@pytest.mark.parametrize("l,delta", [(64, 1e-9), (300, 1e-6), (300, 1e-4), (513, 1e-7)])
def test_warm_basis_is_refined(l, delta):
    # perturbation well inside the first-order regime (|E| = |dZ_ij| / gap << 1)
    Z0 = separated_symmetric(l, seed=3 * l)
    rng = np.random.default_rng(l)
    Dm = rng.standard_normal((l, l))
    Z = Z0 + delta * 0.5 * (Dm + Dm.T) / np.sqrt(l)
    warm = ko.eig_sym(Z0).P
    ctx = kot.Context(device=0)
    P, sig, (sweeps, refine) = run_eig(ctx, Z, warm)
    assert sweeps == 0 and 1 <= refine <= 5
    check_decomposition(Z, P, sig)


@pytest.mark.parametrize("delta", [1e-12, 1e-6])
def test_clustered_spectrum_either_path_is_exact(delta):
    # eigenvalue clusters 1e-7 wide: a random perturbation mixes each cluster, so the refinement
    # may have to give up; whichever path finishes, the decomposition must be FP64-accurate
    l = 240
    Z0 = clustered_symmetric(l, seed=8, width=1e-7)
    rng = np.random.default_rng(9)
    Dm = rng.standard_normal((l, l))
    Z = Z0 + delta * 0.5 * (Dm + Dm.T) / np.sqrt(l)
    ctx = kot.Context(device=0)
    P, sig, (sweeps, refine) = run_eig(ctx, Z, ko.eig_sym(Z0).P)
    assert refine == 0 or sweeps == 0
    check_decomposition(Z, P, sig)


def test_warm_bases_along_an_oracle_solve():
    # the matrices Z of one Algorithm 2 run, each decomposed from the eigenbasis of the matrix
    # four calls earlier (the same evaluation of the previous iteration)
    from paper_2310_14087_gb300 import workloads as wl
    p = wl.paper_regime(2, d=2, n=100, l=50)
    F = ko.build_features(p.X, p.Y, p.Xf, p.Yf, p.sigma, p.lambda1, p.lambda2)
    calls = []
    orig = ko.eig_sym
    try:
        ko.eig_sym = lambda Zm: (calls.append(Zm.copy()) or orig(Zm))
        ko.ssn_solve(F, 1e-6, ko.Options())
    finally:
        ko.eig_sym = orig
    ctx = kot.Context(device=0)
    refined = 0
    for k in range(5, len(calls)):
        P, sig, (sweeps, refine) = run_eig(ctx, calls[k], orig(calls[k - 4]).P)
        refined += refine > 0
        check_decomposition(calls[k], P, sig)
    assert refined > 0


def test_far_basis_falls_back_to_jacobi():
    l = 200
    Z = clustered_symmetric(l, seed=11)
    warm, _ = np.linalg.qr(np.random.default_rng(12).standard_normal((l, l)))
    ctx = kot.Context(device=0)
    P, sig, (sweeps, refine) = run_eig(ctx, Z, warm)
    assert refine == 0 and sweeps > 0
    check_decomposition(Z, P, sig)


def test_repeated_eigenvalue():
    # Z = -lambda1 I (the first matrix of every solve): all Rayleigh quotients agree to
    # rounding, so the refinement's divisions are of rounding noise by rounding noise (or 0/0)
    # and it must hand over to Jacobi -- or, should every E_ij come out small, still return an
    # orthonormal basis, which is an eigenbasis of a multiple of I.
    l = 96
    Z = -1e-3 * np.eye(l)
    warm, _ = np.linalg.qr(np.random.default_rng(5).standard_normal((l, l)))
    ctx = kot.Context(device=0)
    P, sig, (sweeps, refine) = run_eig(ctx, Z, warm)
    assert refine == 0 or sweeps == 0
    assert np.abs(sig + 1e-3).max() <= 1e-17
    assert np.abs(P.T @ P - np.eye(l)).max() <= 1e-13


def test_refinement_off_uses_jacobi_from_warm_basis():
    l = 150
    Z0 = separated_symmetric(l, seed=21)
    Z = Z0 + 1e-6 * np.diag(np.linspace(-1, 1, l))
    warm = ko.eig_sym(Z0).P
    ctx = kot.Context(device=0, eig_refine=0)
    P, sig, (sweeps, refine) = run_eig(ctx, Z, warm)
    assert refine == 0 and sweeps >= 1
    check_decomposition(Z, P, sig)


def test_host_pointer_mode():
    l = 77
    Z0 = separated_symmetric(l, seed=77)
    Z = Z0 + 1e-7 * np.eye(l) * np.arange(l)
    warm = ko.eig_sym(Z0).P
    ctx = kot.Context(device=0, host_pointers=1)
    P = np.zeros((l, l))
    sig = np.zeros(l)
    sweeps, refine = ctx.eig_sym(l, np.ascontiguousarray(Z), np.ascontiguousarray(warm), P, sig)
    assert refine >= 1
    check_decomposition(Z, P, sig)


def test_solve_uses_refinement_and_matches_jacobi_only():
    # the same problem solved with and without refinement reaches the same optimum
    from paper_2310_14087_gb300 import workloads as wl
    p = wl.paper_regime(2, d=2, n=100, l=50)
    out = {}
    for refine in (5, 0):
        ctx = kot.Context(device=0, eig_refine=refine)
        t = lambda a: torch.as_tensor(a, device=DEV)
        ctx.build_features(t(p.X), t(p.Y), t(p.Xf), t(p.Yf), p.sigma, p.lambda1, p.lambda2)
        g = torch.zeros(p.l, dtype=torch.float64, device=DEV)
        out[refine] = ctx.ssn_solve(1e-6, g)
    r5, r0 = out[5], out[0]
    assert r5.status == kot.OK and r0.status == kot.OK
    assert r5.eig_refined > 0
    assert r0.eig_refined == 0
    assert abs(r5.objective - r0.objective) <= 1e-6 * abs(r0.objective)
