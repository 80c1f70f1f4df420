"""NAF basis (Sec. 2: eigenpairs of K = B B^T above the threshold) through the
C ABI, FP64 and mixed forms, at sizes that take every path of the fused
Householder reduction: a single block, rows held in shared memory, rows
reduced in place in global memory (FP64 beyond about 1820 rows, FP32 beyond
about 2720), and one or several warps per row.

Checked against the oracle's eigendecomposition (numpy) through quantities
that do not depend on the free sign and rotation of the eigenvectors: the kept
eigenvalues, the residual |K u - lambda u|, orthonormality and (FP64) the
projector onto the kept subspace.  The threshold sits in the middle of a wide
gap, so both sides keep the same count.
"""
import numpy as np
import pytest

from oracle import ltgw_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2307_04508_gb300 import ltgw
    c = ltgw.Context(0)
    yield c
    c.close()


def _case(n: int, seed: int, pairs: int = 0):
    """B (n x pairs, default 2n) with an exponentially decaying spectrum of
    K (like the RI workloads) and a threshold in the widest gap among the top
    20-50 % of eigenvalues."""
    rng = np.random.default_rng(seed)
    pairs = pairs or 2 * n
    B = rng.standard_normal((n, pairs)) / np.sqrt(pairs)
    B *= np.exp(-3.0 * np.arange(n) / n)[:, None]
    K = B @ B.T
    lam = np.sort(np.linalg.eigvalsh(K))[::-1]
    lo, hi = (0, n - 1) if n < 10 else (int(0.2 * n), int(0.5 * n))
    gaps = lam[lo:hi] - lam[lo + 1:hi + 1]
    m = lo + int(np.argmax(gaps))
    return np.ascontiguousarray(B), K, 0.5 * (lam[m] + lam[m + 1])


@pytest.mark.parametrize("mixed,n", [(False, 3), (False, 4), (False, 5), (False, 33), (False, 150),
                                     (False, 1800), (False, 1900),
                                     (True, 3), (True, 5), (True, 150), (True, 1800), (True, 2800)])
def test_naf_basis_paths(ctx, mixed, n):
    B, K, thr = _case(n, 1000 + n)
    U_ref, lam_kept, lam_all = O.naf_basis(K, thr)
    Ut = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    lam = torch.zeros(n, dtype=torch.float64, device="cuda")
    k = ctx.naf_basis(torch.from_numpy(B).cuda(), 2 * n, 2 * n, thr, Ut, lam, mixed=mixed)
    assert k == U_ref.shape[1]
    U = Ut[:k].cpu().numpy().T
    lg = lam[:k].cpu().numpy()
    lmax = lam_all.max()
    # the mixed form builds K from split-BF16 products: errors of a few 1e-6 * lambda_max
    tol_lam, tol_res, tol_orth = (2e-5, 2e-5, 1e-5) if mixed else (1e-13, 1e-12, 1e-12)
    assert np.all(np.diff(lg) <= 0.0), "eigenvalues must come out descending"
    assert np.abs(lg - lam_kept[::-1]).max() <= tol_lam * lmax
    res = np.linalg.norm(K @ U - U * lg[None, :], axis=0).max()
    assert res <= tol_res * lmax
    assert np.abs(U.T @ U - np.eye(k)).max() <= tol_orth
    if not mixed:
        assert np.abs(U @ U.T - U_ref @ U_ref.T).max() <= 1e-10


def test_naf_basis_mixed_multidrain(ctx):
    """140,000 pairs: more K-splits than a launch takes, so every CTA of the
    metric drains its FP32 accumulators twice (alternating accumulator sets);
    the result must match the single-drain accuracy."""
    n, P = 130, 140000
    B, K, thr = _case(n, 77, P)
    U_ref, lam_kept, lam_all = O.naf_basis(K, thr)
    Ut = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    lam = torch.zeros(n, dtype=torch.float64, device="cuda")
    k = ctx.naf_basis(torch.from_numpy(B).cuda(), P, P, thr, Ut, lam, mixed=True)
    assert k == U_ref.shape[1]
    lg = lam[:k].cpu().numpy()
    assert np.abs(lg - lam_kept[::-1]).max() <= 2e-5 * lam_all.max()
    U = Ut[:k].cpu().numpy().T
    assert np.linalg.norm(K @ U - U * lg[None, :], axis=0).max() <= 2e-5 * lam_all.max()
