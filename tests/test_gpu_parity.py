"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances (FP64 form): Pi relative Frobenius error <= 1e-11 (same mode on
both sides: direct vs direct, Laplace vs Laplace with the same grid), Sigma(i w)
relative max error <= 1e-11, quasi-particle energies within 1e-8 Ha.
NAF-basis quantities are compared through basis-invariant forms (U Pi U^T,
projectors), because the sign and rotation of each eigenvector are free.
"""
import numpy as np
import pytest

from oracle import ltgw_oracle as O
from paper_2307_04508_gb300 import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PI_TOL = 1e-11
SIG_TOL = 1e-11
QP_TOL = 1e-8


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2307_04508_gb300 import ltgw
    c = ltgw.Context(0)
    yield c
    c.close()


def _ltgw():
    from paper_2307_04508_gb300 import ltgw
    return ltgw


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _oracle(prob, n_omega, naf_thresh=-1.0, tau=None, spin=2):
    tx, tw = (None, None) if tau is None else tau
    return O.solve(prob.eps, prob.B_ov, prob.B_tgt, prob.targets, prob.shift, prob.n_occ, prob.n_virt,
                   prob.n_frozen, n_omega=n_omega, naf_thresh=naf_thresh, spin=spin, tau_x=tx, tau_w=tw,
                   return_all=True)


def _check_solve(ctx, prob, n_omega, naf_thresh=-1.0, tau=None, spin=2, device=False):
    L = _ltgw()
    sig_o, e_o, st_o, it = _oracle(prob, n_omega, naf_thresh, tau, spin)
    dev = None
    if device:
        dev = {"eps": _dev(prob.eps), "B_ov": _dev(prob.B_ov), "B_tgt": _dev(prob.B_tgt),
               "targets": _dev(prob.targets.astype(np.int32)), "shift": _dev(prob.shift)}
    sig_g, e_g, st_g = L.solve_problem(ctx, prob, n_omega=n_omega, n_tau=0 if tau is None else len(tau[0]),
                                       naf_thresh=naf_thresh, use_laplace=tau is not None, spin=spin, tau=tau,
                                       device_arrays=dev)
    assert np.all(st_o == 0) and np.all(st_g == 0)
    assert np.abs(sig_g - sig_o).max() <= SIG_TOL * np.abs(sig_o).max()
    assert np.abs(e_g - e_o).max() <= QP_TOL
    st = ctx.stats()
    assert st["n_naf"] == it["n_naf"]
    return st


# ------------------------------------------------------------------ whole path
def test_tiny_direct(ctx):
    _check_solve(ctx, S.make_workload(S.TINY), 24)


def test_tiny_direct_device_pointers(ctx):
    _check_solve(ctx, S.make_workload(S.TINY), 24, device=True)


def test_tiny_laplace_same_grid(ctx):
    tau = O.sinc_laplace_grid(6, -9.0, 2.0)
    _check_solve(ctx, S.make_workload(S.TINY), 24, tau=tau)


def test_tiny_naf_threshold_zero(ctx):
    _check_solve(ctx, S.make_workload(S.TINY), 24, naf_thresh=0.0)


@pytest.mark.parametrize("spin", [1, 2])
def test_ragged_frozen_naf(ctx, spin):
    # sizes off the 64-wide tiles: ragged tails in every contraction
    prob = S.make_problem(7, 45, 131, n_frozen=2, seed=4242, n_targets=4)
    _check_solve(ctx, prob, 21, naf_thresh=1e-3, spin=spin)


def test_ragged_laplace_naf(ctx):
    prob = S.make_problem(9, 70, 150, n_frozen=1, seed=99, n_targets=3)
    tau = O.sinc_laplace_grid(9, -11.0, 2.5)
    _check_solve(ctx, prob, 17, naf_thresh=5e-3, tau=tau)


def test_single_active_occupied(ctx):
    prob = S.make_problem(3, 30, 20, n_frozen=2, seed=7, n_targets=2)
    _check_solve(ctx, prob, 16)


def test_single_naf_function(ctx):
    prob = S.make_problem(4, 24, 40, n_frozen=0, seed=11, n_targets=2)
    K = prob.B_ov @ prob.B_ov.T
    lam = np.linalg.eigvalsh(K)
    thr = 0.5 * (lam[-1] + lam[-2])
    st = _check_solve(ctx, prob, 12, naf_thresh=thr)
    assert st["n_naf"] == 1


def test_mid_workload_direct(ctx):
    """Full mid-size workload: 60 occupied (10 frozen), 540 virtual, 1800
    auxiliary functions, NAF at 1e-2, 32 frequencies, 10 states."""
    _check_solve(ctx, S.make_workload(S.MID), 32, naf_thresh=1e-2, device=True)


def test_mid_workload_laplace(ctx):
    tau = O.sinc_laplace_grid(8, -12.0, 3.0)
    _check_solve(ctx, S.make_workload(S.MID), 32, naf_thresh=1e-2, tau=tau, device=True)


# ------------------------------------------------------------------ single steps
@pytest.mark.parametrize("N,P", [(1, 1), (37, 301), (64, 64), (130, 2000)])
def test_polarizability_direct_and_laplace(ctx, N, P):
    rng = np.random.default_rng(N * 1000 + P)
    Bt = rng.standard_normal((N, P)) * 0.05
    delta = rng.uniform(0.3, 4.0, P)
    om, _ = O.gl_grid(12, 0.5)
    Pi = torch.empty((12, N, N), dtype=torch.float64, device="cuda")
    ctx.polarizability(_dev(Bt), _dev(delta), om, Pi, spin=2)
    torch.cuda.synchronize()
    ref = O.polarizability_direct(Bt, delta, om, 2)
    got = Pi.cpu().numpy()
    assert _rel(got, ref) <= PI_TOL
    assert np.array_equal(got, np.swapaxes(got, 1, 2))  # exactly symmetric
    x, w = O.sinc_laplace_grid(7, -6.0, 2.0)
    ctx.polarizability(_dev(Bt), _dev(delta), om, Pi, spin=2, x=x, w=w)
    torch.cuda.synchronize()
    refl = O.polarizability_lt(O.laplace_moments(Bt, delta, x, w), om, x, 2)
    assert _rel(Pi.cpu().numpy(), refl) <= PI_TOL


def test_screening(ctx):
    prob = S.make_problem(5, 40, 90, seed=5, n_targets=2)
    delta = O.pair_gaps(prob.eps, 5, 40, 0)
    om, _ = O.gl_grid(9, 0.5)
    Pi = O.polarizability_direct(prob.B_ov, delta, om, 2)
    C = torch.empty_like(_dev(Pi))
    ctx.screen(_dev(Pi), C)
    ref = O.screened_interaction(Pi)
    assert _rel(C.cpu().numpy(), ref) <= 1e-12


def test_naf_basis_invariants(ctx):
    prob = S.make_workload(S.MID)
    B_act = np.ascontiguousarray(prob.B_ov[:, 10 * 540:])
    K = B_act @ B_act.T
    lam_ref, V = np.linalg.eigh(K)
    keep = lam_ref > 1e-2
    Ut = torch.empty((1800, 1800), dtype=torch.float64, device="cuda")
    lam = torch.empty(1800, dtype=torch.float64, device="cuda")
    k = ctx.naf_basis(_dev(B_act), B_act.shape[1], B_act.shape[1], 1e-2, Ut, lam)
    assert k == int(keep.sum())
    U = Ut[:k].cpu().numpy().T
    assert np.abs(U.T @ U - np.eye(k)).max() < 1e-12
    assert np.abs(np.sort(lam[:k].cpu().numpy()) - lam_ref[keep]).max() < 1e-13 * lam_ref[-1]
    P_ref = V[:, keep] @ V[:, keep].T
    assert np.abs(U @ U.T - P_ref).max() < 1e-10


def test_pi_invariant_form_mid(ctx):
    """U Pi U^T from the GPU NAF basis against the oracle's, at the mid size."""
    prob = S.make_workload(S.MID)
    _, _, _, it = _oracle(prob, 32, 1e-2)
    U = it["U"]
    Bt = U.T @ prob.B_ov[:, 10 * 540:]
    delta = O.pair_gaps(prob.eps, 60, 540, 10)
    om = it["omegas"][[0, 7, 31]]
    Pi = torch.empty((3, U.shape[1], U.shape[1]), dtype=torch.float64, device="cuda")
    ctx.polarizability(_dev(Bt), _dev(delta), om, Pi, spin=2)
    got = Pi.cpu().numpy()
    for j in range(3):
        assert _rel(U @ got[j] @ U.T, U @ it["Pi"][[0, 7, 31][j]] @ U.T) <= PI_TOL


# ------------------------------------------------------------------ errors
def test_bad_arguments_are_rejected(ctx):
    L = _ltgw()
    prob = S.make_workload(S.TINY)
    p = L.make_params(4, 16, 48, n_frozen=4, n_omega=8)
    T = len(prob.targets)
    out = (np.zeros((T, 8, 2)), np.zeros(T), np.zeros(T, dtype=np.int32))
    with pytest.raises(L.LtgwError) as e:
        ctx.solve(p, prob.eps, prob.B_ov, prob.B_tgt, prob.targets.astype(np.int32), prob.shift, *out)
    assert e.value.status == L.LTGW_ERR_BAD_ARG
    p = L.make_params(4, 16, 48, n_omega=8, naf_thresh=1e9)
    with pytest.raises(L.LtgwError) as e:
        ctx.solve(p, prob.eps, prob.B_ov, prob.B_tgt, prob.targets.astype(np.int32), prob.shift, *out)
    assert e.value.status == L.LTGW_ERR_NO_NAF
    # the context stays usable
    _check_solve(ctx, prob, 8)
