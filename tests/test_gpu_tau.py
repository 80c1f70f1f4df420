"""Imaginary-time (cosine-transform) form of Pi: M^k = R~ diag(e^{-Delta tau_k}) R~^T,
Pi_j = -2 s sum_k gamma_jk M^k, against the oracle fed the same grid (FP64 at
1e-11, split BF16 at 5e-5, FP8 against the oracle's FP8 definition at 2e-5),
a whole FP64 solve at 1e-8 Ha, and the accuracy of both grid forms (Eq. LT's
factorisation and this one, each with the library's own fit) against the
direct-AC oracle as the node count grows."""
import numpy as np
import pytest

from oracle import ltgw_oracle as O
from paper_2307_04508_gb300 import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
HA_TO_MEV = 27211.386245988


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2307_04508_gb300 import ltgw
    c = ltgw.Context(0)
    yield c
    c.close()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("N,P", [(1, 1), (37, 301), (200, 9000)])
def test_tau_polarizability_all_precisions(ctx, N, P):
    from paper_2307_04508_gb300 import ltgw
    rng = np.random.default_rng(3 * N + P)
    Bt = rng.standard_normal((N, P)) * 0.05
    delta = rng.uniform(0.3, 4.0, P)
    om, _ = O.gl_grid(12, 0.5)
    # a ridge keeps the recombination's amplification of the moments' relative
    # errors (about 1e-5 in split BF16 and in FP8 against its own definition) small
    tau, gamma, amp = O.cosine_grid(10, 0.3, 4.0, om, ridge=1e-10)
    ref = O.polarizability_tau(O.tau_moments(Bt, delta, tau), gamma, 2)
    Pi = torch.empty((len(om), N, N), dtype=torch.float64, device="cuda")
    for prec, tol, want in ((ltgw.LTGW_FP64, 1e-11, ref), (ltgw.LTGW_BF16X3, 1e-5 * amp, ref),
                            (ltgw.LTGW_FP8, 1e-5 * amp,
                             O.polarizability_fp8(Bt, delta, om, 2, tau=tau, gamma=gamma))):
        ctx.polarizability_tau(_dev(Bt), _dev(delta), om, tau, gamma, Pi, spin=2, precision=prec)
        err = _rel(Pi.cpu().numpy(), want)
        print(f"tau form N={N} P={P} precision {prec}: {err:.2e} (amplification {amp:.1f})")
        assert err <= tol


def test_tau_solve_fp64_parity(ctx):
    from paper_2307_04508_gb300 import ltgw
    prob = S.make_problem(9, 70, 150, n_frozen=1, seed=99, n_targets=3)
    eps = prob.eps
    n_occ, nf = prob.n_occ, prob.n_frozen
    om, _ = O.gl_grid(17, 0.5)
    tau, gamma, _ = O.cosine_grid(12, eps[n_occ] - eps[n_occ - 1], eps[-1] - eps[nf], om)
    _, e_o, st_o = O.solve(prob.eps, prob.B_ov, prob.B_tgt, prob.targets, prob.shift, n_occ, prob.n_virt, nf,
                           n_omega=17, naf_thresh=5e-3, cos_tau=tau, cos_gamma=gamma)
    p = ltgw.make_params(n_occ, prob.n_virt, prob.n_aux, nf, 17, 12, 0.5, 5e-3, 2, 2, ltgw.LTGW_FP64)
    T = len(prob.targets)
    sig, e, st = np.zeros((T, 17, 2)), np.zeros(T), np.zeros(T, dtype=np.int32)
    ctx.solve(p, prob.eps, prob.B_ov, prob.B_tgt, prob.targets.astype(np.int32), prob.shift, sig, e, st,
              tau_x=np.ascontiguousarray(tau), tau_w=np.ascontiguousarray(gamma))
    assert np.all(st == 0) and np.all(st_o == 0)
    assert np.abs(e - e_o).max() <= 1e-8


def test_grid_forms_against_direct_oracle(ctx):
    """Mid workload, FP64 form, library grids: the per-state QP error against the
    direct-AC oracle for Eq. LT's factorisation and the imaginary-time form."""
    from paper_2307_04508_gb300 import ltgw
    prob = S.make_workload(S.MID)
    _, e_d, _ = O.solve(prob.eps, prob.B_ov, prob.B_tgt, prob.targets, prob.shift, 60, 540, 10, n_omega=32,
                        naf_thresh=1e-2)
    T = len(prob.targets)
    dev = [_dev(a) for a in (prob.eps, prob.B_ov, prob.B_tgt, prob.targets.astype(np.int32), prob.shift)]
    rows = []
    for n_tau in (6, 8, 10, 12, 16):
        errs = []
        for form, prec in ((1, ltgw.LTGW_FP64), (2, ltgw.LTGW_FP64), (1, ltgw.LTGW_BF16X3), (2, ltgw.LTGW_BF16X3)):
            p = ltgw.make_params(60, 540, 1800, 10, 32, n_tau, 0.5, 1e-2, 2, form, prec)
            sig, e, st = np.zeros((T, 32, 2)), np.zeros(T), np.zeros(T, dtype=np.int32)
            ctx.solve(p, *dev, sig, e, st)
            assert np.all(st == 0)
            errs.append(np.abs(e - e_d).max() * HA_TO_MEV)
        rows.append((n_tau, *errs))
        print(f"N_tau {n_tau:2d}: max QP error vs direct AC (meV)  FP64: Eq. LT form {errs[0]:.4f}, "
              f"imaginary-time form {errs[1]:.4f};  split BF16: Eq. LT form {errs[2]:.4f}, "
              f"imaginary-time form {errs[3]:.4f}")
    assert rows[-1][2] < 0.01          # the imaginary-time form converges with the node count
    assert rows[-1][2] < rows[0][2]


def test_laplace_form_beyond_64_frequencies(ctx):
    """Eq. LT's recombination over 100 GL frequencies (launched in chunks of 64)."""
    rng = np.random.default_rng(5)
    N, P = 40, 2000
    Bt = rng.standard_normal((N, P)) * 0.05
    delta = rng.uniform(0.3, 4.0, P)
    om, _ = O.gl_grid(100, 0.5)
    x, w = O.sinc_laplace_grid(9, -8.0, 2.0)
    Pi = torch.empty((len(om), N, N), dtype=torch.float64, device="cuda")
    ctx.polarizability(_dev(Bt), _dev(delta), om, Pi, spin=2, x=x, w=w)
    ref = O.polarizability_lt(O.laplace_moments(Bt, delta, x, w), om, x, 2)
    assert _rel(Pi.cpu().numpy(), ref) <= 1e-11
