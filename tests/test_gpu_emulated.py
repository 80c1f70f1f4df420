"""FP64-accurate product from integer slices on the tensor cores
(ltgw_gemm_emulated) against the oracle's slice_product, which takes the same
digits and sums every kept pair exactly: the two differ only by the order of
the FP64 additions of the pair sums, bounded here by 4 * (pairs + 2) * eps *
sum_k |A_rk| |B_ck| per entry.  Against the exact product the error is the
dropped digits' (about 2^(-7 s) of the row scales); the NAF metric's shape
(a Gram matrix of many long rows) is checked in the symmetric form."""
import numpy as np
import pytest

from oracle import ltgw_oracle as O
from paper_2307_04508_gb300 import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2307_04508_gb300 import ltgw
    c = ltgw.Context(0)
    yield c
    c.close()


def _pairs(s):
    return sum(1 for i in range(1, s + 1) for j in range(1, s + 1) if i + j <= s + 1)


def _check_vs_oracle(got, A, B, s):
    ref = O.slice_product(A, B, s)
    bound = 4 * (_pairs(s) + 2) * EPS * (np.abs(A) @ np.abs(B).T)
    err = np.abs(got - ref)
    assert np.all(err <= bound), (err.max(), (err / np.maximum(bound, 1e-300)).max())
    return ref


# (1, 1, 1): one entry; 130 x 257 x 1500: ragged row tiles on both sides and
# two FP32 drains of 1024 pairs with a ragged tail; 300 x 129 x 5000: more
# K-splits; rows scaled by 2^-300 .. 2^300 and a zero row
@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (130, 257, 1500), (300, 129, 5000)])
@pytest.mark.parametrize("s", [4, 6])
def test_emulated_product_matches_oracle(ctx, m, n, k, s):
    rng = np.random.default_rng(m * 7 + n + k + s)
    A = rng.standard_normal((m, k)) * np.exp2(rng.integers(-300, 300, m))[:, None]
    B = rng.standard_normal((n, k)) * np.exp2(rng.integers(-300, 300, n))[:, None]
    if m > 2:
        A[1] = 0.0
    C = torch.full((m, n), np.nan, dtype=torch.float64, device="cuda")
    ctx.gemm_emulated(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), C, n_slices=s)
    got = C.cpu().numpy()
    _check_vs_oracle(got, A, B, s)
    if m > 2:
        assert not got[1].any()
    # against the exact product (long double, the first 24 rows): per entry within
    # the dropped digits' bound, 2^(-7 s) (1 + (s - 1) / 4) of k times the rows' scales
    r = min(m, 24)
    ea = np.frexp(np.abs(A[:r]).max(axis=1))[1]
    eb = np.frexp(np.abs(B).max(axis=1))[1]
    scale = np.ldexp(np.ldexp(np.full((r, n), float(k)), ea[:, None]), eb[None, :])
    exact = np.matmul(A[:r].astype(np.longdouble), B.astype(np.longdouble).T)
    err = np.abs((got[:r] - exact).astype(np.float64))
    assert np.all(err <= 2.0 ** (-7 * s) * (1 + (s - 1) / 4) * 1.01 * scale + 1e-15 * scale)


def test_emulated_product_strided_and_tiny_rows(ctx):
    """Row strides larger than k, and rows around 1e-300 (their fixed-point
    scale 2^(7 s - e) is beyond the FP64 range: the digits still come out)."""
    rng = np.random.default_rng(4)
    m, n, k = 200, 140, 777
    Abig = rng.standard_normal((m, k + 13))
    Bbig = rng.standard_normal((n, k + 5))
    Abig[:5] *= 1e-300
    Bbig[:3] *= 1e-300
    A, B = Abig[:, :k], Bbig[:, :k]
    dA, dB = torch.from_numpy(Abig).cuda(), torch.from_numpy(Bbig).cuda()
    Cbig = torch.full((m, n + 9), np.nan, dtype=torch.float64, device="cuda")
    ctx.gemm_emulated(dA[:, :k], dB[:, :k], Cbig[:, :n], n_slices=6)
    got = Cbig.cpu().numpy()
    _check_vs_oracle(got[:, :n], np.ascontiguousarray(A), np.ascontiguousarray(B), 6)
    assert np.all(np.isnan(got[:, n:]))   # outside the written columns: untouched


@pytest.mark.parametrize("N,K", [(1, 5), (200, 3000), (390, 2500)])
def test_emulated_symmetric_matches_oracle(ctx, N, K):
    """The NAF metric's form K = R R^T (Eq. nafeq), lower tiles computed and
    mirrored: symmetric bit for bit, and the oracle's value per entry."""
    rng = np.random.default_rng(N + K)
    R = rng.standard_normal((N, K)) * 0.05
    C = torch.full((N, N), np.nan, dtype=torch.float64, device="cuda")
    ctx.gemm_emulated(torch.from_numpy(R).cuda(), None, C, n_slices=6, sym=True)
    got = C.cpu().numpy()
    assert np.array_equal(got, got.T)
    ref = _check_vs_oracle(got, R, R, 6)
    direct = R @ R.T
    rel = np.linalg.norm(got - direct) / np.linalg.norm(direct)
    print(f"sym N={N} K={K}: vs oracle {np.abs(got - ref).max():.2e}, rel vs FP64 product {rel:.2e}")
    assert rel < 1e-11


def test_emulated_bad_arguments(ctx):
    from paper_2307_04508_gb300 import ltgw
    A = torch.ones((4, 8), dtype=torch.float64, device="cuda")
    C = torch.empty((4, 4), dtype=torch.float64, device="cuda")
    for s in (1, 9):
        with pytest.raises(ltgw.LtgwError):
            ctx.gemm_emulated(A, None, C, n_slices=s, sym=True)
    with pytest.raises(ltgw.LtgwError):   # host operand
        ctx.gemm_emulated(A, torch.ones((4, 8), dtype=torch.float64), C, n_slices=6)
    ctx.gemm_emulated(A, None, C, n_slices=6, sym=True)   # the context still works
    assert torch.equal(C, torch.full((4, 4), 8.0, dtype=torch.float64, device="cuda"))


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# (1, 1): one pair; 37 x 301: ragged tiles and K tail; 200 x 9000: several
# row tiles and FP32 drains per split
@pytest.mark.parametrize("N,P,n_om", [(1, 1, 3), (37, 301, 12), (200, 9000, 20)])
@pytest.mark.parametrize("laplace", [False, True])
def test_emulated_polarizability(ctx, N, P, n_om, laplace):
    """ltgw_polarizability_emulated against the oracle's slice form (same
    factors and digits: the FP64 addition order of the pair sums apart, and
    for the Laplace form the last bit of exp) and against the plain FP64 Pi
    (Eq. Pi, or the M^m form of Eq. LT) to the slices' error."""
    rng = np.random.default_rng(3 * N + P)
    Bt = rng.standard_normal((N, P)) * 0.05 * np.exp(-np.arange(N) / 40.0)[:, None]
    delta = rng.uniform(0.3, 4.0, P)
    om, _ = O.gl_grid(n_om, 0.5)
    x = w = None
    if laplace:
        x, w = O.sinc_laplace_grid(7, -6.0, 2.0)
    Pi = torch.full((n_om, N, N), np.nan, dtype=torch.float64, device="cuda")
    ctx.polarizability_emulated(torch.from_numpy(Bt).cuda(), torch.from_numpy(delta).cuda(), om, Pi, spin=2,
                                x=x, w=w, n_slices=6)
    got = Pi.cpu().numpy()
    assert np.array_equal(got, np.swapaxes(got, 1, 2))
    ref = O.polarizability_emulated(Bt, delta, om, 2, x=x, w=w, n_slices=6)
    exact = (O.polarizability_lt(O.laplace_moments(Bt, delta, x, w), om, x, 2) if laplace
             else O.polarizability_direct(Bt, delta, om, 2))
    e_or, e_ex = _rel(got, ref), _rel(got, exact)
    print(f"emulated Pi N={N} P={P} laplace={laplace}: vs oracle slices {e_or:.2e}, vs FP64 Pi {e_ex:.2e}")
    assert e_or <= (1e-12 if laplace else 1e-13)
    assert e_ex <= 1e-11


# ---------------------------------------------------------------- whole solve
# LTGW_FP64_EMU: the FP64 form with the NAF metric, the projections, Pi and
# W_nm from 6 slices; against the plain FP64 oracle with the FP64 form's bars
# (quasi-particle energies within 1e-8 Ha, the same N_NAF) and Sigma(i w)
# within 1e-10 of its largest magnitude (the slices' 2^-42 relative errors
# in Pi, K and the projections, against the FP64 form's rounding)
EMU_SIG_TOL = 1e-10


def _emu_cases():
    tau6 = O.sinc_laplace_grid(6, -9.0, 2.0)
    tau9 = O.sinc_laplace_grid(9, -11.0, 2.5)
    tau8 = O.sinc_laplace_grid(8, -12.0, 3.0)
    return {
        "tiny_direct": (lambda: S.make_workload(S.TINY), 24, -1.0, None, 2),
        "tiny_laplace": (lambda: S.make_workload(S.TINY), 24, -1.0, tau6, 2),
        "ragged_frozen_naf_spin1": (lambda: S.make_problem(7, 45, 131, n_frozen=2, seed=4242, n_targets=4), 21,
                                    1e-3, None, 1),
        "ragged_laplace_naf": (lambda: S.make_problem(9, 70, 150, n_frozen=1, seed=99, n_targets=3), 17, 5e-3,
                               tau9, 2),
        "single_active_occupied": (lambda: S.make_problem(3, 30, 20, n_frozen=2, seed=7, n_targets=2), 16, -1.0,
                                   None, 2),
        "mid_laplace": (lambda: S.make_workload(S.MID), 32, 1e-2, tau8, 2),
    }


@pytest.mark.parametrize("case", list(_emu_cases()))
def test_emulated_solve_matches_oracle(ctx, case):
    from paper_2307_04508_gb300 import ltgw
    make, n_om, thr, tau, spin = _emu_cases()[case]
    prob = make()
    tx, tw = (None, None) if tau is None else tau
    sig_o, e_o, st_o, it = O.solve(prob.eps, prob.B_ov, prob.B_tgt, prob.targets, prob.shift, prob.n_occ,
                                   prob.n_virt, prob.n_frozen, n_omega=n_om, naf_thresh=thr, spin=spin, tau_x=tx,
                                   tau_w=tw, return_all=True)
    sig, e, st = ltgw.solve_problem(ctx, prob, n_omega=n_om, n_tau=0 if tau is None else len(tau[0]),
                                    naf_thresh=thr, use_laplace=tau is not None, spin=spin, tau=tau,
                                    precision=ltgw.LTGW_FP64_EMU)
    stats = ctx.stats()
    print(f"emulated solve {case}: QP {np.abs(e - e_o).max():.2e} Ha, "
          f"Sigma {np.abs(sig - sig_o).max() / np.abs(sig_o).max():.2e}, {stats['ms_total']:.1f} ms")
    assert np.all(st == 0) and np.all(st_o == 0)
    assert stats["n_naf"] == it["n_naf"]
    assert np.abs(e - e_o).max() <= 1e-8
    assert np.abs(sig - sig_o).max() <= EMU_SIG_TOL * np.abs(sig_o).max()


def test_emulated_solve_imaginary_time(ctx):
    """The imaginary-time form (factors e^{-Delta tau_k}, fitted gamma) in the
    emulated form against the oracle's."""
    from paper_2307_04508_gb300 import ltgw
    prob = S.make_problem(9, 70, 150, n_frozen=1, seed=99, n_targets=3)
    eps, n_occ, nf = prob.eps, prob.n_occ, prob.n_frozen
    om, _ = O.gl_grid(17, 0.5)
    tau, gamma, _ = O.cosine_grid(12, eps[n_occ] - eps[n_occ - 1], eps[-1] - eps[nf], om)
    _, e_o, st_o = O.solve(prob.eps, prob.B_ov, prob.B_tgt, prob.targets, prob.shift, n_occ, prob.n_virt, nf,
                           n_omega=17, naf_thresh=5e-3, cos_tau=tau, cos_gamma=gamma)
    p = ltgw.make_params(n_occ, prob.n_virt, prob.n_aux, nf, 17, 12, 0.5, 5e-3, 2, 2, ltgw.LTGW_FP64_EMU)
    T = len(prob.targets)
    sig, e, st = np.zeros((T, 17, 2)), np.zeros(T), np.zeros(T, dtype=np.int32)
    ctx.solve(p, prob.eps, prob.B_ov, prob.B_tgt, prob.targets.astype(np.int32), prob.shift, sig, e, st,
              tau_x=np.ascontiguousarray(tau), tau_w=np.ascontiguousarray(gamma))
    assert np.all(st == 0) and np.all(st_o == 0)
    assert np.abs(e - e_o).max() <= 1e-8
