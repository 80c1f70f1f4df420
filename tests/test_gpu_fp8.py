"""FP8 E4M3 form of the Pi contraction (per-auxiliary-row scales, two-term
E4M3 expansion of every operand value, FP32 accumulation on tcgen05
kind::f8f6f4) against the oracle's FP8 definition, which rounds the same FP32
values to the same codes and sums the products exactly: the two differ only
by the FP32 accumulation, so the bar is 2e-5 relative Frobenius.  Whole
solves in both FP8 modes (Pi and W_nm in FP8, or Pi alone) stay within the
1 meV target of the FP64 oracle."""
import numpy as np
import pytest

from oracle import ltgw_oracle as O
from paper_2307_04508_gb300 import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PI_TOL_FP8_VS_ORACLE = 2e-5
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


# (1, 1): one pair; 301 / 2000 / 9000 pairs: ragged K tails; 270,000 pairs: more than
# 64 K-splits of 4096 pairs, so every CTA drains its FP32 accumulators more than once
@pytest.mark.parametrize("N,P,n_om", [(1, 1, 3), (37, 301, 12), (130, 2000, 9), (200, 9000, 20), (20, 270000, 3)])
def test_fp8_polarizability_direct_and_laplace(ctx, N, P, n_om):
    rng = np.random.default_rng(2 * N + P)
    Bt = rng.standard_normal((N, P)) * 0.05
    delta = rng.uniform(0.3, 4.0, P)
    om, _ = O.gl_grid(n_om, 0.5)
    Pi = torch.empty((n_om, N, N), dtype=torch.float64, device="cuda")
    ctx.polarizability_fp8(_dev(Bt), _dev(delta), om, Pi, spin=2)
    got = Pi.cpu().numpy()
    ref8 = O.polarizability_fp8(Bt, delta, om, 2)
    err = _rel(got, ref8)
    exact = _rel(got, O.polarizability_direct(Bt, delta, om, 2))
    print(f"fp8 direct N={N} P={P}: vs FP8 oracle {err:.2e}, vs exact Pi {exact:.2e}")
    assert err <= PI_TOL_FP8_VS_ORACLE
    assert np.array_equal(got, np.swapaxes(got, 1, 2))
    x, w = O.sinc_laplace_grid(7, -6.0, 2.0)
    ctx.polarizability_fp8(_dev(Bt), _dev(delta), om, Pi, spin=2, x=x, w=w)
    got = Pi.cpu().numpy()
    errl = _rel(got, O.polarizability_fp8(Bt, delta, om, 2, x=x, w=w))
    exactl = _rel(got, O.polarizability_lt(O.laplace_moments(Bt, delta, x, w), om, x, 2))
    print(f"fp8 laplace N={N} P={P}: vs FP8 oracle {errl:.2e}, vs exact Pi {exactl:.2e}")
    assert errl <= PI_TOL_FP8_VS_ORACLE


@pytest.mark.parametrize("mode,bound_mev", [("fp8", 1.0), ("fp8_pi", 1.0)])
def test_fp8_solve_mid_workload(ctx, mode, bound_mev):
    """Mid workload (1800 auxiliary functions, NAF 1e-2): per-state QP error
    against the FP64 oracle fed the same Laplace grid, with Pi and W_nm in FP8
    (LTGW_FP8) or Pi alone in FP8 (LTGW_FP8_PI, W_nm split-BF16), both within
    the 1 meV target (the oracle's two-term expansion puts them near 0.01 meV)."""
    from paper_2307_04508_gb300 import ltgw
    prob = S.make_workload(S.MID)
    tau = O.sinc_laplace_grid(8, -12.0, 3.0)
    _, e_o, st_o = O.solve(prob.eps, prob.B_ov, prob.B_tgt, prob.targets, prob.shift, 60, 540, 10, n_omega=32,
                           naf_thresh=1e-2, tau_x=tau[0], tau_w=tau[1])
    prec = ltgw.LTGW_FP8 if mode == "fp8" else ltgw.LTGW_FP8_PI
    p = ltgw.make_params(60, 540, 1800, 10, 32, 8, 0.5, 1e-2, 2, True, prec)
    T = len(prob.targets)
    sig, e, st = np.zeros((T, 32, 2)), np.zeros(T), np.zeros(T, dtype=np.int32)
    dev = [_dev(a) for a in (prob.eps, prob.B_ov, prob.B_tgt, prob.targets.astype(np.int32), prob.shift)]
    ctx.solve(p, *dev, sig, e, st, tau_x=np.ascontiguousarray(tau[0]), tau_w=np.ascontiguousarray(tau[1]))
    mev = np.abs(e - e_o) * HA_TO_MEV
    print(f"{mode} solve: per-state QP error (meV) " + " ".join(f"{v:.3f}" for v in mev))
    assert np.all(st == 0) and np.all(st_o == 0)
    assert mev.max() <= bound_mev
