"""The contraction autotuner: with it on, the first tensor-core contraction of
a shape times candidate configurations (scales per CTA, K-split count) and
keeps the fastest.  Whatever it picks, results stay within the form's
tolerance of the oracle, and a repeated call with the cached choice gives the
same bits."""
import numpy as np
import pytest

from oracle import ltgw_oracle as O
from paper_2307_04508_gb300 import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture()
def ctx():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2307_04508_gb300 import ltgw
    c = ltgw.Context(0)
    c.set_autotune(True)
    yield c
    c.close()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("fp8", [False, True])
def test_autotuned_polarizability(ctx, fp8):
    rng = np.random.default_rng(11)
    N, P, n_om = 200, 9000, 6
    Bt = rng.standard_normal((N, P)) * 0.05
    delta = rng.uniform(0.3, 4.0, P)
    om, _ = O.gl_grid(n_om, 0.5)
    x, w = O.sinc_laplace_grid(8, -6.0, 2.0)
    outs = []
    for _ in range(2):
        Pi = torch.empty((n_om, N, N), dtype=torch.float64, device="cuda")
        ctx.polarizability_mixed(_dev(Bt), _dev(delta), om, Pi, spin=2, x=x, w=w, fp8=fp8)
        outs.append(Pi.cpu().numpy())
    assert ctx.stats()["tc_autotuned"] >= 1
    assert np.array_equal(outs[0], outs[1]), "the cached configuration must be reused"
    if fp8:
        assert _rel(outs[0], O.polarizability_fp8(Bt, delta, om, 2, x=x, w=w)) <= 2e-5
    else:
        assert _rel(outs[0], O.polarizability_lt(O.laplace_moments(Bt, delta, x, w), om, x, 2)) <= 5e-5


def test_autotuned_solve(ctx):
    from paper_2307_04508_gb300 import ltgw
    prob = S.make_problem(9, 70, 150, n_frozen=1, seed=99, n_targets=3)
    tau = O.sinc_laplace_grid(9, -11.0, 2.5)
    _, e_o, st_o = O.solve(prob.eps, prob.B_ov, prob.B_tgt, prob.targets, prob.shift, prob.n_occ, prob.n_virt,
                           prob.n_frozen, n_omega=17, naf_thresh=5e-3, tau_x=tau[0], tau_w=tau[1])
    p = ltgw.make_params(prob.n_occ, prob.n_virt, prob.n_aux, prob.n_frozen, 17, 9, 0.5, 5e-3, 2, True,
                         ltgw.LTGW_BF16X3)
    T = len(prob.targets)
    for _ in range(2):
        sig, e, st = np.zeros((T, 17, 2)), np.zeros(T), np.zeros(T, dtype=np.int32)
        ctx.solve(p, prob.eps, prob.B_ov, prob.B_tgt, prob.targets.astype(np.int32), prob.shift, sig, e, st,
                  tau_x=np.ascontiguousarray(tau[0]), tau_w=np.ascontiguousarray(tau[1]))
        assert np.all(st == 0) and np.abs(e - e_o).max() <= 1e-3 / 27.211386245988
    assert ctx.stats()["tc_autotuned"] >= 2   # the metric, the projections and Pi are tuned shapes
