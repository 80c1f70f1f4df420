"""evGW through the C ABI against the oracle's evGW (same update rule, same
grids): FP64 at the parity bar of 1e-8 Ha, direct and with a caller-supplied
Laplace grid, with the gap-convergence stop; the split-BF16 form on the mid
workload within 1 meV."""
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


def _run(ctx, prob, n_om, thr, prec, n_cycles, gap_tol=0.0, tau=None):
    from paper_2307_04508_gb300 import ltgw
    p = ltgw.make_params(prob.n_occ, prob.n_virt, prob.n_aux, prob.n_frozen, n_om,
                         0 if tau is None else len(tau[0]), 0.5, thr, 2, tau is not None, prec)
    T = len(prob.targets)
    sig, e, st = np.zeros((T, n_om, 2)), np.zeros(T), np.zeros(T, dtype=np.int32)
    done = ctx.solve_ev(p, prob.eps, prob.B_ov, prob.B_tgt, prob.targets.astype(np.int32), prob.shift, sig, e, st,
                        n_cycles=n_cycles, gap_tol=gap_tol,
                        tau_x=None if tau is None else np.ascontiguousarray(tau[0]),
                        tau_w=None if tau is None else np.ascontiguousarray(tau[1]))
    return e, st, done


@pytest.mark.parametrize("laplace", [False, True])
def test_evgw_fp64_parity(ctx, laplace):
    from paper_2307_04508_gb300 import ltgw
    prob = S.make_problem(9, 70, 150, n_frozen=1, seed=99, n_targets=4)
    tau = O.sinc_laplace_grid(9, -11.0, 2.5) if laplace else None
    kw = dict(n_omega=17, naf_thresh=5e-3)
    if laplace:
        kw.update(tau_x=tau[0], tau_w=tau[1])
    _, e_o, st_o, done_o = O.evgw(prob.eps, prob.B_ov, prob.B_tgt, prob.targets, prob.shift, prob.n_occ,
                                  prob.n_virt, prob.n_frozen, n_cycles=4, **kw)
    e, st, done = _run(ctx, prob, 17, 5e-3, ltgw.LTGW_FP64, 4, tau=tau)
    _, e_g0, _ = O.solve(prob.eps, prob.B_ov, prob.B_tgt, prob.targets, prob.shift, prob.n_occ, prob.n_virt,
                         prob.n_frozen, **kw)
    print(f"evGW fp64 ({'Laplace' if laplace else 'direct'}): {np.abs(e - e_o).max():.2e} Ha from the oracle, "
          f"{np.abs(e - e_g0).max() * HA_TO_MEV:.1f} meV from G0W0")
    assert done == done_o == 4 and np.all(st == 0) and np.all(st_o == 0)
    assert np.abs(e - e_o).max() <= 1e-8


def test_evgw_gap_convergence_stop(ctx):
    from paper_2307_04508_gb300 import ltgw
    prob = S.make_problem(9, 70, 150, n_frozen=1, seed=99, n_targets=4)   # HOMO and LUMO among the targets
    _, e_o, _, done_o = O.evgw(prob.eps, prob.B_ov, prob.B_tgt, prob.targets, prob.shift, prob.n_occ,
                               prob.n_virt, prob.n_frozen, n_cycles=30, gap_tol=1e-6, n_omega=17,
                               naf_thresh=5e-3)
    e, st, done = _run(ctx, prob, 17, 5e-3, ltgw.LTGW_FP64, 30, gap_tol=1e-6)
    print(f"evGW to a 1e-6 Ha gap change: {done} cycles (oracle {done_o})")
    assert 1 <= done < 30 and done == done_o
    assert np.abs(e - e_o).max() <= 1e-8


def test_evgw_mixed_mid(ctx):
    from paper_2307_04508_gb300 import ltgw
    prob = S.make_workload(S.MID)
    tau = O.sinc_laplace_grid(8, -12.0, 3.0)
    _, e_o, _, _ = O.evgw(prob.eps, prob.B_ov, prob.B_tgt, prob.targets, prob.shift, 60, 540, 10, n_cycles=5,
                          n_omega=32, naf_thresh=1e-2, tau_x=tau[0], tau_w=tau[1])
    e, st, done = _run(ctx, prob, 32, 1e-2, ltgw.LTGW_BF16X3, 5, tau=tau)
    err = np.abs(e - e_o).max() * HA_TO_MEV
    print(f"evGW mixed, mid, 5 cycles: max QP error {err:.4f} meV")
    assert done == 5 and np.all(st == 0) and err <= 1.0
