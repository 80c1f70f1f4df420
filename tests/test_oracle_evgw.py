"""Pins of the oracle's evGW (eigenvalue-self-consistent GW, Sec. 3): the
scissor update written out by hand, zero cycles equal G0W0, and the AC route
against the fully-analytic (Casida) route iterated the same way, which share
no step but the update rule."""
import numpy as np

from oracle import casida as C
from oracle import ltgw_oracle as O
from paper_2307_04508_gb300 import synthetic as S


def test_scissor_update_by_hand():
    eps = np.array([-9.0, -1.0, -0.8, -0.5, 0.1, 0.4, 0.9, 2.0])
    targets = np.array([3, 5, 4])               # unsorted on purpose
    e_qp = np.array([-0.6, 0.5, 0.15])          # shifts -0.1 (3), +0.05 (4), +0.1 (5)
    got = O.evgw_energies(eps, targets, e_qp, n_frozen=1)
    want = np.array([-9.0, -1.1, -0.9, -0.6, 0.15, 0.5, 1.0, 2.1])
    assert np.allclose(got, want, atol=1e-15)


def test_zero_cycles_is_g0w0():
    prob = S.make_workload(S.TINY)
    args = (prob.eps, prob.B_ov, prob.B_tgt, prob.targets, prob.shift, prob.n_occ, prob.n_virt, prob.n_frozen)
    _, e0, _ = O.solve(*args, n_omega=24)
    _, e1, _, done = O.evgw(*args, n_cycles=0, n_omega=24)
    assert done == 0 and np.array_equal(e0, e1)


def test_evgw_ac_agrees_with_casida():
    """Three evGW cycles through analytic continuation (128 GL points) and
    through the Casida spectral form, both from the same update rule, on the
    tiny workload's law with four states around the gap."""
    t = S.TINY
    prob = S.make_problem(t["n_occ"], t["n_virt"], t["n_aux"], n_frozen=t["n_frozen"], seed=t["seed"], n_targets=4)
    args = (prob.eps, prob.B_ov, prob.B_tgt, prob.targets, prob.shift, prob.n_occ, prob.n_virt, prob.n_frozen)
    _, e_ac, st, done = O.evgw(*args, n_cycles=3, n_omega=128)
    e_c, _, _, _ = C.g0w0_analytic(*args)
    e_g0 = e_c.copy()
    for _ in range(3):
        cur = O.evgw_energies(prob.eps, prob.targets, e_c, prob.n_frozen)
        e_c, stc, _, _ = C.g0w0_analytic(cur, *args[1:], eps_ref=prob.eps)
    dev = np.abs(e_ac - e_c).max() * 27211.386
    print(f"evGW (3 cycles): AC vs Casida {dev:.4f} meV; shift from G0W0 {np.abs(e_c - e_g0).max() * 27211.386:.1f} meV")
    assert done == 3 and np.all(st == 0) and np.all(stc == 0)
    assert np.abs(e_c - e_g0).max() > 1e-4          # self-consistency moves the energies
    assert dev < 0.05
