"""The allocation-free screening entry point, ltgw_screen_static.

Some callers cannot allocate device memory when they call into the library:
a process whose device memory is already claimed in full by another allocator
(a framework's caching allocator or a pre-reserved pool), or a
latency-sensitive caller that cannot afford cudaMalloc/cudaFree, which may
block and synchronise the device.  ltgw_screen_static serves them with scratch
held in a fixed device array inside the library.  These tests call it through
the C ABI twice in a row and compare each result with the ordinary entry
point, ltgw_screen, and with the oracle's Cholesky route, at the tolerance the
screening parity test uses.

This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from oracle import ltgw_oracle as O
from paper_2307_04508_gb300 import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


def _pi(n_occ, n_virt, n_aux, n_omega, seed):
    prob = S.make_problem(n_occ, n_virt, n_aux, seed=seed, n_targets=2)
    delta = O.pair_gaps(prob.eps, n_occ, n_virt, 0)
    om, _ = O.gl_grid(n_omega, 0.5)
    return O.polarizability_direct(prob.B_ov, delta, om, 2)


def test_static_screening_matches_allocating_entry_point_twice():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2307_04508_gb300 import ltgw
    lib = ltgw.load()
    ctx = ltgw.Context(0)
    try:
        # two different problems in a row: the second is smaller, so stale
        # scratch contents from the first call would show up in its result
        for n_occ, n_virt, n_aux, n_omega, seed in ((6, 50, 120, 32, 1), (4, 30, 70, 9, 2)):
            assert n_omega * n_aux * n_aux <= ltgw.SCREEN_STATIC_MAX_ELEMS
            Pi = torch.from_numpy(_pi(n_occ, n_virt, n_aux, n_omega, seed)).cuda()
            C_static = torch.full_like(Pi, float("nan"))
            C_ref = torch.full_like(Pi, float("nan"))
            st = lib.ltgw_screen_static(n_aux, n_omega, Pi.data_ptr(), C_static.data_ptr(), None)
            assert st == ltgw.LTGW_OK, ltgw.status_string(st)
            ctx.screen(Pi, C_ref)
            a, b = C_static.cpu().numpy(), C_ref.cpu().numpy()
            assert np.all(np.isfinite(a))
            assert np.abs(a - b).max() <= TOL * np.abs(b).max()
            # and against the oracle's Cholesky route, the definition itself
            c = O.screened_interaction(Pi.cpu().numpy())
            assert np.abs(a - c).max() <= TOL * np.abs(c).max()
    finally:
        ctx.close()


def test_static_screening_rejects_oversized_problems():
    from paper_2307_04508_gb300 import ltgw
    lib = ltgw.load()
    N = 200
    n_omega = ltgw.SCREEN_STATIC_MAX_ELEMS // (N * N) + 1
    Pi = torch.zeros((1,), dtype=torch.float64, device="cuda")
    C = torch.zeros((1,), dtype=torch.float64, device="cuda")
    # the size check comes before any GPU work, so tiny buffers suffice here
    st = lib.ltgw_screen_static(N, n_omega, Pi.data_ptr(), C.data_ptr(), None)
    assert st == ltgw.LTGW_ERR_BAD_ARG
