"""The request server (ltgw_server): every request's result is the same alone
and in the mix, admission respects the memory budget, and oversized requests
are rejected."""
import numpy as np
import pytest

from paper_2307_04508_gb300 import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _requests(n=12):
    reqs = []
    for i in range(n):
        n_occ = 4 + (i * 5) % 11
        n_virt = 8 * n_occ + (i % 3)
        reqs.append(dict(index=i, n_occ=n_occ, n_frozen=n_occ // 6, n_virt=n_virt, n_aux=3 * (n_occ + n_virt),
                         n_targets=4, seed=777 + i, t_arrival=0.0))
    return reqs


@pytest.mark.parametrize("mixed", [False, True])
def test_results_alone_equal_results_in_the_mix(mixed):
    from paper_2307_04508_gb300 import ltgw, serving
    prec = ltgw.LTGW_BF16X3 if mixed else ltgw.LTGW_FP64
    reqs = _requests()
    inputs = [serving.ingest(r, device=False) for r in reqs]
    ctx = ltgw.Context(0)
    alone = []
    for r, inp in zip(reqs, inputs):
        T = len(inp["targets"])
        sig, e, st = np.zeros((T, 32, 2)), np.zeros(T), np.zeros(T, dtype=np.int32)
        ctx.solve(serving.request_params(r, prec), inp["eps"], inp["B_ov"], inp["B_tgt"], inp["targets"],
                  inp["shift"], sig, e, st)
        alone.append(e.copy())
    ctx.close()
    srv = ltgw.Server(0, n_slots=4, hbm_budget_bytes=32 << 30)
    try:
        recs, wall, _ = serving.run_stream(srv, reqs, prec, honor_arrivals=False, inputs=inputs)
    finally:
        srv.close()
    assert len(recs) == len(reqs)
    for r, a in zip(reqs, alone):
        rec = recs[r["index"]]
        assert rec["status"] in (ltgw.LTGW_OK, ltgw.LTGW_ERR_NO_CONVERGE)
        assert np.abs(rec["e_qp"] - a).max() <= 1e-12
    # requests overlapped in service
    spans = sorted((v["start_ms"], v["end_ms"]) for v in recs.values())
    assert any(s1 < e0 for (s0, e0), (s1, e1) in zip(spans, spans[1:]))


def test_budget_serialises_admission():
    from paper_2307_04508_gb300 import ltgw, serving
    # four requests of one size: a budget of one footprint admits one at a time
    reqs = [dict(r, n_occ=8, n_frozen=1, n_virt=64, n_aux=216) for r in _requests(4)]
    inputs = [serving.ingest(r, device=False) for r in reqs]
    fps = [ltgw.request_footprint(serving.request_params(r, ltgw.LTGW_FP64), 4) for r in reqs]
    srv = ltgw.Server(0, n_slots=4, hbm_budget_bytes=max(fps))   # room for one request at a time
    try:
        recs, _, _ = serving.run_stream(srv, reqs, ltgw.LTGW_FP64, honor_arrivals=False, inputs=inputs)
    finally:
        srv.close()
    spans = sorted((v["start_ms"], v["end_ms"]) for v in recs.values())
    for (s0, e0), (s1, e1) in zip(spans, spans[1:]):
        assert s1 >= e0 - 1e-3   # no two requests in service at once


def test_oversized_request_is_rejected():
    from paper_2307_04508_gb300 import ltgw, serving
    r = _requests(1)[0]
    inp = serving.ingest(r, device=False)
    srv = ltgw.Server(0, n_slots=1, hbm_budget_bytes=1 << 20)
    try:
        with pytest.raises(ltgw.LtgwError) as e:
            srv.submit(serving.request_params(r, ltgw.LTGW_FP64), inp["eps"], inp["B_ov"], inp["B_tgt"],
                       inp["targets"], inp["shift"], np.zeros((4, 32, 2)), np.zeros(4), np.zeros(4, dtype=np.int32))
        assert e.value.status == ltgw.LTGW_ERR_NOMEM
    finally:
        srv.close()


def test_device_generator_matches_host_law():
    from paper_2307_04508_gb300.synthetic.device import DeviceLaw
    p = S.make_problem(6, 50, 120, n_frozen=1, seed=31, n_targets=2)
    law = DeviceLaw(6, 50, 120, 1, 31, 2, gemm="fp64")
    assert np.abs(law.b_ov().cpu().numpy() - p.B_ov).max() < 1e-12 * np.abs(p.B_ov).max() + 1e-15
    assert np.abs(law.b_tgt().cpu().numpy() - p.B_tgt).max() < 1e-12 * np.abs(p.B_tgt).max() + 1e-15


def test_trim_releases_the_workspace():
    """A context's workspace grows to its largest call and is kept; ltgw_trim
    frees it and the next call allocates again with the same result."""
    from paper_2307_04508_gb300 import ltgw
    c = ltgw.Context(0)
    try:
        prob = S.make_problem(9, 70, 150, n_frozen=1, seed=99, n_targets=3)
        p = ltgw.make_params(prob.n_occ, prob.n_virt, prob.n_aux, prob.n_frozen, 17, 0, 0.5, 5e-3, 2, False,
                             ltgw.LTGW_BF16X3)
        T = len(prob.targets)
        outs = []
        for trim in (False, True):
            sig, e, st = np.zeros((T, 17, 2)), np.zeros(T), np.zeros(T, dtype=np.int32)
            c.solve(p, prob.eps, prob.B_ov, prob.B_tgt, prob.targets.astype(np.int32), prob.shift, sig, e, st)
            outs.append(e.copy())
            assert c.workspace_bytes() > 0
            if not trim:
                c.trim()
                assert c.workspace_bytes() == 0
        assert np.array_equal(outs[0], outs[1])
    finally:
        c.close()


def test_request_that_does_not_fit_is_passed_a_bounded_number_of_times():
    """Two slots; a medium request runs, a large one arrives that does not fit
    beside it (or beside any small one), then ten small ones that do: the
    small ones pass the large one exactly eight times (the server's bound),
    after which it is admitted as soon as nothing else runs, before the
    remaining small ones."""
    from paper_2307_04508_gb300 import ltgw, serving

    def req(i, n_occ, n_virt, n_aux):
        return dict(index=i, n_occ=n_occ, n_frozen=n_occ // 6, n_virt=n_virt, n_aux=n_aux, n_targets=4,
                    seed=900 + i, t_arrival=0.0)
    reqs = [req(0, 30, 240, 810), req(1, 40, 320, 1080)] + [req(2 + i, 6, 48, 162) for i in range(10)]
    fp = [ltgw.request_footprint(serving.request_params(r, ltgw.LTGW_FP64), 4) for r in reqs]
    budget = fp[1] + (8 << 20)
    assert fp[0] + fp[2] <= budget < fp[0] + fp[1] and fp[1] + fp[2] > budget
    inputs = [serving.ingest(r, device=False) for r in reqs]
    srv = ltgw.Server(0, n_slots=2, hbm_budget_bytes=budget)
    try:
        recs, _, _ = serving.run_stream(srv, reqs, ltgw.LTGW_FP64, honor_arrivals=False, inputs=inputs)
    finally:
        srv.close()
    assert all(recs[r["index"]]["status"] in (ltgw.LTGW_OK, ltgw.LTGW_ERR_NO_CONVERGE) for r in reqs)
    big_start = recs[1]["start_ms"]
    passed = sum(1 for r in reqs[2:] if recs[r["index"]]["start_ms"] < big_start)
    assert passed == 8, passed
