"""Driver of the request server (ltgw_server) for a stream of G0W0 requests.

Requests are submitted at their arrival times; each request's inputs are
generated at arrival ("ingest": on the device for large requests, on the host
otherwise) and handed to the server, which admits them onto its worker slots
as slots and memory free up.  Latencies come from the server's completion
records (submit -> results); ingest time is reported separately.
"""
from __future__ import annotations

import time

import numpy as np

from . import ltgw
from . import synthetic as S

N_OMEGA, N_TAU, NAF_THRESH = 32, 8, 1e-2


def request_params(r: dict, precision: int):
    return ltgw.make_params(r["n_occ"], r["n_virt"], r["n_aux"], r["n_frozen"], N_OMEGA, N_TAU, 0.5, NAF_THRESH,
                            2, True, precision)


def ingest(r: dict, device: bool = True):
    """Inputs of one request: device tensors (generated on the GPU) or host arrays."""
    if device:
        import torch
        from .synthetic.device import DeviceLaw
        law = DeviceLaw(r["n_occ"], r["n_virt"], r["n_aux"], r["n_frozen"], r["seed"], r["n_targets"], gemm="tf32")
        inp = {"eps": torch.from_numpy(law.eps).cuda(), "B_ov": law.b_ov(), "B_tgt": law.b_tgt(),
               "targets": torch.from_numpy(law.targets.astype(np.int32)).cuda(),
               "shift": torch.from_numpy(law.shift).cuda()}
        torch.cuda.synchronize()
        return inp
    p = S.make_problem(r["n_occ"], r["n_virt"], r["n_aux"], r["n_frozen"], r["seed"], r["n_targets"])
    return {"eps": p.eps, "B_ov": p.B_ov, "B_tgt": p.B_tgt, "targets": p.targets.astype(np.int32), "shift": p.shift}


def run_stream(server: "ltgw.Server", requests, precision: int, device_ingest: bool = True,
               honor_arrivals: bool = True, inputs=None):
    """Submit every request at its arrival time; return per-request records."""
    recs = {}
    t0 = time.perf_counter()
    ingest_s = 0.0
    tickets = {}
    for k, r in enumerate(requests):
        if honor_arrivals:
            wait = t0 + r["t_arrival"] - time.perf_counter()
            if wait > 0:
                time.sleep(wait)
        ti = time.perf_counter()
        inp = inputs[k] if inputs is not None else ingest(r, device_ingest)
        ingest_s += time.perf_counter() - ti
        T = len(inp["targets"])
        sig, e, st = np.zeros((T, N_OMEGA, 2)), np.zeros(T), np.zeros(T, dtype=np.int32)
        tk = server.submit(request_params(r, precision), inp["eps"], inp["B_ov"], inp["B_tgt"], inp["targets"],
                           inp["shift"], sig, e, st)
        tickets[tk] = r["index"]
        recs[r["index"]] = {"e_qp": e, "qp_status": st, "sigma": sig}
        for c in server.poll():
            recs[tickets[c["ticket"]]].update(c)
    server.wait_all()
    wall = time.perf_counter() - t0
    for c in server.poll(4096):
        recs[tickets[c["ticket"]]].update(c)
    return recs, wall, ingest_s


def run_stream_pipelined(server: "ltgw.Server", requests, precision: int, mem_budget_bytes: int = 96 << 30):
    """Device ingest on a producer thread (its own stream), running ahead of the
    arrivals within mem_budget_bytes of generated inputs; each request is
    submitted at max(arrival, ready).  Records carry latency from submit
    (service + queueing) and from arrival (+ ingest wait)."""
    import queue
    import threading

    import torch

    ready = queue.Queue()
    held = {"bytes": 0}
    cv = threading.Condition()
    stop = {"flag": False}

    def nbytes(inp):
        return sum(v.numel() * v.element_size() for v in inp.values() if hasattr(v, "numel"))

    def producer():
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            for r in requests:
                with cv:
                    cv.wait_for(lambda: held["bytes"] < mem_budget_bytes or stop["flag"])
                if stop["flag"]:
                    return
                t = time.perf_counter()
                inp = ingest(r, device=True)
                s.synchronize()
                b = nbytes(inp)
                with cv:
                    held["bytes"] += b
                ready.put((r, inp, b, time.perf_counter() - t))

    th = threading.Thread(target=producer, daemon=True)
    t0 = time.perf_counter()
    th.start()
    recs, tickets, sizes = {}, {}, {}
    ingest_s = 0.0

    def drain(max_out=256):
        for c in server.poll(max_out):
            k = tickets[c["ticket"]]
            recs[k].update(c)
            recs[k]["latency_from_arrival_ms"] = (recs[k]["t_submit"] - t0 - requests[k]["t_arrival"]) * 1e3 + c["latency_ms"]
            with cv:
                held["bytes"] -= sizes.pop(k)
                recs[k]["inputs"] = None
                cv.notify_all()

    try:
        for _ in range(len(requests)):
            while True:
                try:
                    r, inp, b, dt = ready.get(timeout=0.005)
                    break
                except queue.Empty:
                    drain()
            ingest_s += dt
            wait = t0 + r["t_arrival"] - time.perf_counter()
            while wait > 0:
                drain()
                time.sleep(min(wait, 0.002))
                wait = t0 + r["t_arrival"] - time.perf_counter()
            T = len(inp["targets"])
            sig, e, st = np.zeros((T, N_OMEGA, 2)), np.zeros(T), np.zeros(T, dtype=np.int32)
            k = r["index"]
            recs[k] = {"e_qp": e, "qp_status": st, "sigma": sig, "t_submit": time.perf_counter(), "inputs": inp}
            sizes[k] = b
            tk = server.submit(request_params(r, precision), inp["eps"], inp["B_ov"], inp["B_tgt"],
                               inp["targets"], inp["shift"], sig, e, st)
            tickets[tk] = k
            drain()
        server.wait_all()
        drain(4096)
    finally:
        stop["flag"] = True
        with cv:
            cv.notify_all()
        th.join(timeout=60)
    return recs, time.perf_counter() - t0, ingest_s


def summarize(recs, wall_s: float, ingest_s: float) -> dict:
    lat = np.array([v["latency_ms"] for v in recs.values()])
    svc = np.array([v["service_ms"] for v in recs.values()])
    ok = sum(1 for v in recs.values() if v["status"] in (ltgw.LTGW_OK, ltgw.LTGW_ERR_NO_CONVERGE))
    out = {"requests": len(recs), "completed": ok, "wall_s": wall_s, "solves_per_s": len(recs) / wall_s,
           "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
           "service_p50_ms": float(np.percentile(svc, 50)), "ingest_s": ingest_s}
    la = [v["latency_from_arrival_ms"] for v in recs.values() if "latency_from_arrival_ms" in v]
    if la:
        out["p50_from_arrival_ms"] = float(np.percentile(la, 50))
        out["p99_from_arrival_ms"] = float(np.percentile(la, 99))
    return out
