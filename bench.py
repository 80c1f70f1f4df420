"""Benchmark of the LT-GW G0W0 hot path on one GB300 (or N independent replicas).

One step = one whole G0W0 solve through the C ABI: frozen-core slice, NAF
metric + eigensolver + projection, Laplace grid, Pi(tau_k) moments and their
frequency recombination, screening, W_nm, Sigma(i w), Pade and Newton.

Workload (default, --workload large): the large synthetic system, 320
occupied orbitals (60 frozen), 3500 virtual, 9000 auxiliary functions, NAF at
1e-2, 32 Gauss-Legendre frequencies, 10 Laplace points, 20 quasi-particle
states, the RI tensor streamed by blocks of occupied orbitals.  Default form:
mixed precision (split-BF16 tensor-core contractions, FP64 eigensolver /
screening / Pade / Newton); the plain FP64 form is timed on the same inputs
beside it, and both forms' quasi-particle energies are compared with the
oracle's stored results for this workload.  --workload mid / tiny: the smaller
systems (whole tensor resident).

Prints one JSON line.  --impl reference times the CPU oracle (direct AC-GW,
FP64, numpy) on the same workload instead (large: a bounded sample per step,
extrapolated to one solve).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

HA2MEV = 27211.386245988


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="large",
                    choices=["tiny", "mid", "large", "serving", "sweep", "eig", "request", "emu"])
    ap.add_argument("--req-occ", type=int, default=8,
                    help="request: n_occ of one serving-law request (launch-overhead measurement)")
    ap.add_argument("--eig-n", type=int, default=9000,
                    help="eig: size of the NAF metric whose eigensolver is timed (profiling workload)")
    ap.add_argument("--emu-pairs", type=int, default=140000,
                    help="emu: occupied-virtual pairs of the Pi contraction timed in both FP64 forms")
    ap.add_argument("--emu-slices", type=int, default=6, help="emu: integer slices per operand row")
    ap.add_argument("--sweep-size", default="mid", choices=["mid", "large"],
                    help="sweep: the workload whose GL x Laplace grids are swept")
    ap.add_argument("--occ-block", type=int, default=20, help="large: occupied orbitals per streamed block")
    ap.add_argument("--requests", type=int, default=512, help="serving: requests in the stream")
    ap.add_argument("--rate", type=float, default=None,
                    help="serving: Poisson arrival rate (requests/s); default 0.7 x the mixed form's measured "
                         "capacity (the whole stream closed loop)")
    ap.add_argument("--slots", type=int, default=4, help="serving: server worker slots")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="large: skip the end-to-end (host inputs) measurement")
    ap.add_argument("--no-fp64-form", action="store_true",
                    help="large: skip the plain FP64 form's solve (about three minutes) beside the timed form")
    ap.add_argument("--no-autotune", action="store_true",
                    help="mid / large: fixed contraction configurations instead of the library's autotuner")
    ap.add_argument("--precision", default="bf16x3", choices=["fp64", "bf16x3", "fp8", "fp8pi", "fp64emu"],
                    help="bf16x3: every contraction on the tensor cores with split-BF16 operands (eigensolver, "
                         "screening, Pade, Newton in FP64); fp8: Pi and W_nm in FP8 E4M3; fp8pi: Pi in FP8, the "
                         "rest as bf16x3; fp64: every step in FP64; fp64emu: FP64 with the contractions from "
                         "integer slices on the tensor cores")
    return ap.parse_args()


def workload(name, req_occ=8):
    """tiny / mid, or "request": one request of the serving law with n_occ = req_occ
    (frozen n_occ // 6, n_virt = 10 n_occ, N_aux = 3 (n_occ + n_virt), 4 states)."""
    from paper_2307_04508_gb300 import synthetic as S
    if name == "request":
        cfg = dict(n_occ=req_occ, n_frozen=req_occ // 6, n_virt=10 * req_occ, n_aux=33 * req_occ,
                   seed=20230720 + req_occ, n_targets=4, n_omega=32, n_tau=8, naf_thresh=1e-2)
    else:
        cfg = dict(S.MID if name == "mid" else S.TINY)
    prob = S.make_workload(cfg)
    desc = (f"{name}: n_occ={cfg['n_occ']} ({cfg['n_frozen']} frozen), n_virt={cfg['n_virt']}, "
            f"N_aux={cfg['n_aux']}, NAF eps={cfg['naf_thresh']}, N_omega={cfg['n_omega']}, "
            f"N_tau={cfg['n_tau']}, {cfg['n_targets']} QP states, LT+NAF+FC, synthetic Philox law")
    return cfg, prob, desc


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                if out:
                    self.rows.append([c.strip() for c in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if len(r) > 3 + i and "Active" in r[3 + i]
                          and "Not" not in r[3 + i]})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def fp64_alu_peak_tflops(sm_mhz=2070.0):
    # 152 SMs x 2 FP64 FMA per clock per SM (1.25 TFLOP/s nominal at 2070 MHz).
    return 152 * 2 * 2 * sm_mhz * 1e6 / 1e12


def oracle_solve(prob, cfg):
    from oracle import ltgw_oracle as O
    return O.solve(prob.eps, prob.B_ov, prob.B_tgt, prob.targets, prob.shift, prob.n_occ, prob.n_virt,
                   prob.n_frozen, n_omega=cfg["n_omega"], naf_thresh=cfg["naf_thresh"])


def run_reference(args):
    """The oracle (direct AC-GW, numpy FP64) on this host's cores, rank 0 only.
    mid / tiny: whole solves.  large: each step is the bounded sample of
    cpu_oracle_sample (half an occupied orbital's pairs), extrapolated to one
    solve; N_NAF is taken from the oracle's stored results for this workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = os.cpu_count()
    if args.workload == "large":
        from paper_2307_04508_gb300 import synthetic as S
        cfg = S.LARGE
        gold = golden_large()
        n_naf = gold["n_naf"] if gold else 2258
        prep = None
        for _ in range(args.warmup):
            _, _, _, prep, _ = cpu_oracle_sample(cfg, n_naf, frac=0.5, prep=prep)
        secs, desc = [], ""
        for _ in range(args.steps):
            sec, _, desc, prep, _ = cpu_oracle_sample(cfg, n_naf, frac=0.5, prep=prep)
            secs.append(sec)
        v = len(secs) / sum(secs)
        line = {"impl": "reference", "metric": "G0W0 solves/s", "value": v, "unit": "solves/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * np.mean(secs),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {"workload": LARGE_DESC, "form": "CPU oracle, direct AC-GW (no LT)"},
                "cpu_baseline": {"value": v, "unit": "solves/s", "cores": cores, "kind": "oracle",
                                 "sample": f"each step: {desc}"},
                "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    cfg, prob, desc = workload(args.workload)
    for _ in range(args.warmup):
        oracle_solve(prob, cfg)
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle_solve(prob, cfg)
        ts.append(time.perf_counter() - t0)
    v = len(ts) / sum(ts)
    line = {"impl": "reference", "metric": "G0W0 solves/s", "value": v, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(ts) / len(ts),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": desc, "form": "CPU oracle, direct AC-GW (no LT)"},
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} full solves of the {args.workload} workload"},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _solve_loop(ctx, p, dev, out_dev, stream, flush, steps, clk=None):
    """Time `steps` device-resident solves with CUDA events (L2 flushed between)."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    stats = []
    torch.cuda.synchronize()
    for i in range(steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        ev[i][0].record(stream)
        ctx.solve(p, dev["eps"], dev["B_ov"], dev["B_tgt"], dev["targets"], dev["shift"], *out_dev, stream=stream)
        ev[i][1].record(stream)
        stats.append(ctx.stats())
    torch.cuda.synchronize()
    return np.array([a.elapsed_time(b) for a, b in ev]), stats


PREC = {"fp64": 0, "bf16x3": 1, "fp8": 2, "fp8pi": 3, "fp64emu": 4}   # ltgw.LTGW_FP64 / BF16X3 / FP8 / FP8_PI / FP64_EMU
DTYPE = {"fp64": "f64", "bf16x3": "bf16x3", "fp8": "fp8e4m3", "fp8pi": "fp8e4m3 (Pi) + bf16x3",
         "fp64emu": "f64 (emulated: 6 x 7-bit integer slices on bf16 tensor cores)"}


def pi_roofline(prec, pi_flops, pi_ms, pk, src, traffic=None):
    """Roofline of the Pi-build kernel: algorithmic flops (SYRK as N^2 K) per launch
    over its CUDA-event time; split-BF16 does three tensor products per useful one."""
    if prec == "fp64":
        a = pi_flops / (pi_ms / 1e3) / 1e12
        peak = fp64_alu_peak_tflops(pk.get("sm_max_mhz", 2070.0))
        return {"bound": "alu", "kernel": "gemm_tile_kernel<double> (Pi(tau_k) moments, FP64 SYRK)", "achieved": a,
                "peak": peak, "unit": "TFLOP/s", "frac": a / peak,
                "peak_source": "FP64 FMA: 152 SMs x 2 FMA/clk x max SM clock (recipe unit counts)",
                "flops_per_launch": pi_flops, "ms_per_launch": pi_ms, "traffic": traffic}
    if prec == "fp64emu":
        a = 21 * pi_flops / (pi_ms / 1e3) / 1e12
        return {"bound": "tensor", "kernel": "tc_tma_ts_kernel (Pi(tau_k) moments from integer slices: 21 digit "
                                             "pairs, one BF16 product each)",
                "achieved": a, "peak": pk["bf16_tflops"], "unit": "TFLOP/s", "frac": a / pk["bf16_tflops"],
                "peak_source": f"bf16_tflops (burst) of {src} MEASURED_PEAKS.json",
                "flops_per_launch": 21 * pi_flops, "ms_per_launch": pi_ms, "traffic": traffic,
                "note": "issued tensor flops; the stage time includes the slicing and the FP64 pair sums"}
    if prec in ("fp8", "fp8pi"):
        a = 3 * pi_flops / (pi_ms / 1e3) / 1e12
        peak = 2.0 * pk["bf16_tflops"]
        return {"bound": "tensor", "kernel": "tc_fp8_kernel (Pi(tau_k) moments, FP8 E4M3 tcgen05 kind::f8f6f4)",
                "achieved": a, "peak": peak, "unit": "TFLOP/s", "frac": a / peak,
                "peak_source": f"2 x bf16_tflops (the nominal fp8 / bf16 dense ratio, 4.5 / 2.25 PFLOP/s) of {src} "
                               "MEASURED_PEAKS.json",
                "flops_per_launch": 3 * pi_flops, "ms_per_launch": pi_ms, "traffic": traffic,
                "note": "algorithmic flops (SYRK as N^2 K, three E4M3 products per useful one: the two-term "
                        "expansions); the padded 128 x 128 tiles do more MMA work; the quantisation pass before "
                        "the kernel is not in ms_per_launch"}
    tc = 3 * pi_flops / (pi_ms / 1e3) / 1e12
    return {"bound": "tensor", "kernel": "tc_tma_ts_kernel (Pi(tau_k) moments, split-BF16 tcgen05, A in TMEM)",
            "achieved": tc, "peak": pk["bf16_tflops"], "unit": "TFLOP/s", "frac": tc / pk["bf16_tflops"],
            "peak_source": f"bf16_tflops (burst, kernel of {pi_ms:.3f} ms) of {src} MEASURED_PEAKS.json",
            "flops_per_launch": 3 * pi_flops, "ms_per_launch": pi_ms, "traffic": traffic,
            "note": "algorithmic flops (SYRK as N^2 K, three BF16 products per useful one); the padded "
                    "128 x 128 tiles do more MMA work"}


def pi_error_vs_fp64(ctx, prob, N, n_omega, prec, stream):
    """Relative Frobenius error of Pi(i w_j) in the given tensor-core form against
    the FP64 form, both through the library's entry points, on the first N
    auxiliary rows of the active pairs (the NAF-basis Pi's shape), direct form
    (Eq. Pi) on the n_omega GL frequencies."""
    import torch
    from paper_2307_04508_gb300 import ltgw
    nf, no, nv = prob.n_frozen, prob.n_occ, prob.n_virt
    Bs = torch.from_numpy(np.ascontiguousarray(prob.B_ov[:N, nf * nv:])).cuda()
    delta = torch.from_numpy(np.ascontiguousarray(
        (prob.eps[no:][None, :] - prob.eps[nf:no][:, None]).reshape(-1))).cuda()
    om, _ = ltgw.gl_grid(n_omega, 0.5)
    ref = torch.empty((n_omega, N, N), dtype=torch.float64, device="cuda")
    got = torch.empty_like(ref)
    ctx.polarizability(Bs, delta, om, ref, spin=2, stream=stream)
    ctx.polarizability_mixed(Bs, delta, om, got, spin=2, stream=stream, fp8=prec in ("fp8", "fp8pi"))
    torch.cuda.synchronize()
    return float(torch.linalg.norm(got - ref) / torch.linalg.norm(ref))


def replicas_value(total_ms, steps, world, dist=None, device="cpu"):
    """Whole-job solves/s of `world` independent replicas, each timing `steps`
    solves in total_ms: the slowest rank's time bounds the job (max over ranks
    through `dist` when world > 1).  Returns (value, the max total_ms)."""
    total_ms = float(total_ms)
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return world * steps / (total_ms / 1e3), total_ms


def run_gpu(args):
    import torch
    from paper_2307_04508_gb300 import ltgw

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    cfg, prob, desc = workload(args.workload, args.req_occ)
    ctx = ltgw.Context(local)
    ctx.set_autotune(not args.no_autotune)   # the warm-up solves time and fix the configurations
    stream = torch.cuda.Stream()
    T = len(prob.targets)
    mixed = args.precision != "fp64"

    def params(prec):
        return ltgw.make_params(prob.n_occ, prob.n_virt, prob.n_aux, prob.n_frozen, cfg["n_omega"], cfg["n_tau"],
                                0.5, cfg["naf_thresh"], 2, True, prec)

    p = params(PREC[args.precision])
    p64 = params(ltgw.LTGW_FP64)
    dev = {"eps": torch.from_numpy(prob.eps).cuda(), "B_ov": torch.from_numpy(prob.B_ov).cuda(),
           "B_tgt": torch.from_numpy(prob.B_tgt).cuda(),
           "targets": torch.from_numpy(prob.targets.astype(np.int32)).cuda(),
           "shift": torch.from_numpy(prob.shift).cuda()}
    out_dev = (torch.empty((T, cfg["n_omega"], 2), dtype=torch.float64, device="cuda"),
               torch.empty(T, dtype=torch.float64, device="cuda"), torch.empty(T, dtype=torch.int32, device="cuda"))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # 256 MB > L2
    ctx.set_timing(True)
    # warm-up (also fits and caches the Laplace grid)
    for _ in range(max(args.warmup, 3)):
        ctx.solve(p, dev["eps"], dev["B_ov"], dev["B_tgt"], dev["targets"], dev["shift"], *out_dev, stream=stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    with ClockSampler(local) as clk:
        step_ms, stats = _solve_loop(ctx, p, dev, out_dev, stream, flush, args.steps)
    e_main = out_dev[1].cpu().numpy().copy()
    value, total_ms = replicas_value(step_ms.sum(), args.steps, world, dist, "cuda")
    st = stats[-1]
    launches = int(sum(x["kernel_launches"] for x in stats))
    N, n_ov = st["n_naf"], (prob.n_occ - prob.n_frozen) * prob.n_virt
    pi_flops = cfg["n_tau"] * N * N * n_ov            # useful flops of one Pi build (N^2 K per SYRK)
    pi_ms = float(np.mean([x["ms_pi_kernel"] for x in stats]))
    tri_ms = float(np.mean([x["ms_tridiag"] for x in stats]))
    pk, src = peaks()
    alu_peak = fp64_alu_peak_tflops(pk.get("sm_max_mhz", 2070.0))
    # DRAM bytes per launch (read + write) from the ncu captures summarised in profiles/
    # (tc_tma_ts_pi_mid.md, hh_fused_double_mid.md); mid workload only
    traffic_pi = 112.52e6 + 44.94e6 if args.workload == "mid" and args.precision == "bf16x3" else None
    traffic_tri = 25.98e6 + 0.05e6 if args.workload == "mid" else None
    roof_pi = pi_roofline(args.precision, pi_flops, pi_ms, pk, src, traffic_pi)
    # Householder reduction of the N_aux x N_aux metric: 4/3 N^3 algorithmic flops,
    # N - 2 steps of one grid barrier each (latency-bound at mid size)
    tri_flops = 4.0 / 3.0 * prob.n_aux ** 3
    tri_ach = tri_flops / (tri_ms / 1e3) / 1e12
    # FP64 in both forms (the mixed form lowers only the dense contractions)
    roof_tri = {"bound": "alu", "kernel": "hh_fused_kernel<double> (NAF Householder tridiagonalisation, FP64)",
                "achieved": tri_ach, "peak": alu_peak, "unit": "TFLOP/s", "frac": tri_ach / alu_peak,
                "peak_source": "FP64 FMA: 152 SMs x 2 FMA/clk x max SM clock (recipe unit counts)",
                "flops_per_launch": tri_flops, "ms_per_launch": tri_ms,
                "us_per_step": 1e3 * tri_ms / max(1, prob.n_aux - 2),
                "note": "full-storage fused form does 2 N^3 FP64 flops (the 4/3 N^3 counted here exploit "
                        "symmetry); one grid barrier (1.2 us measured alone) and five block barriers per "
                        "reflector on top",
                "traffic": traffic_tri}
    roofline = roof_tri if tri_ms > pi_ms else roof_pi
    clocks = clk.summary()
    line = {"metric": "G0W0 solves/s", "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.precision], "data": "synthetic",
            "config": {"workload": desc, "precision": args.precision,
                       "l2": "256 MB buffer written between steps; inputs 553 MB > L2",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
            "pi_build_tflops": pi_flops / (pi_ms / 1e3) / 1e12, "n_naf": N,
            "stage_ms": {k: st[k] for k in ("ms_naf", "ms_tridiag", "ms_pi", "ms_screen", "ms_wnm", "ms_sigma_qp",
                                            "ms_total")},
            "roofline": roofline, "roofline_pi_build": roof_pi, "gpu_launches": launches, "clocks": clocks,
            "peaks_source": src, "autotuned_shapes": st.get("tc_autotuned", 0)}
    if mixed:
        # the plain FP64 form on the same workload, for the "vs plain FP64 form" part of the metric
        ms64, _ = _solve_loop(ctx, p64, dev, out_dev, stream, flush, max(3, args.steps // 2))
        e64 = out_dev[1].cpu().numpy()
        line["fp64_form"] = {"solves_per_s": len(ms64) / (ms64.sum() / 1e3), "ms_per_solve": float(ms64.mean())}
        line["speedup_vs_fp64_form"] = value / line["fp64_form"]["solves_per_s"]
        line["qp_max_mev_vs_fp64_form"] = float(np.abs(e_main - e64).max() * HA2MEV)
        line["qp_mev_vs_fp64_form_per_state"] = (np.abs(e_main - e64) * HA2MEV).tolist()
        line["pi_rel_frob_vs_fp64_form"] = pi_error_vs_fp64(ctx, prob, N, cfg["n_omega"], args.precision, stream)
        # evGW, five cycles after G0W0 (the NAF basis and projections formed once), both forms
        ev = {}
        for name, pp in (("mixed", p), ("fp64", p64)):
            T_ = len(prob.targets)
            sg, ee, ss = (np.zeros((T_, cfg["n_omega"], 2)), np.zeros(T_), np.zeros(T_, dtype=np.int32))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.solve_ev(pp, dev["eps"], dev["B_ov"], dev["B_tgt"], dev["targets"], dev["shift"], sg, ee, ss,
                         n_cycles=5, stream=stream)
            ev[name] = {"ms": 1e3 * (time.perf_counter() - t0), "e": ee.copy()}
        line["evgw_5_cycles"] = {"ms_mixed": ev["mixed"]["ms"], "ms_fp64_form": ev["fp64"]["ms"],
                                 "speedup": ev["fp64"]["ms"] / ev["mixed"]["ms"],
                                 "qp_max_mev_vs_fp64_form": float(np.abs(ev["mixed"]["e"] - ev["fp64"]["e"]).max()
                                                                  * HA2MEV),
                                 "note": "host wall time of one ltgw_solve_ev call (device inputs)"}
    # end-to-end: host (pinned) inputs and outputs through the same C ABI call
    pin = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in
           {"eps": prob.eps, "B_ov": prob.B_ov, "B_tgt": prob.B_tgt,
            "targets": prob.targets.astype(np.int32), "shift": prob.shift}.items()}
    out_host = (torch.empty((T, cfg["n_omega"], 2), dtype=torch.float64).pin_memory(),
                torch.empty(T, dtype=torch.float64).pin_memory(), torch.empty(T, dtype=torch.int32).pin_memory())
    # bytes the call moves host -> device: every input but the frozen-core
    # columns of B_ov, which it never reads and does not copy
    h2d = (sum(v.numel() * v.element_size() for v in pin.values())
           - prob.n_aux * prob.n_frozen * prob.n_virt * pin["B_ov"].element_size())
    d2h = sum(v.numel() * v.element_size() for v in out_host)
    for _ in range(2):
        ctx.solve(p, pin["eps"], pin["B_ov"], pin["B_tgt"], pin["targets"], pin["shift"], *out_host, stream=stream)
    torch.cuda.synchronize()
    e2e_steps = max(3, args.steps // 2)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ctx.solve(p, pin["eps"], pin["B_ov"], pin["B_tgt"], pin["targets"], pin["shift"], *out_host, stream=stream)
    torch.cuda.synchronize()
    line["e2e"] = {"value": world * e2e_steps / (time.perf_counter() - t0), "unit": "solves/s",
                   "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # bounded oracle sample: full solves of the same workload on the host cores
        t0 = time.perf_counter()
        n = 0
        e_o = None
        while n < 2 and (time.perf_counter() - t0) < 25.0:
            _, e_o, _ = oracle_solve(prob, cfg)
            n += 1
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": n / dt, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"{n} full direct-AC solve(s) of the same workload (numpy FP64)"}
        line["qp_max_mev_vs_fp64_direct_oracle"] = float(np.abs(e_main - e_o).max() * HA2MEV)
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


def run_serving(args):
    """The serving stream: requests of mixed sizes (n_occ log-uniform in [8, 200],
    N_aux = 3 (n_occ + n_virt)) arriving as a Poisson process, inputs generated on
    the device at arrival, admitted onto the request server's slots.  The same
    stream (same requests, same arrival times) is served in the mixed form and
    in the plain FP64 form; the arrival rate is 0.7 x the mixed form's capacity
    (the whole stream closed loop)."""
    import torch
    from paper_2307_04508_gb300 import ltgw, serving
    from paper_2307_04508_gb300 import synthetic as S

    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    # the server's admission budget and the ingest thread's budget for generated
    # inputs share the device: 55 % + 15 % of it, leaving room for the contexts
    total = torch.cuda.get_device_properties(0).total_memory
    budget, ingest_budget = int(0.55 * total), int(0.15 * total)
    mixed_prec = PREC[args.precision] if args.precision != "fp64" else ltgw.LTGW_BF16X3

    def serve(reqs, prec, clk=None):
        srv = ltgw.Server(0, n_slots=args.slots, hbm_budget_bytes=budget)
        try:
            recs, wall, ingest_s = serving.run_stream_pipelined(srv, reqs, prec, mem_budget_bytes=ingest_budget)
        finally:
            srv.close()
        return recs, wall, ingest_s

    # capacity: the whole stream closed loop (all arriving at once), mixed form
    burst = S.serving_stream(args.requests, rate_hz=1e9)
    recs_c, wall_c, _ = serve(burst, mixed_prec)
    capacity = len(recs_c) / wall_c
    rate = args.rate if args.rate else 0.7 * capacity
    reqs = S.serving_stream(args.requests, rate_hz=rate)
    out = {}
    with ClockSampler(local) as clk:
        for name, prec in (("mixed", mixed_prec), ("fp64", ltgw.LTGW_FP64)):
            recs, wall, ingest_s = serve(reqs, prec)
            sm = serving.summarize(recs, wall, ingest_s)
            out[name] = {"recs": recs, "summary": sm}
    failures = [{"form": name, "index": k, "status": v.get("status"), "message": v.get("message", "")}
                for name in out for k, v in out[name]["recs"].items()
                if v.get("status") not in (ltgw.LTGW_OK, ltgw.LTGW_ERR_NO_CONVERGE)]
    ok = (ltgw.LTGW_OK, ltgw.LTGW_ERR_NO_CONVERGE)
    both = [k for k in out["fp64"]["recs"] if out["fp64"]["recs"][k].get("status") in ok
            and out["mixed"]["recs"].get(k, {}).get("status") in ok]
    dev = max(float(np.abs(out["mixed"]["recs"][k]["e_qp"] - out["fp64"]["recs"][k]["e_qp"]).max())
              for k in both) * HA2MEV if both else None
    sm, s64 = out["mixed"]["summary"], out["fp64"]["summary"]

    def lat(x):
        return {"p50": x["p50_ms"], "p99": x["p99_ms"], "p50_from_arrival": x.get("p50_from_arrival_ms"),
                "p99_from_arrival": x.get("p99_from_arrival_ms"), "service_p50": x["service_p50_ms"]}
    line = {"metric": "G0W0 solves/s (serving stream)", "value": sm["solves_per_s"], "unit": "solves/s",
            "n_gpus": 1, "steps": len(reqs), "warmup": 0, "ms_per_step": 1e3 * sm["wall_s"] / len(reqs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.precision]
            if args.precision != "fp64" else "bf16x3", "data": "synthetic",
            "config": {"workload": f"serving: {len(reqs)} requests, Poisson {rate:.3f}/s "
                                   + ("" if args.rate else f"= 0.7 x the measured capacity {capacity:.3f} solves/s "
                                   "(the same stream closed loop, device ingest included), ")
                                   + "n_occ log-uniform [8,200], n_virt = u n_occ (u in [8,12]), "
                                   "N_aux = 3(n_occ+n_virt), NAF 1e-2, N_omega 32, N_tau 8, 4 states; inputs "
                                   "generated on the device at arrival; both forms on the same arrival times",
                       "slots": args.slots, "hbm_budget_bytes": budget},
            "latency_ms": lat(sm), "completed": sm["completed"], "ingest_s": sm["ingest_s"],
            "fp64_form": {"solves_per_s": s64["solves_per_s"], "latency_ms": lat(s64), "completed": s64["completed"],
                          "wall_s": s64["wall_s"]},
            "speedup_vs_fp64_form": sm["solves_per_s"] / s64["solves_per_s"],
            "qp_max_mev_mixed_vs_fp64_form": dev, "qp_compared_requests": len(both),
            "capacity_solves_per_s": capacity, "failures": failures,
            "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)


LARGE_DESC = ("large: n_occ=320 (60 frozen), n_virt=3500, "
              "N_aux=9000, NAF 1e-2, N_omega=32, N_tau=10 (library minimax Laplace grid), 20 QP states, "
              "LT+NAF+FC, seed 20230712; RI tensor from the synthetic Philox law in FP64 (QR on the host, "
              "normals and loading GEMM on the device), held by the caller in 13 blocks of 20 occupied orbitals and streamed "
              "through ltgw_solve_streamed (the library holds two blocks, never the whole tensor)")


def golden_large():
    """The oracle's stored results for the large workload (tests/golden/large_g0w0.json), or None."""
    path = os.path.join(ROOT, "tests", "golden", "large_g0w0.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        return json.load(fh)


def large_inputs(cfg, occ_block, host=False):
    """The large workload's inputs, generated on the device in FP64: eps, targets,
    shift (host numpy), the active B_ov blocks (device tensors, or pinned host
    copies with host=True) and B_tgt.  Returns (law, blocks, B_tgt, seconds)."""
    import torch
    from paper_2307_04508_gb300.synthetic.device import DeviceLaw
    t0 = time.perf_counter()
    law = DeviceLaw(cfg["n_occ"], cfg["n_virt"], cfg["n_aux"], cfg["n_frozen"], cfg["seed"], cfg["n_targets"],
                    gemm="fp64", host_qr=True)
    blocks = []
    for i0 in range(cfg["n_frozen"], cfg["n_occ"], occ_block):
        blocks.append(law.b_ov_block(i0, min(cfg["n_occ"], i0 + occ_block)))
    B_tgt = law.b_tgt()
    torch.cuda.synchronize()
    return law, blocks, B_tgt, time.perf_counter() - t0


def cpu_oracle_sample(cfg, n_naf, frac=1.0, prep=None, L=None):
    """Time the oracle (direct AC, numpy FP64, this host's cores) on a bounded
    sample of the large workload and extrapolate one whole solve.  The sample
    runs each of the oracle's steps on a slice whose cost scales in a known
    way: the NAF metric, the projection and Pi (Eq. Pi, all N_omega
    frequencies) on the pairs of `frac` of one occupied orbital (x n_pairs /
    sample pairs); the eigendecomposition on the leading n_s x n_s block of the
    sampled metric (x (N_aux / n_s)^3); the screening on 2 of the N_omega
    matrices (x N_omega / 2); W_nm for 1 target at 1 frequency (x T N_omega);
    Sigma, Pade and Newton in full on stand-in W.  Returns (seconds per
    extrapolated solve, sample seconds, description, prep)."""
    from oracle import ltgw_oracle as O
    from paper_2307_04508_gb300 import synthetic as S
    no, nv, na, nf, seed = cfg["n_occ"], cfg["n_virt"], cfg["n_aux"], cfg["n_frozen"], cfg["seed"]
    n_act, T, n_om = no - nf, cfg["n_targets"], cfg["n_omega"]
    n_orb_act = no + nv - nf
    if prep is None:   # inputs of the sample (untimed): the law on the host in FP64
        eps = S.orbital_energies(seed, no, nv, nf)
        L = S.aux_loading(seed, na, no, nv) if L is None else L
        R = L @ S.pair_normals_ov(seed, na, no, nv, nf, nf + 1)
        Rt = L @ S.pair_normals_row(seed, na, no + nv, no - 1)
        prep = {"eps": eps, "L": L, "R": R, "Rt": Rt}
    eps, L = prep["eps"], prep["L"]
    m = max(64, int(round(frac * nv)))
    R = np.ascontiguousarray(prep["R"][:, :m])
    n_s = min(na, max(256, int(round(3000 * frac ** (1 / 3)))))
    parts = {}
    t0 = time.perf_counter()
    t = time.perf_counter()
    K = O.naf_metric(R)
    parts["naf_metric"] = (time.perf_counter() - t) * n_act * nv / m
    t = time.perf_counter()
    O.naf_basis(np.ascontiguousarray(K[:n_s, :n_s]), cfg["naf_thresh"])
    parts["naf_eig"] = (time.perf_counter() - t) * (na / n_s) ** 3
    U = np.ascontiguousarray(L[:, :n_naf])           # timing stand-in of the kept basis (same shape)
    t = time.perf_counter()
    Bt = O.naf_project(R, U)
    parts["naf_project"] = (time.perf_counter() - t) * n_act * nv / m
    t = time.perf_counter()
    Bt_tgt = O.naf_project(prep["Rt"][:, nf:], U)[None]
    parts["naf_project"] += (time.perf_counter() - t) * T
    om, wt = O.gl_grid(n_om, 0.5)
    delta = (eps[no:no + nv][:m] - eps[nf]).astype(np.float64)
    t = time.perf_counter()
    Pi = O.polarizability_direct(Bt, delta, om, 2)
    parts["pi"] = (time.perf_counter() - t) * n_act * nv / m
    t = time.perf_counter()
    C = O.screened_interaction(Pi[:2])
    parts["screen"] = (time.perf_counter() - t) * n_om / 2
    t = time.perf_counter()
    O.w_nm(C[:1], Bt_tgt)
    parts["w_nm"] = (time.perf_counter() - t) * T * n_om
    W = -np.abs(np.random.default_rng(0).standard_normal((T, n_orb_act, n_om))) * 1e-3
    t = time.perf_counter()
    eF = O.fermi_level(eps, no)
    sig = O.sigma_iw(W, eps[nf:], eF, om, wt)
    sel = O.pade_nodes(n_om)
    for k in range(T):
        a = O.pade_coefficients(1j * om[sel], sig[k][sel])
        O.qp_newton(eps[no - 1], 0.0, eF, 1j * om[sel], a)
    parts["sigma_pade_qp"] = time.perf_counter() - t
    sample_s = time.perf_counter() - t0
    desc = (f"oracle steps on a slice, extrapolated to one solve: NAF metric, projection and direct Pi "
            f"({n_om} frequencies) on {m} of the {n_act * nv} active pairs (x {n_act * nv / m:.0f}); eigh of the "
            f"leading {n_s} x {n_s} metric block (x ({na}/{n_s})^3); screening of 2 of {n_om} matrices; W_nm for "
            f"1 target x 1 frequency (x {T * n_om}); Sigma/Pade/Newton in full; N_NAF = {n_naf}")
    return sum(parts.values()), sample_s, desc, prep, parts


def run_large(args):
    """The large system (FP64 form, or its mixed forms), streamed
    by occupied blocks from inputs resident in HBM.  `value`: solves/s of the
    chosen form; the plain FP64 form beside it (one solve); QP errors against
    the oracle's stored results; e2e through the same C ABI call with the
    blocks in pinned host memory."""
    import torch
    from paper_2307_04508_gb300 import ltgw
    from paper_2307_04508_gb300 import synthetic as S

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    cfg = S.LARGE
    ob = args.occ_block
    law, blocks, B_tgt, gen_s = large_inputs(cfg, ob)
    eps = torch.from_numpy(law.eps).cuda()
    targets = torch.from_numpy(law.targets.astype(np.int32)).cuda()
    shift = torch.from_numpy(law.shift).cuda()
    T = len(law.targets)
    n_om = cfg["n_omega"]
    src = ltgw.BlockSource(blocks, cfg["n_frozen"], ob, cfg["n_virt"])

    def params(prec):
        return ltgw.make_params(cfg["n_occ"], cfg["n_virt"], cfg["n_aux"], cfg["n_frozen"], n_om, cfg["n_tau"],
                                0.5, cfg["naf_thresh"], 2, True, PREC[prec])

    p, p64 = params(args.precision), params("fp64")
    ctx = ltgw.Context(0)
    ctx.set_timing(True)
    ctx.set_autotune(not args.no_autotune)   # the warm-up solves time and fix the configurations
    stream = torch.cuda.Stream()
    out = (torch.empty((T, n_om, 2), dtype=torch.float64, device="cuda"),
           torch.empty(T, dtype=torch.float64, device="cuda"), torch.empty(T, dtype=torch.int32, device="cuda"))

    def timed(pp, n):
        ms, stats = [], []
        for _ in range(n):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            ctx.solve_streamed(pp, eps, src, ob, B_tgt, targets, shift, *out, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            stats.append(ctx.stats())
        return np.array(ms), stats

    timed(p, max(args.warmup, 3))
    if dist:
        dist.barrier()
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        step_ms, stats = timed(p, args.steps)
    e_main = out[1].cpu().numpy().copy()
    st_main = out[2].cpu().numpy().copy()
    value, total_ms = replicas_value(step_ms.sum(), args.steps, world, dist, "cuda")
    st = stats[-1]
    N, n_ov = st["n_naf"], (cfg["n_occ"] - cfg["n_frozen"]) * cfg["n_virt"]
    pi_flops = cfg["n_tau"] * N * N * n_ov
    pi_ms = float(np.mean([x["ms_pi_kernel"] for x in stats]))
    tri_ms = float(np.mean([x["ms_tridiag"] for x in stats]))
    pk, src_pk = peaks()
    alu_peak = fp64_alu_peak_tflops(pk.get("sm_max_mhz", 2070.0))
    roof_pi = pi_roofline(args.precision, pi_flops, pi_ms, pk, src_pk, LARGE_TRAFFIC.get(("pi", args.precision)))
    tri_flops = 4.0 / 3.0 * cfg["n_aux"] ** 3
    tri_ach = tri_flops / (tri_ms / 1e3) / 1e12
    roof_tri = {"bound": "alu", "kernel": "hh_fused_kernel<double> (NAF Householder tridiagonalisation, FP64)",
                "achieved": tri_ach, "peak": alu_peak, "unit": "TFLOP/s", "frac": tri_ach / alu_peak,
                "peak_source": "FP64 FMA: 152 SMs x 2 FMA/clk x max SM clock (recipe unit counts)",
                "flops_per_launch": tri_flops, "ms_per_launch": tri_ms,
                "note": "4/3 N^3 algorithmic flops of the reduction (symmetry exploited); N = N_aux = 9000",
                "traffic": LARGE_TRAFFIC.get(("hh", "any"))}
    roofline = roof_tri if tri_ms > pi_ms else roof_pi
    gold = golden_large()
    line = {"metric": "G0W0 solves/s", "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.precision], "data": "synthetic",
            "config": {"workload": LARGE_DESC, "precision": args.precision,
                       "l2": "inputs 65.5 GB (> L2) streamed each step; no flush needed",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                           "note": "per solve over the timed steps (one request at a time)"},
            "pi_build_tflops": pi_flops / (pi_ms / 1e3) / 1e12, "n_naf": N,
            "stage_ms": {k: float(np.mean([x[k] for x in stats])) for k in
                         ("ms_naf", "ms_naf_metric", "ms_tridiag", "ms_eig_vectors", "ms_naf_project", "ms_pi",
                          "ms_pi_kernel", "ms_screen", "ms_wnm", "ms_sigma_qp", "ms_total")},
            "roofline": roofline, "roofline_pi_build": roof_pi,
            "gpu_launches": int(sum(x["kernel_launches"] for x in stats)), "clocks": clk.summary(),
            "peaks_source": src_pk, "input_generation_s": gen_s, "qp_status": st_main.tolist()}
    if gold is not None:
        ed = np.array(gold["direct"]["e_qp"])
        line["qp_mev_vs_fp64_oracle_per_state"] = (np.abs(e_main - ed) * HA2MEV).tolist()
        line["qp_max_mev_vs_fp64_oracle"] = float(np.abs(e_main - ed).max() * HA2MEV)
        line["oracle_reference"] = ("tests/golden/large_g0w0.json: the oracle's direct AC-GW solve (Eq. Pi, no "
                                    "Laplace transform) on the same law, written on the host in FP64")
    if args.precision != "fp64" and not args.no_fp64_form:
        ms64, _ = timed(p64, 1)
        e64 = out[1].cpu().numpy().copy()
        line["fp64_form"] = {"solves_per_s": 1e3 / float(ms64.mean()), "ms_per_solve": float(ms64.mean()),
                             "solves_timed": 1}
        line["speedup_vs_fp64_form"] = value / line["fp64_form"]["solves_per_s"]
        line["qp_max_mev_vs_fp64_form"] = float(np.abs(e_main - e64).max() * HA2MEV)
        if gold is not None:
            line["fp64_form"]["qp_max_mev_vs_fp64_oracle"] = float(
                np.abs(e64 - np.array(gold["direct"]["e_qp"])).max() * HA2MEV)
        if args.precision != "fp64emu":
            # the FP64-accurate form with its contractions from integer slices: one
            # warm-up solve (the autotuner fixes its shapes), one timed
            pe = params("fp64emu")
            timed(pe, 1)
            mse, ste = timed(pe, 1)
            ee = out[1].cpu().numpy().copy()
            line["fp64_emulated_form"] = {
                "solves_per_s": 1e3 / float(mse.mean()), "ms_per_solve": float(mse.mean()), "solves_timed": 1,
                "qp_max_ha_vs_fp64_form": float(np.abs(ee - e64).max()),
                "stage_ms": {k: float(ste[-1][k]) for k in ("ms_naf_metric", "ms_tridiag", "ms_eig_vectors",
                                                            "ms_naf_project", "ms_pi", "ms_screen", "ms_wnm")}}
            if gold is not None:
                line["fp64_emulated_form"]["qp_max_mev_vs_fp64_oracle"] = float(
                    np.abs(ee - np.array(gold["direct"]["e_qp"])).max() * HA2MEV)
            line["speedup_vs_fp64_emulated_form"] = value / line["fp64_emulated_form"]["solves_per_s"]
    if args.no_e2e:
        if rank == 0:
            print(json.dumps(line), flush=True)
        ctx.close()
        return
    # end to end: the caller's blocks and B_tgt in pinned host memory, outputs to host
    host_blocks = [b.cpu().pin_memory() for b in blocks]
    del src, blocks
    torch.cuda.empty_cache()
    hsrc = ltgw.BlockSource(host_blocks, cfg["n_frozen"], ob, cfg["n_virt"])
    h_in = {"eps": np.ascontiguousarray(law.eps), "B_tgt": B_tgt.cpu().pin_memory(),
            "targets": np.ascontiguousarray(law.targets.astype(np.int32)), "shift": np.ascontiguousarray(law.shift)}
    del B_tgt
    h_out = (np.zeros((T, n_om, 2)), np.zeros(T), np.zeros(T, dtype=np.int32))
    ctx.solve_streamed(p, h_in["eps"], hsrc, ob, h_in["B_tgt"], h_in["targets"], h_in["shift"], *h_out,
                       stream=stream)
    n_e2e = max(1, min(args.steps, 5))
    hsrc.bytes_copied = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        ctx.solve_streamed(p, h_in["eps"], hsrc, ob, h_in["B_tgt"], h_in["targets"], h_in["shift"], *h_out,
                           stream=stream)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    h2d = hsrc.bytes_copied / n_e2e + sum(v.nbytes if isinstance(v, np.ndarray) else v.numel() * v.element_size()
                                          for v in h_in.values())
    line["e2e"] = {"value": world * n_e2e / dt, "unit": "solves/s", "h2d_bytes_per_step": int(h2d),
                   "d2h_bytes_per_step": int(sum(a.nbytes for a in h_out)), "steps": n_e2e,
                   "note": "ltgw_solve_streamed with host inputs: every active block crosses the link once per "
                           "solve from pinned memory (the split copy kept from the metric's pass feeds the "
                           "projection), overlapped with the previous block's work; B_tgt, eps, targets, shift "
                           "from host; results to host"}
    line["e2e_qp_max_mev_vs_device_inputs"] = float(np.abs(h_out[1] - e_main).max() * HA2MEV)
    del host_blocks, hsrc
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sec, sample_s, desc, _, parts = cpu_oracle_sample(cfg, N, L=law.L.cpu().numpy())
        line["cpu_baseline"] = {"value": 1.0 / sec, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"{desc}; sample ran {sample_s:.1f} s",
                                "extrapolated_s_per_solve": sec, "parts_s": parts}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


# DRAM bytes (read + write) per launch at the large workload, from the ncu
# captures summarised in profiles/ (None until captured for the current kernels):
# the Householder reduction at N_aux = 9000, profiles/hh_fused_double_large.md
# (dram__bytes_read.sum 1.835 TB + dram__bytes_write.sum 1.881 TB)
LARGE_TRAFFIC = {("hh", "any"): 1.835e12 + 1.881e12}


def run_sweep(args):
    """GL x Laplace grid sweep (the paper's grid comparison of Sec. 4.1, here on
    the synthetic workloads): for N_omega in {32, 64, 128} and N_tau in
    {8, 10, 12, 14, 18} (Eq. LT's form, library grid) the solve time and the
    largest QP deviation from the reference, direct AC (no Laplace transform)
    with 128 GL points, all in the split-BF16 form.  Times exclude the input
    generation of the streamed large workload."""
    import torch
    from paper_2307_04508_gb300 import ltgw
    from paper_2307_04508_gb300 import synthetic as S

    torch.cuda.set_device(0)
    ctx = ltgw.Context(0)
    ctx.set_timing(True)
    stream = torch.cuda.Stream()
    large = args.sweep_size == "large"
    if large:
        from paper_2307_04508_gb300.synthetic.device import DeviceLaw
        cfg = S.LARGE
        law = DeviceLaw(cfg["n_occ"], cfg["n_virt"], cfg["n_aux"], cfg["n_frozen"], cfg["seed"], cfg["n_targets"],
                        gemm="fp32")
        dims = (cfg["n_occ"], cfg["n_virt"], cfg["n_aux"], cfg["n_frozen"])
        B_tgt = law.b_tgt()
        eps = torch.from_numpy(law.eps).cuda()
        targets = torch.from_numpy(law.targets.astype(np.int32)).cuda()
        shift = torch.from_numpy(law.shift).cuda()
        grids = [(32, 0), (32, 8), (32, 12), (32, 18), (128, 8), (128, 12), (128, 18)]
        reps = 1
    else:
        cfg = dict(S.MID)
        prob = S.make_workload(cfg)
        dims = (prob.n_occ, prob.n_virt, prob.n_aux, prob.n_frozen)
        dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in
               (prob.eps, prob.B_ov, prob.B_tgt, prob.targets.astype(np.int32), prob.shift)]
        grids = [(n_om, n_tau) for n_om in (32, 64, 128) for n_tau in (0, 8, 10, 12, 14, 18)]
        reps = 3
    T = cfg["n_targets"] if large else len(prob.targets)

    def run(n_om, n_tau):
        p = ltgw.make_params(*dims, n_om, n_tau, 0.5, cfg["naf_thresh"], 2, n_tau > 0, ltgw.LTGW_BF16X3)
        out = (torch.empty((T, n_om, 2), dtype=torch.float64, device="cuda"),
               torch.empty(T, dtype=torch.float64, device="cuda"), torch.empty(T, dtype=torch.int32, device="cuda"))
        ms = []
        for r in range(reps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if large:
                ctx.solve_streamed(p, eps, lambda i0, i1, dst, strm: law.fill_block(i0, i1, dst), args.occ_block,
                                   B_tgt, targets, shift, *out, stream=stream)
            else:
                ctx.solve(p, *dev, *out, stream=stream)
            torch.cuda.synchronize()
            if r:   # the first run warms up
                ms.append(1e3 * (time.perf_counter() - t0) - ctx.stats()["ms_generate"])
        return float(np.median(ms)), out[1].cpu().numpy().copy(), out[2].cpu().numpy().copy()

    t_ref, e_ref, st_ref = run(128, 0)
    rows = []
    with ClockSampler(0) as clk:
        for n_om, n_tau in grids:
            t, e, st = run(n_om, n_tau)
            rows.append({"n_omega": n_om, "n_tau": n_tau, "ms": t, "speedup_vs_reference": t_ref / t,
                         "qp_max_mev_vs_reference": float(np.abs(e - e_ref).max() * HA2MEV),
                         "converged": bool(np.all(st == 0))})
    line = {"metric": "GL x Laplace grid sweep (speed-up and QP deviation vs direct AC, 128 GL)",
            "unit": "ms per solve", "workload": args.sweep_size, "precision": "bf16x3",
            "reference": {"n_omega": 128, "n_tau": 0, "ms": t_ref, "converged": bool(np.all(st_ref == 0))},
            "rows": rows, "clocks": clk.summary(), "data": "synthetic"}
    print(json.dumps(line), flush=True)
    ctx.close()


def run_eig(args):
    """The NAF eigensolver alone (ltgw_naf_basis, FP64) on the metric of an
    --eig-n x --eig-n block of the synthetic law's RI tensor without its
    rotation (--eig-n pairs), a few GB on the device: the profiling workload
    of the eigensolver's kernels at the large workload's N_aux."""
    import torch
    from paper_2307_04508_gb300 import ltgw
    from paper_2307_04508_gb300.synthetic import device as D
    torch.cuda.set_device(0)
    n = args.eig_n
    nv = 3500
    occ = max(1, (n + nv - 1) // nv)
    # sigma_r Z[r, pairs] / sqrt(n_occ n_virt): the law without its rotation U
    # (the metric's eigenvalues do not depend on U; no QR needed here)
    sig = 0.5 * torch.exp(-6.0 * torch.arange(n, dtype=torch.float64, device="cuda") / n) / np.sqrt(320 * nv)
    B = (D.pair_normals_ov(20230712, n, 320, nv, 60, 60 + occ)[:, :n] * sig[:, None]).contiguous()
    Ut = torch.empty((n, n), dtype=torch.float64, device="cuda")
    lam = torch.empty(n, dtype=torch.float64, device="cuda")
    ctx = ltgw.Context(0)
    ctx.set_timing(True)
    thresh = 1e-2 * occ / 260.0   # the large workload's threshold, scaled to this block's share of the pairs
    rows = []
    for it in range(args.warmup + args.steps):
        k = ctx.naf_basis(B, n, n, thresh, Ut, lam)
        st = ctx.stats()
        if it >= args.warmup:
            rows.append(st)
    tri = float(np.mean([r["ms_tridiag"] for r in rows]))
    line = {"metric": "NAF eigensolver (profiling workload)", "n": n, "n_naf": k, "steps": args.steps,
            "ms_tridiag": tri, "ms_eig_vectors": float(np.mean([r["ms_eig_vectors"] for r in rows])),
            "ms_naf_metric": float(np.mean([r["ms_naf_metric"] for r in rows])),
            "tridiag_tflops": 4.0 / 3.0 * n ** 3 / (tri / 1e3) / 1e12, "launches": rows[-1]["kernel_launches"]}
    print(json.dumps(line), flush=True)
    ctx.close()


def run_emu(args):
    """The Pi contraction at the large workload's shape (N = 2258 natural
    auxiliary functions, the 10-point Laplace form, 32 frequencies) over
    --emu-pairs occupied-virtual pairs (the pair gaps of the large law's
    first active occupied orbitals; R~ rows Gaussian with the decaying norms
    of NAF-projected rows): the plain FP64 form (ltgw_polarizability, FP64
    pipe) beside the FP64-accurate slice form (ltgw_polarizability_emulated,
    tensor cores), each timed with CUDA events on the launching stream after
    warm-up; the slice form's error against the FP64 one."""
    import torch
    from paper_2307_04508_gb300 import ltgw
    from paper_2307_04508_gb300 import synthetic as S
    torch.cuda.set_device(0)
    cfg = S.LARGE
    N, P, n_tau, n_om = 2258, args.emu_pairs, cfg["n_tau"], cfg["n_omega"]
    nv, nf, no = cfg["n_virt"], cfg["n_frozen"], cfg["n_occ"]
    eps = S.orbital_energies(cfg["seed"], no, nv, nf)
    n_i = (P + nv - 1) // nv
    delta = (eps[no:no + nv][None, :] - eps[nf:nf + n_i][:, None]).reshape(-1)[:P]
    gen = torch.Generator(device="cuda")
    gen.manual_seed(cfg["seed"])
    row = 0.05 * torch.exp(-6.0 * torch.arange(N, dtype=torch.float64, device="cuda") / N)
    Bt = torch.randn((N, P), generator=gen, dtype=torch.float64, device="cuda") * row[:, None]
    d_delta = torch.from_numpy(np.ascontiguousarray(delta)).cuda()
    om, _ = ltgw.gl_grid(n_om, 0.5)
    gap = float(delta.min())
    x, w, lt_err = ltgw.laplace_grid(n_tau, gap * gap + om[0] * om[0], max(float(delta.max()) ** 2, 1e4))
    Pi64 = torch.empty((n_om, N, N), dtype=torch.float64, device="cuda")
    PiE = torch.empty_like(Pi64)
    ctx = ltgw.Context(0)
    ctx.set_timing(True)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]

    def timed(fn):
        ms = []
        for it in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            ev[0].record(stream)
            fn()
            ev[1].record(stream)
            torch.cuda.synchronize()
            if it >= args.warmup:
                ms.append(ev[0].elapsed_time(ev[1]))
        return float(np.mean(ms))

    ms_e = timed(lambda: ctx.polarizability_emulated(Bt, d_delta, om, PiE, spin=2, x=x, w=w,
                                                     n_slices=args.emu_slices, stream=stream))
    st = ctx.stats()
    ms_64 = timed(lambda: ctx.polarizability(Bt, d_delta, om, Pi64, spin=2, x=x, w=w, stream=stream))
    rel = float(torch.linalg.vector_norm(PiE - Pi64) / torch.linalg.vector_norm(Pi64))
    mx = float((PiE - Pi64).abs().max() / Pi64.abs().max())
    s = args.emu_slices
    pairs = sum(1 for i in range(1, s + 1) for j in range(1, s + 1) if i + j <= s + 1)
    useful = float(N) * N * P * n_tau * 2.0 / 2.0   # N^2 P per moment (SYRK: half of 2 N^2 P)
    nI = (N + 127) // 128
    issued = 2.0 * pairs * n_tau * (nI * (nI + 1) // 2) * 128 * 128 * ((P + 63) // 64 * 64)
    pk, _src = peaks()
    bf16 = pk["bf16_tflops"]
    line = {"metric": "Pi contraction, FP64-accurate forms (ms per call)", "n": N, "pairs": P, "n_tau": n_tau,
            "n_omega": n_om, "n_slices": s, "digit_pairs": pairs, "steps": args.steps, "warmup": args.warmup,
            "ms_fp64_form": ms_64, "ms_emulated": ms_e, "ms_emulated_contractions": st["ms_pi_kernel"],
            "speedup": ms_64 / ms_e, "rel_frobenius_vs_fp64_form": rel, "max_rel_vs_fp64_form": mx,
            "laplace_max_rel_err": lt_err,
            "fp64_form_tflops": useful / (ms_64 / 1e3) / 1e12, "emulated_useful_tflops": useful / (ms_e / 1e3) / 1e12,
            "emulated_issued_bf16_tflops": issued / (st["ms_pi_kernel"] / 1e3) / 1e12,
            "bf16_peak_tflops": bf16, "launches": st["kernel_launches"],
            "note": "useful = N^2 P per Laplace moment (the symmetric product); issued = the BF16 tensor work the "
                    "slice form launches: one product per digit pair, padded lower tiles"}
    print(json.dumps(line), flush=True)
    ctx.close()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.workload == "large":
        run_large(args)
    elif args.workload == "sweep":
        run_sweep(args)
    elif args.workload == "eig":
        run_eig(args)
    elif args.workload == "emu":
        run_emu(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
