"""Write the oracle's results for the large synthetic workload to large_g0w0.json.

The large workload: 320 occupied orbitals (60 frozen), 3500 virtual, 9000
auxiliary functions, NAF threshold 1e-2, 32 Gauss-Legendre frequencies, the
20 states around the gap, inputs from the seeded law of
``paper_2307_04508_gb300.synthetic`` (seed 20230712) in FP64 on the host.
The RI tensor (65.5 GB in FP64) is never held whole: the oracle's blocked
solve asks for it one block of occupied orbitals at a time, twice (the NAF
metric, then the projection).

Two solves share the NAF basis: the conventional direct form (Eq. Pi) and the
Laplace form (Eq. LT and the M^m factorisation) on a fixed 10-point grid that
is stored with the results, so that a solve on another machine can be fed the
same grid.  Stored: quasi-particle energies and Newton status per state,
Sigma^c_n(i w_l) at every GL node, the number of kept auxiliary functions and
the kept/dropped eigenvalues nearest to the threshold.

Only the oracle and the input generator are called.  About 40 minutes on
eight x86 cores (four passes of 1.5e14 flops: loading GEMM twice, NAF metric,
direct Pi) and 45 GB of memory.

    python tests/golden/make_large_golden.py [--small]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import ltgw_oracle as O  # noqa: E402
from paper_2307_04508_gb300 import synthetic as S  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
# the fixed Laplace grid of the stored Laplace-form solve (any rule of this
# form is a valid grid for a mode-for-mode comparison)
LT_GRID = dict(n_tau=10, t_lo=-9.0, t_hi=2.5)


def log(msg):
    print(f"[{time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--small", action="store_true", help="a reduced workload, to check the script quickly")
    ap.add_argument("--occ-block", type=int, default=10)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    cfg = dict(S.LARGE)
    if args.small:
        cfg.update(n_occ=40, n_frozen=8, n_virt=300, n_aux=900, n_targets=6)
    out = args.out or os.path.join(HERE, "large_g0w0_small.json" if args.small else "large_g0w0.json")
    no, nv, na, nf, seed = cfg["n_occ"], cfg["n_virt"], cfg["n_aux"], cfg["n_frozen"], cfg["seed"]
    t_start = time.time()
    timing = {}

    t0 = time.time()
    eps = S.orbital_energies(seed, no, nv, nf)
    targets = S.gap_targets(no, cfg["n_targets"])
    shift = S.uniform(seed, S.STREAM_SHIFT, len(targets), -0.05, 0.05)
    L = S.aux_loading(seed, na, no, nv)
    B_tgt = np.empty((len(targets), na, no + nv))
    for t, p in enumerate(targets):
        B_tgt[t] = L @ S.pair_normals_row(seed, na, no + nv, int(p))
    timing["inputs_s"] = time.time() - t0
    log(f"inputs: {timing['inputs_s']:.1f} s")

    def ov_block(i0, i1):
        return L @ S.pair_normals_ov(seed, na, no, nv, i0, i1)

    blocks = O.occ_blocks(no, nf, args.occ_block)
    t0 = time.time()
    K = O.naf_metric_blocked(ov_block, blocks)
    timing["naf_metric_s"] = time.time() - t0
    log(f"K: {timing['naf_metric_s']:.1f} s")
    t0 = time.time()
    U, lam_kept, lam_all = O.naf_basis(K, cfg["naf_thresh"])
    del K
    timing["naf_eig_s"] = time.time() - t0
    thr = cfg["naf_thresh"]
    log(f"eig: {timing['naf_eig_s']:.1f} s, N_NAF {U.shape[1]}")
    t0 = time.time()
    Bt = O.naf_project_blocked(ov_block, blocks, U, nv)
    Bt_tgt = np.stack([O.naf_project(B_tgt[t][:, nf:], U) for t in range(len(targets))])
    del B_tgt
    timing["naf_project_s"] = time.time() - t0
    log(f"projection: {timing['naf_project_s']:.1f} s")

    res = {}
    x, w = O.sinc_laplace_grid(LT_GRID["n_tau"], LT_GRID["t_lo"], LT_GRID["t_hi"])
    for mode, tx, tw in (("laplace", x, w), ("direct", None, None)):
        t0 = time.time()
        sig, e, st = O.solve_projected(eps, Bt, Bt_tgt, targets, shift, no, nv, nf, cfg["n_omega"], 0.5, 2,
                                       tau_x=tx, tau_w=tw)
        timing[f"{mode}_s"] = time.time() - t0
        log(f"{mode}: {timing[f'{mode}_s']:.1f} s, E_QP {e}")
        res[mode] = {"e_qp": e.tolist(), "status": st.tolist(), "sigma_re": sig.real.tolist(),
                     "sigma_im": sig.imag.tolist()}
    res["laplace"]["tau_x"] = x.tolist()
    res["laplace"]["tau_w"] = w.tolist()
    omegas, _ = O.gl_grid(cfg["n_omega"], 0.5)
    dropped = lam_all[lam_all <= thr]
    doc = {
        "what": "oracle (oracle/ltgw_oracle.py, solve_blocked's steps) on the large synthetic workload",
        "written_by": "tests/golden/make_large_golden.py" + (" --small" if args.small else ""),
        "workload": {k: cfg[k] for k in ("n_occ", "n_virt", "n_aux", "n_frozen", "seed", "n_targets", "n_omega",
                                         "n_tau", "naf_thresh")},
        "law": "paper_2307_04508_gb300.synthetic host generator, FP64 QR and loading GEMM",
        "spin": 2, "omega0": 0.5, "targets": targets.tolist(), "omegas": omegas.tolist(),
        "n_naf": int(U.shape[1]), "lambda_max": float(lam_all[-1]),
        "lambda_kept_min": float(lam_kept.min()),
        "lambda_dropped_max": float(dropped.max()) if len(dropped) else None,
        "laplace_grid": dict(LT_GRID, rule="oracle.ltgw_oracle.sinc_laplace_grid"),
        "occ_block": args.occ_block,
        "numpy": np.__version__, "timing_s": timing, "total_s": time.time() - t_start,
        "direct": res["direct"], "laplace": res["laplace"],
    }
    with open(out, "w") as fh:
        json.dump(doc, fh, indent=1)
    log(f"wrote {out} in {time.time() - t_start:.0f} s")


if __name__ == "__main__":
    main()
