"""Parity at the large workload: 320 occupied orbitals (60 frozen), 3500
virtual, 9000 auxiliary functions, NAF threshold 1e-2, 32 frequencies, the 20
states around the gap, the RI tensor streamed in blocks of 20 occupied
orbitals through ltgw_solve_streamed.

The expected values are the oracle's, stored in tests/golden/large_g0w0.json
by tests/golden/make_large_golden.py (host FP64 law, the oracle's blocked
solve).  Here the same law is evaluated in FP64 on the device (QR and loading
GEMM in FP64, the same Philox counters); the two agree to rounding, which is
checked on one sampled block, far below every tolerance below.

Tolerances: the FP64 form against the oracle mode for mode (Laplace form with
the stored grid on both sides, Sec. 2 Eq. LT): quasi-particle energies within
1e-8 Ha, Sigma(i w) within 1e-11 of its largest magnitude, the same number of
natural auxiliary functions; the emulated FP64 form (contractions from 6
integer slices) the same with Sigma within 1e-10.  The mixed forms (library Laplace grid, split
BF16 or FP8 contractions) against the oracle's direct AC-GW form (Eq. Pi, no
Laplace transform): within 1 meV per state.
"""
import json
import os

import numpy as np
import pytest

from paper_2307_04508_gb300 import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HA2MEV = 27211.386245988
QP_TOL = 1e-8
SIG_TOL = 1e-11
MEV_TOL = 1.0
OCC_BLOCK = 20
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "large_g0w0.json")


@pytest.fixture(scope="module")
def gold():
    with open(GOLDEN) as fh:
        return json.load(fh)


@pytest.fixture(scope="module")
def large():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2307_04508_gb300 import ltgw
    from paper_2307_04508_gb300.synthetic.device import DeviceLaw
    cfg = S.LARGE
    law = DeviceLaw(cfg["n_occ"], cfg["n_virt"], cfg["n_aux"], cfg["n_frozen"], cfg["seed"], cfg["n_targets"],
                    gemm="fp64")
    blocks = [law.b_ov_block(i0, min(cfg["n_occ"], i0 + OCC_BLOCK))
              for i0 in range(cfg["n_frozen"], cfg["n_occ"], OCC_BLOCK)]
    B_tgt = law.b_tgt()
    torch.cuda.synchronize()
    d = {"cfg": cfg, "law": law, "blocks": blocks, "B_tgt": B_tgt,
         "src": ltgw.BlockSource(blocks, cfg["n_frozen"], OCC_BLOCK, cfg["n_virt"]),
         "eps": torch.from_numpy(law.eps).cuda(), "targets": torch.from_numpy(law.targets.astype(np.int32)).cuda(),
         "shift": torch.from_numpy(law.shift).cuda(), "ctx": ltgw.Context(0)}
    yield d
    d["ctx"].close()
    del d
    torch.cuda.empty_cache()


def _solve(large, precision, tau=None):
    from paper_2307_04508_gb300 import ltgw
    cfg = large["cfg"]
    p = ltgw.make_params(cfg["n_occ"], cfg["n_virt"], cfg["n_aux"], cfg["n_frozen"], cfg["n_omega"], cfg["n_tau"],
                         0.5, cfg["naf_thresh"], 2, True, precision)
    T = cfg["n_targets"]
    sig, e, st = np.zeros((T, cfg["n_omega"], 2)), np.zeros(T), np.zeros(T, dtype=np.int32)
    tx, tw = (None, None) if tau is None else (np.ascontiguousarray(tau[0]), np.ascontiguousarray(tau[1]))
    large["ctx"].solve_streamed(p, large["eps"], large["src"], OCC_BLOCK, large["B_tgt"], large["targets"],
                                large["shift"], sig, e, st, tau_x=tx, tau_w=tw)
    return sig[..., 0] + 1j * sig[..., 1], e, st, large["ctx"].stats()


def test_device_law_matches_host_law(large, gold):
    """The device's FP64 evaluation of the law equals the host's (which wrote
    the stored values) to rounding, on the first active occupied orbital's
    block and on the energies, targets and shifts."""
    cfg, law = large["cfg"], large["law"]
    assert gold["workload"]["seed"] == cfg["seed"] and gold["workload"]["n_aux"] == cfg["n_aux"]
    assert gold["targets"] == law.targets.tolist()
    assert np.array_equal(law.eps, S.orbital_energies(cfg["seed"], cfg["n_occ"], cfg["n_virt"], cfg["n_frozen"]))
    L = S.aux_loading(cfg["seed"], cfg["n_aux"], cfg["n_occ"], cfg["n_virt"])
    nf, nv = cfg["n_frozen"], cfg["n_virt"]
    host = L @ S.pair_normals_ov(cfg["seed"], cfg["n_aux"], cfg["n_occ"], nv, nf, nf + 1)
    dev = large["blocks"][0][:, :nv].cpu().numpy()
    assert np.abs(dev - host).max() <= 1e-12 * np.abs(host).max()


# LTGW_FP64 and LTGW_FP64_EMU (the contractions from integer slices, Sigma to
# the slices' 2^-42 relative errors)
@pytest.mark.parametrize("precision,sig_tol", [(0, SIG_TOL), (4, 1e-10)])
def test_fp64_form_matches_oracle(large, gold, precision, sig_tol):
    """Laplace form with the stored grid on both sides (reading c-1)."""
    lt = gold["laplace"]
    sig, e, st, stats = _solve(large, precision, tau=(np.array(lt["tau_x"]), np.array(lt["tau_w"])))
    e_o = np.array(lt["e_qp"])
    sig_o = np.array(lt["sigma_re"]) + 1j * np.array(lt["sigma_im"])
    print(f"large precision {precision}: QP {np.abs(e - e_o).max():.2e} Ha, "
          f"Sigma {np.abs(sig - sig_o).max() / np.abs(sig_o).max():.2e}, {stats['ms_total'] / 1e3:.1f} s")
    assert stats["n_naf"] == gold["n_naf"]
    assert np.all(st == 0) and lt["status"] == [0] * len(st)
    assert np.abs(e - e_o).max() <= QP_TOL, np.abs(e - e_o).max()
    assert np.abs(sig - sig_o).max() <= sig_tol * np.abs(sig_o).max()


@pytest.mark.parametrize("precision", [1, 2, 3])   # LTGW_BF16X3, LTGW_FP8, LTGW_FP8_PI
def test_mixed_forms_within_1_mev_of_oracle(large, gold, precision):
    """Library Laplace grid and tensor-core contractions against the oracle's
    direct AC-GW (no Laplace transform)."""
    sig, e, st, stats = _solve(large, precision)
    assert np.all(st == 0)
    err = np.abs(e - np.array(gold["direct"]["e_qp"])) * HA2MEV
    assert err.max() <= MEV_TOL, err
