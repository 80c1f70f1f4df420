"""The C-ABI library builds, loads, and exports every entry point that
include/*.h declares; host-only entry points work without a GPU."""
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(ltgw_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2307_04508_gb300 import build, ltgw
    build.build()
    return ltgw.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"


def test_binding_covers_declared_symbols():
    from paper_2307_04508_gb300 import ltgw
    assert set(_declared()) <= set(ltgw.SIGNATURES)


def test_gl_grid_matches_library_legendre(lib):
    from paper_2307_04508_gb300 import ltgw
    for n in (1, 2, 7, 24, 32, 128):
        om, wt = ltgw.gl_grid(n, 0.5)
        x, w = np.polynomial.legendre.leggauss(n)
        assert np.allclose(om, 0.5 * (1 + x) / (1 - x), rtol=1e-13, atol=0)
        assert np.allclose(wt, w / (1 - x) ** 2, rtol=1e-10, atol=0)


def test_bad_grid_arguments(lib):
    from paper_2307_04508_gb300 import ltgw
    with pytest.raises(ltgw.LtgwError):
        ltgw.gl_grid(0)
    with pytest.raises(ltgw.LtgwError):
        ltgw.laplace_grid(4, 1.0, 0.5)


def test_create_without_device_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    from paper_2307_04508_gb300 import ltgw
    with pytest.raises(ltgw.LtgwError) as e:
        ltgw.Context(0)
    assert e.value.status == ltgw.LTGW_ERR_DEVICE


def test_request_footprint_host_estimate(lib):
    """ltgw_request_footprint is host arithmetic: it covers the staged inputs,
    grows with every size, and counts the extra operands of the tensor-core
    forms (FP8 codes on top of the split-BF16 copies) and the emulated form's
    slices on top of the FP64 form's arrays."""
    from paper_2307_04508_gb300 import ltgw

    def fp(n_occ=40, n_virt=400, n_aux=1320, prec=ltgw.LTGW_FP64, n_tgt=4, naf=1e-2):
        p = ltgw.make_params(n_occ, n_virt, n_aux, n_occ // 6, 32, 8, 0.5, naf, 2, True, prec)
        return ltgw.request_footprint(p, n_tgt)

    base = fp()
    assert base >= 1320 * 40 * 400 * 8
    assert fp(n_occ=60) > base and fp(n_virt=500) > base and fp(n_aux=1500) > base and fp(n_tgt=8) > base
    assert fp(naf=-1.0) > base   # without NAF every auxiliary function stays
    assert fp(prec=ltgw.LTGW_FP8) > fp(prec=ltgw.LTGW_BF16X3)
    assert fp(prec=ltgw.LTGW_FP64_EMU) > base
    p = ltgw.make_params(40, 400, 1320, 6, 32, 8, 0.5, 1e-2, 2, True, 0)
    assert ltgw.request_footprint(p, 0) == 0
