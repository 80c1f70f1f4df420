"""Pins of the oracle's FP8 E4M3 form of the Pi contraction.

The E4M3 rounding is checked against the format's own definition (every one of
the 256 codes decoded from its bit fields) and against PyTorch's float8_e4m3fn
conversion; the per-row scaling and the de-scaling chain against a case where
quantisation is exact, so that the FP8 Pi must equal the exact Pi."""
import numpy as np
import pytest

from oracle import ltgw_oracle as O


def _e4m3_table():
    """All finite E4M3 values from the bit fields: sign, 4-bit exponent (bias 7),
    3-bit mantissa; exponent 0 is subnormal (M 2^-9); S.1111.111 is NaN."""
    vals = {}
    for code in range(256):
        sgn, ex, man = code >> 7, (code >> 3) & 15, code & 7
        if ex == 15 and man == 7:
            continue
        v = man * 2.0 ** -9 if ex == 0 else (1 + man / 8) * 2.0 ** (ex - 7)
        vals[code] = -v if sgn else v
    return vals


def test_e4m3_grid_fixed_points_ties_and_saturation():
    tab = _e4m3_table()
    assert len(tab) == 254 and max(tab.values()) == 448.0 and min(v for v in tab.values() if v > 0) == 2.0 ** -9
    pos = sorted({(v, c) for c, v in tab.items() if v >= 0})
    vals = np.array([v for v, _ in pos])
    assert np.array_equal(O.e4m3_round(vals), vals)
    assert np.array_equal(O.e4m3_round(-vals), -vals)
    # midpoints go to the even code (mantissa bit 0 clear), nudged points to the nearer value
    for (a, ca), (b, cb) in zip(pos[:-1], pos[1:]):
        mid = 0.5 * (a + b)
        even = a if ca % 2 == 0 else b
        assert O.e4m3_round(mid) == even, (a, b)
        assert O.e4m3_round(mid - 1e-6 * (b - a)) == a
        assert O.e4m3_round(mid + 1e-6 * (b - a)) == b
    for big in (448.0 + 1e-3, 464.0, 479.0, 1e6):
        assert O.e4m3_round(big) == 448.0 and O.e4m3_round(-big) == -448.0


def test_e4m3_matches_torch_float8():
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("this PyTorch has no float8_e4m3fn")
    rng = np.random.default_rng(5)
    v = (rng.standard_normal(200000) * np.exp(rng.uniform(-9, 6, 200000))).astype(np.float32)
    v = v[np.abs(v) < 440.0]
    ref = torch.from_numpy(v).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(O.e4m3_round(v.astype(np.float64)), ref)


def test_row_quantize_scales_each_row_to_448():
    rng = np.random.default_rng(6)
    X = rng.standard_normal((7, 300)).astype(np.float32) * np.exp(rng.uniform(-8, 8, 7))[:, None].astype(np.float32)
    X[3] = 0.0
    q, inv = O.fp8_row_quantize(X)
    assert inv[3] == 0.0 and not np.any(q[3])
    live = [r for r in range(7) if r != 3]
    assert np.allclose(np.abs(q[live]).max(axis=1), 448.0)
    rel = np.abs(q[live] / inv[live, None] - X[live]) / np.abs(X[live]).max(axis=1)[:, None]
    assert rel.max() <= 2.0 ** -4 * 448.0 / 448.0   # half a spacing of the top binade, relative to the row max


def test_fp8_pi_exact_when_operands_are_representable():
    """E4M3 values with power-of-two row maxima and unit pair factors (all
    Delta = 1, w = 0): every rounding is exact and the FP8 Pi is the exact Pi."""
    tab = np.array(sorted(_e4m3_table().values()))
    rng = np.random.default_rng(7)
    N, P = 9, 400
    B = rng.choice(tab[np.abs(tab) <= 448.0], size=(N, P))
    B[:, 0] = 448.0
    B *= (2.0 ** rng.integers(-12, -2, N))[:, None]
    delta = np.ones(P)
    got = O.polarizability_fp8(B, delta, np.array([0.0]), spin=2)
    ref = O.polarizability_direct(B, delta, np.array([0.0]), spin=2)
    assert np.allclose(got, ref, rtol=1e-13, atol=0)


@pytest.mark.parametrize("laplace", [False, True])
def test_fp8_pi_error_in_the_fp8_range(laplace):
    rng = np.random.default_rng(8)
    N, P = 40, 3000
    B = rng.standard_normal((N, P)) * 0.05
    delta = rng.uniform(0.3, 4.0, P)
    om, _ = O.gl_grid(6, 0.5)
    if laplace:
        x, w = O.sinc_laplace_grid(7, -6.0, 2.0)
        ref = O.polarizability_lt(O.laplace_moments(B, delta, x, w), om, x, 2)
        got = O.polarizability_fp8(B, delta, om, 2, x=x, w=w)
    else:
        ref = O.polarizability_direct(B, delta, om, 2)
        got = O.polarizability_fp8(B, delta, om, 2)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert 1e-4 < err < 2e-2
    assert np.array_equal(got, np.swapaxes(got, 1, 2))
