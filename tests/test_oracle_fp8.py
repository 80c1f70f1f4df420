"""Pins of the oracle's FP8 E4M3 form of the Pi contraction.

The E4M3 rounding is checked against the format's own definition (every one of
the 256 codes decoded from its bit fields) and against PyTorch's float8_e4m3fn
conversion; the per-row scaling and the de-scaling chain against a case where
quantisation is exact, so that the FP8 Pi must equal the exact Pi; the
two-term expansion (h + l per value, three products) against its own exact
cases and its error bound."""
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


def test_pi_scale_table_imaginary_time_branch():
    """The imaginary-time factors are e^{-Delta tau_k}, rounded once to FP32:
    checked on gaps whose products with tau are exact multiples of ln 2 (the
    factors are then powers of two) and on Delta tau = 1 and 2 against the
    decimal expansions of e^-1 and e^-2; a wrong sign would give factors above 1."""
    ln2 = 0.6931471805599453
    delta = np.array([ln2, 2.0 * ln2, 1.0, 0.0])
    S = O.pi_scale_table(delta, tau=np.array([0.0, 1.0, 2.0]))
    assert S.dtype == np.float32 and S.shape == (3, 4)
    assert np.array_equal(S[0], np.ones(4, dtype=np.float32))
    assert np.allclose(S[1, :2], [0.5, 0.25], rtol=2e-16 * 4, atol=0)
    assert np.allclose(S[2, :2], [0.25, 0.0625], rtol=2e-16 * 8, atol=0)
    assert S[1, 2] == np.float32(0.36787944117144233) and S[2, 2] == np.float32(0.1353352832366127)
    assert S[1, 3] == 1.0 and S[2, 3] == 1.0
    assert np.all(S <= 1.0)


def test_two_term_split_residual_and_bound():
    """h = e4m3(xs), l = e4m3(xs - h): the residual is formed exactly (it is
    a difference of two FP32 numbers within a factor two) and h + l carries
    the 3 + 3 mantissa bits: |xs - h - l| <= 2^-4 |xs - h| + 2^-10 (half the
    subnormal spacing)."""
    rng = np.random.default_rng(11)
    X = (rng.standard_normal((6, 4000)) * np.exp(rng.uniform(-6, 6, (6, 1)))).astype(np.float32)
    h, l, inv = O.fp8_row_split(X)
    xs = (X * inv[:, None]).astype(np.float32).astype(np.float64)
    assert np.array_equal(O.e4m3_round(h), h) and np.array_equal(O.e4m3_round(l), l)
    assert np.array_equal((xs - h).astype(np.float32).astype(np.float64), xs - h)
    assert np.all(np.abs(xs - h - l) <= 2.0 ** -4 * np.abs(xs - h) + 2.0 ** -10)
    assert np.abs(xs - h - l).max() < 2.0 ** -7 * 448.0


def test_two_term_product_exact_cases():
    """Values that are exact two-term E4M3 expansions in their row's scaled
    units (row maxima 448, power-of-two scales): with l = 0 in one operand the
    product is exact; in general it misses exactly l_a l_b."""
    tab = np.array(sorted(_e4m3_table().values()))
    pos = tab[(tab >= 2.0 ** -3) & (tab < 448.0)]   # so that the l grid (2^-6 of h's binade) stays above 2^-9
    rng = np.random.default_rng(12)
    N, P = 5, 300

    def make(lo_nonzero):
        h = rng.choice(pos, size=(N, P)) * rng.choice([-1.0, 1.0], size=(N, P))
        sp = 2.0 ** (np.floor(np.log2(np.abs(h))) - 3)          # h's spacing
        # l away from zero (a negative l at a power of two would cross into the binade below)
        l = (rng.integers(0, 4, (N, P)) * np.sign(h) * sp / 8.0) if lo_nonzero else np.zeros((N, P))
        h[:, 0], l[:, 0] = 448.0, 0.0                            # the row maxima
        return h, l, (2.0 ** rng.integers(-12, -2, N))[:, None]
    ha, la, sa = make(True)
    hb, lb, sb = make(False)
    A, B = (ha + la) * sa, (hb + lb) * sb
    assert np.allclose(O.fp8_split_product(A, B), A @ B.T, rtol=1e-14, atol=0)
    hb2, lb2, sb2 = make(True)
    B2 = (hb2 + lb2) * sb2
    miss = (la * sa) @ (lb2 * sb2).T
    assert np.allclose(O.fp8_split_product(A, B2), A @ B2.T - miss, rtol=1e-13, atol=1e-13 * np.abs(A @ B2.T).max())


@pytest.mark.parametrize("form", ["direct", "laplace", "tau"])
def test_fp8_pi_error_in_the_fp8_range(form):
    rng = np.random.default_rng(8)
    N, P = 40, 3000
    B = rng.standard_normal((N, P)) * 0.05
    delta = rng.uniform(0.3, 4.0, P)
    om, _ = O.gl_grid(6, 0.5)
    if form == "laplace":
        x, w = O.sinc_laplace_grid(7, -6.0, 2.0)
        ref = O.polarizability_lt(O.laplace_moments(B, delta, x, w), om, x, 2)
        got = O.polarizability_fp8(B, delta, om, 2, x=x, w=w)
    elif form == "tau":
        # gamma = I: each "frequency" is one moment M^k itself, so the error is
        # the moments' own (a fitted gamma's cancellation would magnify it)
        tau, gamma = np.geomspace(0.1 / 4.0, 8.0 / 0.3, len(om)), np.eye(len(om))
        ref = O.polarizability_tau(O.tau_moments(B, delta, tau), gamma, 2)
        got = O.polarizability_fp8(B, delta, om, 2, tau=tau, gamma=gamma)
    else:
        ref = O.polarizability_direct(B, delta, om, 2)
        got = O.polarizability_fp8(B, delta, om, 2)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    # the two-term expansion keeps about 7 significant bits per value
    assert 1e-6 < err < 2e-3, err
    assert np.array_equal(got, np.swapaxes(got, 1, 2))
