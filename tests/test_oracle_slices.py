"""Pins for the oracle's FP64-accurate product from integer slices
(slice_rows, slice_product): the digits rebuild the rounded fixed-point rows
exactly and stay in their ranges; products of operands whose digits all fall
within the kept pairs equal the exact product bit for bit; otherwise the error
stays within the bound of the dropped digits and the rounding, against an
exact rational product, and falls by about 2^7 per extra slice."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import ltgw_oracle as O


def _exact_product(A, B):
    """A B^T in rationals (every float64 is a dyadic rational)."""
    Af = [[Fraction(float(v)) for v in row] for row in A]
    Bf = [[Fraction(float(v)) for v in row] for row in B]
    return [[sum((a * b for a, b in zip(ra, rb)), Fraction(0)) for rb in Bf] for ra in Af]


@pytest.mark.parametrize("s", [2, 4, 6, 8])
def test_digits_rebuild_the_rounded_rows(s):
    rng = np.random.default_rng(s)
    X = rng.standard_normal((9, 37)) * np.exp2(rng.integers(-30, 30, 9))[:, None]
    X[3] = 0.0                                      # a zero row: e = 0, zero digits
    X[5, :] = -X[5, :].max()                        # a row whose maximum is its negative extreme
    d, e = O.slice_rows(X, s)
    assert d.shape == (s,) + X.shape
    assert np.all(d == np.rint(d))
    assert np.abs(d[0]).max() <= 128 and (s == 1 or np.abs(d[1:]).max() <= 64)
    for r in range(X.shape[0]):
        m = np.abs(X[r]).max()
        if m == 0:
            assert e[r] == 0 and not d[:, r].any()
            continue
        assert 2.0 ** (e[r] - 1) <= m < 2.0 ** e[r]
        for k in range(X.shape[1]):
            q = sum(int(d[i, r, k]) * 128 ** (s - 1 - i) for i in range(s))
            # X_rk 2^(7 s - e) rounded to the nearest integer (ties to even)
            t = Fraction(float(X[r, k])) * Fraction(2) ** (7 * s - int(e[r]))
            fl = t.numerator // t.denominator
            rem = t - fl
            want = fl + (1 if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2) else 0)
            assert q == want


def test_product_exact_when_no_digit_pair_is_dropped():
    """Integer operands of at most 21 significant bits have at most 3 nonzero
    digits per row (the trailing s-3 digits vanish), so with s = 6 every pair
    (i + j <= 6 <= 7) is kept and the product is exact; small k keeps the
    exact sums below 2^53, where float64 holds them exactly."""
    rng = np.random.default_rng(11)
    A = rng.integers(-(2 ** 20), 2 ** 20, (7, 16)).astype(np.float64)
    B = rng.integers(-(2 ** 20), 2 ** 20, (5, 16)).astype(np.float64)
    A[:, 0] = 2.0 ** 20                              # every row's maximum just below 2^21
    B[:, 0] = -(2.0 ** 20)
    exact = np.array(_exact_product(A, B), dtype=object)
    got = O.slice_product(A, B, 6)
    assert got.shape == (7, 5)
    assert all(Fraction(float(got[i, j])) == exact[i, j] for i in range(7) for j in range(5))
    # A with 28 significant bits (4 digits) needs the pair (4, 3) at level 7:
    # still kept with s = 6 against 21-bit B
    A4 = rng.integers(-(2 ** 27), 2 ** 27, (4, 8)).astype(np.float64)
    A4[:, 1] = 2.0 ** 27
    B3 = rng.integers(-(2 ** 20), 2 ** 20, (3, 8)).astype(np.float64)
    B3[:, 2] = 2.0 ** 20
    got = O.slice_product(A4, B3, 6)
    exact = _exact_product(A4, B3)
    assert all(Fraction(float(got[i, j])) == exact[i][j] for i in range(4) for j in range(3))


def test_product_of_scaled_rows_is_scaled():
    """Rows scaled by powers of two give the product scaled by the same powers
    (the row exponents carry the scale; the digits do not change)."""
    rng = np.random.default_rng(5)
    A, B = rng.standard_normal((6, 50)), rng.standard_normal((4, 50))
    pa, pb = rng.integers(-40, 40, 6), rng.integers(-40, 40, 4)
    base = O.slice_product(A, B, 5)
    got = O.slice_product(np.ldexp(A, pa[:, None]), np.ldexp(B, pb[:, None]), 5)
    assert np.array_equal(got, np.ldexp(np.ldexp(base, pa[:, None]), pb[None, :]))


@pytest.mark.parametrize("s", [3, 4, 5, 6])
def test_error_within_the_dropped_digit_bound(s):
    """|D - A B^T| per entry is at most k 2^(e_A + e_B) times the rounding of
    both rows (2^(-7 s) for q_a r_b + r_a q_b + r_a r_b) plus the dropped pairs
    (both digits beyond the leading one: at most 64 * 64 2^(-7 L) each, 2 s + 1 - L
    pairs at level L > s + 1), plus the float64 level sums; the exact product
    in rationals.  The bound is also not loose by more than about 2^10."""
    rng = np.random.default_rng(100 + s)
    k = 24
    A, B = rng.standard_normal((5, k)), rng.standard_normal((4, k))
    got = O.slice_product(A, B, s)
    exact = _exact_product(A, B)
    _, ea = O.slice_rows(A, s)
    _, eb = O.slice_rows(B, s)
    dropped = sum((2 * s + 1 - L) * 4096.0 * 2.0 ** (-7 * L) for L in range(s + 2, 2 * s + 1))
    unit = 2.0 ** (-7 * s) * (1 + 2.0 ** (-7 * s)) + dropped
    worst = 0.0
    for i in range(5):
        for j in range(4):
            err = abs(Fraction(float(got[i, j])) - exact[i][j])
            scale = 2.0 ** (int(ea[i]) + int(eb[j]))
            bound = k * scale * unit + 8 * np.finfo(float).eps * k * scale
            assert err <= Fraction(bound), (i, j, float(err), bound)
            worst = max(worst, float(err) / (k * scale * unit))
    assert worst > 2.0 ** -12


def test_error_falls_by_about_2_to_the_7_per_slice():
    rng = np.random.default_rng(3)
    A, B = rng.standard_normal((40, 300)), rng.standard_normal((30, 300))
    exact = np.matmul(A.astype(np.longdouble), B.astype(np.longdouble).T)
    errs = [float(np.linalg.norm((O.slice_product(A, B, s) - exact).astype(np.float64)) /
                  np.linalg.norm(exact.astype(np.float64))) for s in (3, 4, 5)]
    for a, b in zip(errs, errs[1:]):
        assert 2.0 ** 4 < a / b < 2.0 ** 10, errs
    assert errs[-1] < 1e-9


def test_symmetric_product_is_symmetric():
    """With B = A the kept digit pairs are symmetric in (i, j), so the
    product is exactly symmetric."""
    rng = np.random.default_rng(8)
    A = rng.standard_normal((12, 70))
    D = O.slice_product(A, A, 6)
    assert np.array_equal(D, D.T)


@pytest.mark.parametrize("laplace", [False, True])
def test_emulated_polarizability_against_fp64_forms(laplace):
    """Pi from slices equals the plain FP64 Pi (Eq. Pi, or the M^m form of
    Eq. LT) to the slices' error, symmetric, and tightens with more slices."""
    rng = np.random.default_rng(21)
    N, P = 30, 900
    Bt = rng.standard_normal((N, P)) * 0.05 * np.exp(-np.arange(N) / 10.0)[:, None]
    delta = rng.uniform(0.3, 4.0, P)
    om, _ = O.gl_grid(6, 0.5)
    if laplace:
        x, w = O.sinc_laplace_grid(7, -6.0, 2.0)
        ref = O.polarizability_lt(O.laplace_moments(Bt, delta, x, w), om, x, 2)
    else:
        x = w = None
        ref = O.polarizability_direct(Bt, delta, om, 2)
    errs = []
    for s in (4, 6, 8):
        got = O.polarizability_emulated(Bt, delta, om, 2, x=x, w=w, n_slices=s)
        assert np.array_equal(got, np.swapaxes(got, 1, 2))
        errs.append(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    assert errs[0] < 1e-6 and errs[1] < 1e-11 and errs[2] < 1e-14, errs
    assert errs[0] > 1e3 * errs[1], errs
