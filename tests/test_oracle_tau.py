"""Pins of the imaginary-time (cosine-transform) form of Pi and of the
library's grid fit for it (host code, no GPU).

The oracle's form is checked against the direct Pi (Eq. Pi) where the
exponential sum is exact (every pair at one gap, coefficients solved for it)
and where it is converged (its own least-squares grid with many nodes); the
library's host grid fit against its reported error on an independent sample."""
import numpy as np
import pytest

from oracle import ltgw_oracle as O


def test_tau_form_exact_for_one_gap():
    """All pairs at one gap d: gamma_jk chosen so that sum_k gamma_jk e^{-d tau_k}
    equals d / (w_j^2 + d^2) makes the form exact (4 frequencies, 3 nodes, so a
    transposed gamma or a wrong sign in the exponent fails)."""
    rng = np.random.default_rng(21)
    N, P, d = 6, 40, 0.7
    B = rng.standard_normal((N, P))
    delta = np.full(P, d)
    om = np.array([0.1, 0.5, 2.0, 9.0])
    tau = np.array([0.3, 1.1, 4.0])
    gamma = np.zeros((4, 3))
    for j, w in enumerate(om):
        c = rng.uniform(0.2, 1.0, 3)
        gamma[j] = c * (d / (w * w + d * d)) / (c @ np.exp(-d * tau))
    got = O.polarizability_tau(O.tau_moments(B, delta, tau), gamma, 2)
    ref = O.polarizability_direct(B, delta, om, 2)
    assert np.allclose(got, ref, rtol=1e-13, atol=0)


def test_tau_form_converges_to_direct_pi():
    rng = np.random.default_rng(22)
    N, P = 12, 500
    B = rng.standard_normal((N, P)) * 0.1
    delta = rng.uniform(0.3, 4.0, P)
    om, _ = O.gl_grid(16, 0.5)
    ref = O.polarizability_direct(B, delta, om, 2)
    errs = []
    for n in (6, 10, 16):
        tau, gamma, _ = O.cosine_grid(n, 0.3, 4.0, om)
        got = O.polarizability_tau(O.tau_moments(B, delta, tau), gamma, 2)
        errs.append(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-5


def test_library_cosine_grid_error_curve():
    """The library's host fit: its reported scaled error holds on an independent
    sample and falls with the node count; coefficients stay moderate."""
    from paper_2307_04508_gb300 import ltgw
    try:
        ltgw.load()
    except OSError as e:
        pytest.skip(f"library not built: {e}")
    om, _ = O.gl_grid(32, 0.5)
    dmin, dmax = 0.27, 4.0
    D = np.geomspace(dmin, dmax, 7919)
    prev = np.inf
    for n in (6, 8, 10, 12, 16):
        tau, gamma, err, amp = ltgw.cosine_grid(n, dmin, dmax, om)
        worst = 0.0
        for j, w in enumerate(om):
            f = D / (w * w + D * D)
            dpk = min(max(w, dmin), dmax)
            fmax = dpk / (w * w + dpk * dpk)
            worst = max(worst, np.abs(np.exp(-D[:, None] * tau[None, :]) @ gamma[j] - f).max() / fmax)
        assert worst <= 1.05 * err + 1e-12
        assert err < prev
        assert np.abs(gamma).max() < 1e4
        D2 = np.geomspace(dmin, dmax, 997)
        assert amp >= max(np.abs(np.exp(-D2[:, None] * tau[None, :]) * gamma[j][None, :]).sum(1).max()
                          / (min(max(w, dmin), dmax) / (w * w + min(max(w, dmin), dmax) ** 2))
                          for j, w in enumerate(om)) * 0.99
        prev = err
    assert prev < 3e-5
