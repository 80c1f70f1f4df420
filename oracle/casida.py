"""Fully-analytic RI-G0W0 (Casida form of the RPA) for tiny inputs.

TEST INFRASTRUCTURE ONLY: an independent route to the self-energy that the
analytic-continuation oracle is checked against.  The paper uses the
"fully-analytic" G0W0 as its accuracy reference (Sec. 1 and Sec. 4.1.1); this
module is the RI version of that O(N^6) approach, valid for the same
closed-shell reading as the oracle (spin factor s).

With V = R_ov^T R_ov (pairs x pairs) and D = diag(Delta):
  Omega_nu^2, Z = eigenpairs of D^2 + 2 s D^1/2 V D^1/2       (RPA excitations)
  |w^nu_nm|^2 = s (sum_P R^P_nm sum_ia R^P_ia Delta_ia^1/2 Z_ia,nu)^2 / Omega_nu
  Sigma^c_n(E) = sum_m sum_nu |w^nu_nm|^2 / (E - eps_m + sgn_m Omega_nu)
with sgn_m = +1 for occupied and -1 for virtual m.  This spectral form is what
Eq. CorrelationSelfEnergy integrates to when W^c is written through the
Woodbury identity, so AC and Casida agree up to the frequency quadrature and
the Pade continuation.
"""
from __future__ import annotations

import numpy as np


def rpa_excitations(B_act: np.ndarray, delta: np.ndarray, spin: int = 2):
    """Omega (ascending) and Z from D^2 + 2 s D^1/2 V D^1/2."""
    sd = np.sqrt(delta)
    V = B_act.T @ B_act
    Mat = np.diag(delta ** 2) + 2.0 * spin * (sd[:, None] * V * sd[None, :])
    om2, Z = np.linalg.eigh(Mat)
    if om2.min() <= 0:
        raise ValueError("RPA instability: non-positive Omega^2")
    return np.sqrt(om2), Z


def residues(B_act, B_row, delta, Omega, Z, spin: int = 2):
    """|w^nu_nm|^2 for one target row B_row [P][m]; returns [m][nu]."""
    T = B_act @ (np.sqrt(delta)[:, None] * Z)      # [P][nu]
    amp = B_row.T @ T                              # [m][nu]
    return spin * amp ** 2 / Omega[None, :]


def sigma_analytic(E, eps_m, occ_mask, res, Omega):
    """Sigma^c_n(E) for complex or real E; also returns dSigma/dE."""
    sgn = np.where(occ_mask, 1.0, -1.0)
    den = E - eps_m[:, None] + sgn[:, None] * Omega[None, :]
    return np.sum(res / den), -np.sum(res / den ** 2)


def g0w0_analytic(eps, B_ov, B_tgt, targets, shift, n_occ, n_virt, n_frozen=0, spin=2,
                  tol=1e-12, max_iter=200, eps_ref=None):
    """QP energies E_n = eps_n + Re Sigma^c_n(E_n) + shift_n by Newton from eps_n,
    together with a callable giving Sigma^c_n at any complex energy.  With
    eps_ref, Sigma^c is built from eps but the equation reads
    E_n = eps_ref_n + Re Sigma^c_n(E_n) + shift_n (Newton from eps_ref_n)."""
    eps = np.asarray(eps, dtype=np.float64)
    ref = eps if eps_ref is None else np.asarray(eps_ref, dtype=np.float64)
    B_act = B_ov[:, n_frozen * n_virt:]
    occ = eps[n_frozen:n_occ]
    virt = eps[n_occ:n_occ + n_virt]
    delta = (virt[None, :] - occ[:, None]).reshape(-1)
    Omega, Z = rpa_excitations(B_act, delta, spin)
    eps_m = eps[n_frozen:]
    occ_mask = np.arange(n_frozen, len(eps)) < n_occ
    out, status, sig_fns = [], [], []
    for t, n in enumerate(targets):
        res = residues(B_act, B_tgt[t][:, n_frozen:], delta, Omega, Z, spin)
        E = ref[n]
        st = 1
        for _ in range(max_iter):
            s, ds = sigma_analytic(E, eps_m, occ_mask, res, Omega)
            dE = -(E - ref[n] - s.real - shift[t]) / (1.0 - ds.real)
            E += dE
            if abs(dE) < tol:
                st = 0
                break
        out.append(E)
        status.append(st)
        sig_fns.append(lambda z, res=res: sigma_analytic(z, eps_m, occ_mask, res, Omega)[0])
    return np.array(out), np.array(status), sig_fns, Omega
