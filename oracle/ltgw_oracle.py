"""CPU FP64 oracle for the LT-GW G0W0 hot path (Toelle, Niemeyer, Neugebauer,
"Accelerating Analytic-Continuation GW Calculations with a Laplace
Transformation and Natural Auxiliary Functions", arXiv:2307.04508).

TEST INFRASTRUCTURE ONLY.  This module is the slow, plain reference that the
CUDA path is checked against.  Only the tests, the smoke check and the CPU
baseline leg of the benchmark may import it; the product never does.  It
shares no code with the CUDA path.

Everything is float64 and follows the paper's statement of the problem in the
paper's order:

  frozen-core slice (Sec. 3)  ->  NAF metric K (Eq. nafeq, ov block only)
  ->  eigenvectors of K above the threshold (NAF eigen-equation)
  ->  R~ = R U (Eq. naftrafo)
  ->  Pi(i w) directly (Eq. Pi) or through the Laplace moments M^m (Eq. LT and
      the M^m factorisation that follows it)
  ->  W^c_nm(i w) = sum_PQ R^P_nm {[1 - Pi]^-1 - 1}_PQ R^Q_nm
      (Eq. ScreenedCoulombOrbital)
  ->  Sigma^c_n(i w) by the modified Gauss-Legendre quadrature of
      Eq. CorrelationSelfEnergy
  ->  N-point Pade continued fraction (Vidberg & Serene, J. Low Temp. Phys. 29,
      179 (1977), appendix)  ->  quasi-particle equation solved by Newton.

Readings of points the paper leaves open (each one fixed once):
  * spin: closed-shell spatial orbitals, Pi = -2 s sum_ia ..., s = 2 by
    default (s = 1 is the literal spin-orbital form of Eq. Pi);
  * the NAF metric sums occupied-virtual pairs of active occupied orbitals
    only, without the closed-shell factor 2, and keeps eigenvalues strictly
    greater than the threshold; a negative threshold switches NAF off;
  * frozen-core orbitals leave Pi, K and the m-sum of Sigma, and cannot be
    targets;
  * eps_F = (eps_HOMO + eps_LUMO) / 2;
  * Sigma is evaluated on all N_omega Gauss-Legendre nodes; the Pade fraction
    passes through every second node (indices 0, 2, 4, ...; ceil(N_omega/2)
    points) in ascending order.  The paper, too, continues from a smaller
    frequency set (70 points) than it integrates on (128); through all nodes
    the fraction amplifies 1e-15 relative noise in Sigma to ~1e-8 Ha in the
    quasi-particle energy, through every second node to ~1e-13 Ha;
  * eta = 0 (the real quasi-particle equation);
  * Newton from eps_n, stop when |dE| < 1e-12 Ha, at most 100 steps.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "gl_grid", "fermi_level", "active_ov", "naf_metric", "naf_basis", "naf_project",
    "pair_gaps", "polarizability_direct", "laplace_moments", "polarizability_lt",
    "screened_interaction", "w_nm", "sigma_iw", "pade_coefficients", "pade_eval",
    "qp_newton", "solve", "solve_projected", "occ_blocks", "naf_metric_blocked", "naf_project_blocked",
    "solve_blocked", "sinc_laplace_grid", "pade_nodes",
    "E4M3_MAX", "e4m3_round", "fp8_row_quantize", "fp8_row_split", "fp8_split_product", "pi_scale_table",
    "polarizability_fp8", "SLICE_BITS", "slice_rows", "slice_product",
    "pi_factor_table", "polarizability_emulated",
    "cosine_grid", "tau_moments", "polarizability_tau", "evgw_energies", "evgw",
]


# ----------------------------------------------------------------------------
# Grids
# ----------------------------------------------------------------------------
def gl_grid(n_omega: int, omega0: float = 0.5):
    """Modified Gauss-Legendre rule on [0, inf) (Sec. 2, after Eq.
    CorrelationSelfEnergy): Legendre nodes x in (-1, 1) mapped by
    omega = omega0 (1 + x) / (1 - x), weight w * 2 omega0 / (1 - x)^2.
    Nodes are returned in ascending omega."""
    x, w = np.polynomial.legendre.leggauss(n_omega)
    omega = omega0 * (1.0 + x) / (1.0 - x)
    weight = w * 2.0 * omega0 / (1.0 - x) ** 2
    order = np.argsort(omega)
    return omega[order], weight[order]


def sinc_laplace_grid(n_tau: int, t_lo: float, t_hi: float):
    """A Laplace quadrature for 1/X = int_0^inf exp(-X tau) d tau (Eq. LT):
    substitute tau = e^t and apply the trapezoid rule with n_tau equidistant
    nodes on [t_lo, t_hi].  Returns (x_m, w_m) with 1/X ~ sum w_m exp(-X x_m).
    Not minimax; any rule of this form is a valid Laplace grid for the
    LT-mode checks, which feed the same grid to both sides."""
    t = np.linspace(t_lo, t_hi, n_tau)
    h = t[1] - t[0] if n_tau > 1 else 1.0
    x = np.exp(t)
    w = h * np.exp(t)
    return x, w


# ----------------------------------------------------------------------------
# Frozen core and pair data
# ----------------------------------------------------------------------------
def fermi_level(eps: np.ndarray, n_occ: int) -> float:
    """eps_F, read as the midpoint of the HOMO-LUMO gap."""
    return 0.5 * (eps[n_occ - 1] + eps[n_occ])


def active_ov(B_ov: np.ndarray, n_occ: int, n_virt: int, n_frozen: int) -> np.ndarray:
    """Frozen-core slice (Sec. 3): drop the pairs i*n_virt+a with i < n_frozen."""
    assert B_ov.shape[1] == n_occ * n_virt
    return B_ov[:, n_frozen * n_virt:]


def pair_gaps(eps: np.ndarray, n_occ: int, n_virt: int, n_frozen: int) -> np.ndarray:
    """Delta_ia = eps_a - eps_i for active i (outer) and all a (inner)."""
    occ = eps[n_frozen:n_occ]
    virt = eps[n_occ:n_occ + n_virt]
    return (virt[None, :] - occ[:, None]).reshape(-1)


# ----------------------------------------------------------------------------
# Natural auxiliary functions (Sec. 2, Eqs. nafeq and naftrafo)
# ----------------------------------------------------------------------------
def naf_metric(B_act: np.ndarray) -> np.ndarray:
    """K_PQ = sum_{ia} R^P_ia R^Q_ia over active occupied-virtual pairs."""
    return B_act @ B_act.T


def naf_basis(K: np.ndarray, thresh: float):
    """Diagonalise K and keep the eigenvectors whose eigenvalue exceeds the
    threshold; they form the columns of U.  Returns (U, kept eigenvalues,
    all eigenvalues ascending)."""
    lam, V = np.linalg.eigh(K)
    keep = lam > thresh
    return V[:, keep], lam[keep], lam


def naf_project(B: np.ndarray, U: np.ndarray) -> np.ndarray:
    """R^{P~}_nm = sum_P R^P_nm U_{P P~}: here B is [P][nm], output [P~][nm]."""
    return U.T @ B


# ----------------------------------------------------------------------------
# Polarisability (Eq. Pi and its Laplace form)
# ----------------------------------------------------------------------------
def polarizability_direct(Bt: np.ndarray, delta: np.ndarray, omegas: np.ndarray, spin: int = 2) -> np.ndarray:
    """Pi_PQ(i w) = -2 s sum_ia R^P_ia Delta / (w^2 + Delta^2) R^Q_ia for every w."""
    out = np.empty((len(omegas), Bt.shape[0], Bt.shape[0]))
    for j, w in enumerate(omegas):
        d = delta / (w * w + delta * delta)
        out[j] = -2.0 * spin * ((Bt * d[None, :]) @ Bt.T)
    return out


def laplace_moments(Bt: np.ndarray, delta: np.ndarray, x: np.ndarray, w: np.ndarray) -> np.ndarray:
    """M^m_PQ = sum_ia R^P_ia w_m Delta_ia exp(-Delta_ia^2 x_m) R^Q_ia."""
    out = np.empty((len(x), Bt.shape[0], Bt.shape[0]))
    for m in range(len(x)):
        c = w[m] * delta * np.exp(-delta * delta * x[m])
        out[m] = (Bt * c[None, :]) @ Bt.T
    return out


def polarizability_lt(M: np.ndarray, omegas: np.ndarray, x: np.ndarray, spin: int = 2) -> np.ndarray:
    """Pi_PQ(i w) ~ -2 s sum_m M^m_PQ exp(-w^2 x_m)."""
    out = np.empty((len(omegas),) + M.shape[1:])
    for j, om in enumerate(omegas):
        e = np.exp(-om * om * x)
        out[j] = -2.0 * spin * np.tensordot(e, M, axes=(0, 0))
    return out


# ----------------------------------------------------------------------------
# Imaginary-time (cosine-transform) form of Pi
# ----------------------------------------------------------------------------
# The alternative to Eq. LT's factorisation in X = w^2 + Delta^2: the
# Fourier-cosine representation Delta / (w^2 + Delta^2) = int_0^inf cos(w t)
# e^{-Delta t} dt, discretised on nodes tau_k with per-frequency coefficients
# gamma_jk, so that Pi_j = -2 s sum_k gamma_jk M^k with
# M^k = R~ diag(e^{-Delta tau_k}) R~^T.
def cosine_grid(n_tau: int, dmin: float, dmax: float, omegas, ridge: float = 0.0, n_samples: int = 2000):
    """A grid for the imaginary-time form: geometric tau from 0.1/dmax to 8/dmin and,
    per frequency, the least-squares (SVD) coefficients of the error scaled by the
    target's largest value over log-spaced Delta in [dmin, dmax], optionally with
    ridge times the squared coefficients of unit-norm columns.  Returns
    (tau, gamma [n_omega][n_tau], amplification = max sum_k |gamma_jk| e^{-Delta tau_k}
    over the target's largest value)."""
    tau = np.geomspace(0.1 / dmax, 8.0 / dmin, n_tau)
    D = np.geomspace(dmin, dmax, n_samples)
    E = np.exp(-D[:, None] * tau[None, :])
    gamma = np.empty((len(omegas), n_tau))
    amp = 0.0
    for j, om in enumerate(omegas):
        f = D / (om * om + D * D)
        s = f.max()
        A = E / s
        cn = np.linalg.norm(A, axis=0)
        As = np.vstack([A / cn, np.sqrt(ridge) * np.eye(n_tau)])
        y = np.concatenate([f / s, np.zeros(n_tau)])
        gamma[j] = np.linalg.lstsq(As, y, rcond=None)[0] / cn
        amp = max(amp, (np.abs(E * gamma[j][None, :]).sum(1) / s).max())
    return tau, gamma, amp


def tau_moments(Bt: np.ndarray, delta: np.ndarray, tau: np.ndarray) -> np.ndarray:
    """M^k_PQ = sum_ia R^P_ia exp(-Delta_ia tau_k) R^Q_ia."""
    out = np.empty((len(tau), Bt.shape[0], Bt.shape[0]))
    for k in range(len(tau)):
        out[k] = (Bt * np.exp(-delta * tau[k])[None, :]) @ Bt.T
    return out


def polarizability_tau(M: np.ndarray, gamma: np.ndarray, spin: int = 2) -> np.ndarray:
    """Pi_j = -2 s sum_k gamma_jk M^k."""
    return -2.0 * spin * np.tensordot(gamma, M, axes=(1, 0))


# ----------------------------------------------------------------------------
# FP8 E4M3 form of the Pi contraction (per-auxiliary-row scales)
# ----------------------------------------------------------------------------
# Not a step of the paper: the low-precision variant of the Pi contraction.
# Its plain definition: every operand value, after a per-row scale that maps
# the row's largest magnitude to the largest finite E4M3 value, is written as
# a two-term E4M3 expansion x ~ h + l (h = e4m3(x), l = e4m3(x - h), both in
# the row's scaled units), and the products h_a h_b + h_a l_b + l_a h_b of two
# operands are summed exactly (l_a l_b, below the expansion's own error, is
# left out).  The values fed to the rounding are formed in FP32 exactly as a
# GPU forms them (FP32 copy of R~, FP32 per-pair scale, FP32 products), so
# that both sides take every rounding decision on the same number.
E4M3_MAX = 448.0


def e4m3_round(v) -> np.ndarray:
    """Round to the FP8 E4M3 grid (OCP 8-bit floating point: 4 exponent bits,
    bias 7, 3 mantissa bits, subnormals below 2^-6 with spacing 2^-9, largest
    finite value 448, no infinities), round half to even, saturating at +-448."""
    v = np.asarray(v, dtype=np.float64)
    a = np.abs(v)
    _, e = np.frexp(a)                      # a = f 2^e with f in [0.5, 1)
    e = np.maximum(e - 1, -6)               # binade 2^e <= a < 2^(e+1); subnormals share 2^-6's spacing
    q = np.ldexp(1.0, e - 3)                # 3 mantissa bits: spacing 2^(e-3)
    r = np.minimum(np.rint(a / q) * q, E4M3_MAX)
    return np.copysign(r, v)


def fp8_row_quantize(X):
    """Per-row scaling onto the E4M3 grid: inv_r = 448 / max_j |X_rj| (FP32;
    0 for a zero row), codes = e4m3(X_rj * inv_r) with the product in FP32.
    X ~ codes / inv_r.  Returns (codes as float64, inv as float32)."""
    X = np.asarray(X, dtype=np.float32)
    m = np.abs(X).max(axis=1)
    inv = np.zeros_like(m)
    nz = m > 0
    inv[nz] = np.float32(E4M3_MAX) / m[nz]
    return e4m3_round(X * inv[:, None]), inv


def fp8_row_split(X):
    """Per-row scaling onto the E4M3 grid as a two-term expansion: inv_r as in
    fp8_row_quantize, xs = X_rj * inv_r (FP32), h = e4m3(xs), l = e4m3(xs - h)
    (the difference is exact in FP32).  X ~ (h + l) / inv_r.  Returns (h, l as
    float64, inv as float32)."""
    X = np.asarray(X, dtype=np.float32)
    m = np.abs(X).max(axis=1)
    inv = np.zeros_like(m)
    nz = m > 0
    inv[nz] = np.float32(E4M3_MAX) / m[nz]
    xs = (X * inv[:, None]).astype(np.float32).astype(np.float64)
    h = e4m3_round(xs)
    return h, e4m3_round(xs - h), inv


def fp8_split_product(A, B):
    """(h_A h_B^T + h_A l_B^T + l_A h_B^T) / (inv_A inv_B^T) for the two-term
    expansions of the rows of A and B (fp8_row_split), summed exactly."""
    ha, la, ia = fp8_row_split(A)
    hb, lb, ib = fp8_row_split(B)
    da = np.where(ia > 0, ia, 1.0).astype(np.float64)
    db = np.where(ib > 0, ib, 1.0).astype(np.float64)
    return (ha @ hb.T + ha @ lb.T + la @ hb.T) / da[:, None] / db[None, :]


def pi_factor_table(delta, omegas=None, x=None, w=None, tau=None) -> np.ndarray:
    """Per-pair factors in FP64: Delta / (w_j^2 + Delta^2) per frequency (Eq. Pi),
    w_m Delta exp(-Delta^2 x_m) per Laplace point (the M^m form) or
    exp(-Delta tau_k) per imaginary-time node."""
    delta = np.asarray(delta, dtype=np.float64)
    if tau is not None:
        rows = [np.exp(-delta * t) for t in tau]
    elif x is None:
        rows = [delta / (om * om + delta * delta) for om in omegas]
    else:
        rows = [w[m] * delta * np.exp(-delta * delta * x[m]) for m in range(len(x))]
    return np.array(rows)


def pi_scale_table(delta, omegas=None, x=None, w=None, tau=None) -> np.ndarray:
    """The factors of pi_factor_table, each formed in FP64 and rounded once to FP32."""
    return pi_factor_table(delta, omegas, x, w, tau).astype(np.float32)


def polarizability_fp8(Bt, delta, omegas, spin: int = 2, x=None, w=None, tau=None, gamma=None) -> np.ndarray:
    """Pi in the FP8 E4M3 form: B32 = fp32(R~); for each frequency (Eq. Pi) or
    Laplace point (M^m form) with FP32 factors s_k, A_k = fp32(B32 * s_k);
    M_k = fp8_split_product(A_k, B32) (two-term E4M3 expansions per auxiliary
    row, three products summed exactly), lower triangle mirrored; then Pi as
    in polarizability_direct, polarizability_lt or (tau, gamma)
    polarizability_tau."""
    B32 = np.asarray(Bt, dtype=np.float32)
    S = pi_scale_table(delta, omegas, x, w, tau)
    M = np.empty((len(S), B32.shape[0], B32.shape[0]))
    for k in range(len(S)):
        Mk = fp8_split_product((B32 * S[k][None, :]).astype(np.float32), B32)
        # qA qB^T is not exactly symmetric (the two operands carry different
        # scales): the lower triangle (P >= Q) is formed and mirrored
        M[k] = np.tril(Mk) + np.tril(Mk, -1).T
    if tau is not None:
        return polarizability_tau(M, gamma, spin)
    if x is None:
        return -2.0 * spin * M
    return polarizability_lt(M, omegas, x, spin)


# ----------------------------------------------------------------------------
# FP64-accurate product from integer slices (not a step of the paper: an
# emulation of FP64 contractions on tensor cores that multiply small integers
# exactly)
# ----------------------------------------------------------------------------
# Its plain definition: each row r of an operand X is written in fixed point
# relative to e_r, the exponent of the row's largest magnitude (max|X_r| <
# 2^e_r), Q = rint(X_r 2^(7 s - e_r)) (nearest, ties to even), and Q in s
# balanced base-128 digits a_1 (most significant) .. a_s, so that
# X_r ~ 2^e_r sum_i a_i 2^(-7 i) with |a_i| <= 64 (|a_1| <= 128).  Products of
# two such operands keep the digit pairs with i + j <= s + 1 and sum them
# exactly: D = sum_{i+j<=s+1} 2^(-7(i+j)) (a_i b_j^T) 2^(e_A + e_B).
SLICE_BITS = 7


def slice_rows(X, n_slices: int):
    """(digits [n_slices][rows][cols] as float64 integers, e [rows]) of the
    fixed-point rows of X (see above)."""
    X = np.asarray(X, dtype=np.float64)
    m = np.abs(X).max(axis=1)
    _, e = np.frexp(m)                          # m = f 2^e, f in [0.5, 1): m < 2^e
    e = np.where(m > 0, e, 0).astype(np.int64)
    Q = np.rint(np.ldexp(X, (SLICE_BITS * n_slices - e)[:, None]))   # exact scaling, exact rounding
    digits = np.empty((n_slices,) + X.shape)
    for i in range(n_slices - 1, -1, -1):       # least significant first, balanced
        t = np.floor((Q + 64.0) / 128.0)
        digits[i] = Q - 128.0 * t
        Q = t
    digits[0] += 128.0 * Q                      # what is left belongs to the leading digit
    return digits, e


def slice_product(A, B, n_slices: int = 6) -> np.ndarray:
    """A B^T from the integer slices of A's and B's rows, digit pairs with
    i + j <= n_slices + 1, each pair's integer product summed exactly."""
    a, ea = slice_rows(A, n_slices)
    b, eb = slice_rows(B, n_slices)
    D = np.zeros((A.shape[0], B.shape[0]))
    for L in range(2, n_slices + 2):
        acc = np.zeros((A.shape[0], B.shape[0]), dtype=np.int64)
        for i in range(1, L):
            j = L - i
            if i <= n_slices and j <= n_slices:
                acc += a[i - 1].astype(np.int64) @ b[j - 1].astype(np.int64).T
        D += np.ldexp(acc.astype(np.float64), -SLICE_BITS * L)
    return np.ldexp(np.ldexp(D, ea[:, None]), eb[None, :])


def polarizability_emulated(Bt, delta, omegas, spin: int = 2, x=None, w=None, n_slices: int = 6) -> np.ndarray:
    """Pi with every contraction from integer slices: for each frequency (Eq.
    Pi) or Laplace point (M^m form) with FP64 factors f_t (pi_factor_table),
    A_t = R~ diag(f_t) in FP64 (one rounding per entry), M_t =
    slice_product(A_t, R~, n_slices), lower triangle (P >= Q) mirrored; then
    Pi as in polarizability_direct or polarizability_lt."""
    Bt = np.asarray(Bt, dtype=np.float64)
    S = pi_factor_table(delta, omegas, x, w)
    M = np.empty((len(S), Bt.shape[0], Bt.shape[0]))
    for t in range(len(S)):
        Mt = slice_product(Bt * S[t][None, :], Bt, n_slices)
        M[t] = np.tril(Mt) + np.tril(Mt, -1).T
    if x is None:
        return -2.0 * spin * M
    return polarizability_lt(M, omegas, x, spin)


# ----------------------------------------------------------------------------
# Screened interaction (Eq. ScreenedCoulombOrbital)
# ----------------------------------------------------------------------------
def screened_interaction(Pi: np.ndarray) -> np.ndarray:
    """C(i w) = [1 - Pi(i w)]^-1 - 1 through a Cholesky factorisation of the
    symmetric positive definite 1 - Pi (Pi is negative semidefinite)."""
    n = Pi.shape[-1]
    eye = np.eye(n)
    out = np.empty_like(Pi)
    for j in range(Pi.shape[0]):
        A = eye - Pi[j]
        L = np.linalg.cholesky(A)
        Linv = np.linalg.solve(L, eye)
        out[j] = Linv.T @ Linv - eye
    return out


def w_nm(C: np.ndarray, Bt_tgt: np.ndarray) -> np.ndarray:
    """W^c_nm(i w_j) = sum_PQ R^P_nm C_j,PQ R^Q_nm for each target n (first
    index of Bt_tgt [T][P][m]) and every orbital m; returns [T][m][j]."""
    T, N, M = Bt_tgt.shape
    out = np.empty((T, M, C.shape[0]))
    for t in range(T):
        b = Bt_tgt[t]
        for j in range(C.shape[0]):
            out[t, :, j] = np.einsum("pm,pm->m", b, C[j] @ b)
    return out


# ----------------------------------------------------------------------------
# Self-energy on the imaginary axis (Eq. CorrelationSelfEnergy)
# ----------------------------------------------------------------------------
def sigma_iw(W: np.ndarray, eps_m: np.ndarray, eps_F: float, omegas: np.ndarray,
             weights: np.ndarray, eval_at=None) -> np.ndarray:
    """Sigma^c_n(i w_l) = -(1/pi) sum_m sum_j g_j z/(z^2 + w_j^2) W_nm(i w_j),
    z = i w_l + eps_F - eps_m, with the modified Gauss-Legendre nodes w_j and
    weights g_j.  W is [T][m][j]; the evaluation frequencies w_l default to the
    nodes themselves.  Returns complex [T][l]."""
    T = W.shape[0]
    eval_at = omegas if eval_at is None else np.asarray(eval_at, dtype=np.float64)
    out = np.empty((T, len(eval_at)), dtype=np.complex128)
    for l, wl in enumerate(eval_at):
        z = 1j * wl + eps_F - eps_m                                # [m]
        kern = z[:, None] / (z[:, None] ** 2 + omegas[None, :] ** 2)  # [m][j]
        kern = kern * weights[None, :]
        out[:, l] = -np.einsum("tmj,mj->t", W, kern) / np.pi
    return out


# ----------------------------------------------------------------------------
# Analytic continuation: N-point Pade (Vidberg & Serene, appendix)
# ----------------------------------------------------------------------------
def pade_coefficients(z: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Continued-fraction coefficients a_p = g_p(z_p) with g_1(z_i) = u_i and
    g_p(z) = [g_{p-1}(z_{p-1}) - g_{p-1}(z)] / [(z - z_{p-1}) g_{p-1}(z)]."""
    n = len(z)
    g = np.array(u, dtype=np.complex128)   # g_{p}(z_i) for i >= p, updated in place
    a = np.empty(n, dtype=np.complex128)
    a[0] = g[0]
    for p in range(1, n):
        g[p:] = (g[p - 1] - g[p:]) / ((z[p:] - z[p - 1]) * g[p:])
        a[p] = g[p]
    return a


def pade_eval(z_nodes: np.ndarray, a: np.ndarray, z: complex):
    """C_N(z) = a_1 / (1 + a_2 (z - z_1) / (1 + a_3 (z - z_2) / (1 + ...))),
    evaluated from the innermost level outwards, with its derivative dC/dz."""
    n = len(a)
    t = 1.0 + 0j          # innermost denominator level
    dt = 0.0 + 0j
    for p in range(n - 1, 0, -1):
        num = a[p] * (z - z_nodes[p - 1])
        dnum = a[p]
        new_t = 1.0 + num / t
        new_dt = dnum / t - num * dt / (t * t)
        t, dt = new_t, new_dt
    val = a[0] / t
    dval = -a[0] * dt / (t * t)
    return val, dval


def qp_newton(eps_n: float, shift: float, eps_F: float, z_nodes: np.ndarray, a: np.ndarray,
              eta: float = 0.0, tol: float = 1e-12, max_iter: int = 100):
    """Solve E = eps_n + Re Sigma^c_n(E) + shift with Sigma^c_n(E) = C_N(E - eps_F + i eta)
    by Newton from E = eps_n.  Returns (E, status): status 0 converged, 1 not."""
    E = eps_n
    for _ in range(max_iter):
        s, ds = pade_eval(z_nodes, a, complex(E - eps_F, eta))
        f = E - eps_n - s.real - shift
        fp = 1.0 - ds.real
        dE = -f / fp
        E = E + dE
        if abs(dE) < tol:
            return E, 0
    return E, 1


# ----------------------------------------------------------------------------
# Whole path
# ----------------------------------------------------------------------------
def pade_nodes(n_omega: int) -> np.ndarray:
    """Indices of the Gauss-Legendre nodes the continuation passes through."""
    return np.arange(0, n_omega, 2)


def solve(eps, B_ov, B_tgt, targets, shift, n_occ, n_virt, n_frozen=0, n_omega=24,
          omega0=0.5, naf_thresh=-1.0, spin=2, tau_x=None, tau_w=None, return_all=False, cos_tau=None,
          cos_gamma=None, eps_qp_ref=None):
    """One G0W0 solve.  Direct Pi (Eq. Pi) unless a Laplace grid (tau_x, tau_w)
    is given, in which case Pi is built from the moments M^m, or an
    imaginary-time grid (cos_tau [n_tau], cos_gamma [n_omega][n_tau]), in which
    case Pi_j = -2 s sum_k gamma_jk M^k with M^k = R~ diag(e^{-Delta tau_k}) R~^T.
    eps_qp_ref: energies of the quasi-particle equation's reference eps_n (and
    Newton's start) when they differ from the energies of Pi and Sigma (evGW).
    B_ov [P][i*n_virt+a] (all occupied i), B_tgt [T][P][m] (all orbitals m).
    Returns (sigma [T][n_omega] complex, e_qp [T], status [T]) and, with
    return_all, a dict of intermediates."""
    eps = np.asarray(eps, dtype=np.float64)
    targets = np.asarray(targets)
    if np.any(targets < n_frozen):
        raise ValueError("frozen-core orbitals cannot be targets")
    B_act = active_ov(B_ov, n_occ, n_virt, n_frozen)
    inter = {}
    if naf_thresh >= 0.0:
        K = naf_metric(B_act)
        U, lam_kept, lam_all = naf_basis(K, naf_thresh)
        Bt = naf_project(B_act, U)
        Bt_tgt = np.stack([naf_project(B_tgt[t][:, n_frozen:], U) for t in range(len(targets))])
        inter.update(K=K, U=U, lam=lam_all, n_naf=U.shape[1])
    else:
        Bt = B_act
        Bt_tgt = np.ascontiguousarray(B_tgt[:, :, n_frozen:])
        inter.update(U=None, n_naf=Bt.shape[0])
    out = solve_projected(eps, Bt, Bt_tgt, targets, shift, n_occ, n_virt, n_frozen, n_omega, omega0, spin,
                          tau_x, tau_w, return_all, cos_tau, cos_gamma, eps_qp_ref)
    if return_all:
        out[3].update(inter)
    return out


def solve_projected(eps, Bt, Bt_tgt, targets, shift, n_occ, n_virt, n_frozen=0, n_omega=24, omega0=0.5,
                    spin=2, tau_x=None, tau_w=None, return_all=False, cos_tau=None, cos_gamma=None,
                    eps_qp_ref=None):
    """The solve after the NAF step: Pi, the screening, W_nm, Sigma(i w), the
    Pade fraction and Newton, from the active-pair block Bt [N][n_act*n_virt]
    (in the NAF basis, or the raw block without NAF) and the targets' blocks
    Bt_tgt [T][N][m] over the active orbitals m.  Other arguments as `solve`."""
    eps = np.asarray(eps, dtype=np.float64)
    targets = np.asarray(targets)
    omegas, weights = gl_grid(n_omega, omega0)
    eF = fermi_level(eps, n_occ)
    delta = pair_gaps(eps, n_occ, n_virt, n_frozen)
    inter = {"omegas": omegas, "weights": weights, "eps_F": eF}
    if cos_tau is not None:
        M = tau_moments(Bt, delta, np.asarray(cos_tau))
        Pi = polarizability_tau(M, np.asarray(cos_gamma), spin)
        inter["M"] = M
    elif tau_x is None:
        Pi = polarizability_direct(Bt, delta, omegas, spin)
    else:
        M = laplace_moments(Bt, delta, np.asarray(tau_x), np.asarray(tau_w))
        Pi = polarizability_lt(M, omegas, np.asarray(tau_x), spin)
        inter["M"] = M
    C = screened_interaction(Pi)
    W = w_nm(C, Bt_tgt)
    eps_m = eps[n_frozen:]
    sig = sigma_iw(W, eps_m, eF, omegas, weights)
    sel = pade_nodes(n_omega)
    z_nodes = 1j * omegas[sel]
    e_qp = np.empty(len(targets))
    status = np.empty(len(targets), dtype=np.int32)
    coefs = []
    ref = eps if eps_qp_ref is None else np.asarray(eps_qp_ref, dtype=np.float64)
    for t, n in enumerate(targets):
        a = pade_coefficients(z_nodes, sig[t][sel])
        coefs.append(a)
        e_qp[t], status[t] = qp_newton(ref[n], shift[t], eF, z_nodes, a)
    if return_all:
        inter.update(Bt=Bt, Bt_tgt=Bt_tgt, Pi=Pi, C=C, W=W, pade=np.array(coefs), delta=delta)
        return sig, e_qp, status, inter
    return sig, e_qp, status


# ----------------------------------------------------------------------------
# The same solve for an RI tensor supplied one block of occupied orbitals at a
# time (Eqs. nafeq and naftrafo: K is a sum over the active pairs, so it is
# summed block by block; the projection acts column by column)
# ----------------------------------------------------------------------------
def occ_blocks(n_occ: int, n_frozen: int, occ_block: int):
    """The active occupied ranges [i0, i1) of occ_block orbitals (the last may be shorter)."""
    return [(i0, min(n_occ, i0 + occ_block)) for i0 in range(n_frozen, n_occ, occ_block)]


def naf_metric_blocked(ov_block, blocks) -> np.ndarray:
    """K_PQ = sum over blocks of sum_{ia in block} R^P_ia R^Q_ia; ov_block(i0, i1)
    returns R [P][(i - i0) n_virt + a] for i0 <= i < i1."""
    K = None
    for i0, i1 in blocks:
        R = ov_block(i0, i1)
        K = naf_metric(R) if K is None else K + naf_metric(R)
    return K


def naf_project_blocked(ov_block, blocks, U: np.ndarray, n_virt: int) -> np.ndarray:
    """R~ = U^T R for the active pairs, assembled block by block: [N][n_act n_virt]."""
    n_pairs = sum(i1 - i0 for i0, i1 in blocks) * n_virt
    out = np.empty((U.shape[1], n_pairs))
    c = 0
    for i0, i1 in blocks:
        R = ov_block(i0, i1)
        out[:, c:c + R.shape[1]] = naf_project(R, U)
        c += R.shape[1]
    return out


def solve_blocked(eps, ov_block, B_tgt, targets, shift, n_occ, n_virt, n_frozen, occ_block, n_omega=24,
                  omega0=0.5, naf_thresh=0.0, spin=2, tau_x=None, tau_w=None, return_all=False):
    """`solve` with B_ov supplied by ov_block(i0, i1) for the active occupied
    blocks of occ_block orbitals (NAF required, naf_thresh >= 0): K summed over
    the blocks, then the kept eigenvectors, the blockwise projection and
    solve_projected.  Other arguments as `solve`."""
    if naf_thresh < 0.0:
        raise ValueError("solve_blocked needs NAF (naf_thresh >= 0)")
    targets = np.asarray(targets)
    if np.any(targets < n_frozen):
        raise ValueError("frozen-core orbitals cannot be targets")
    blocks = occ_blocks(n_occ, n_frozen, occ_block)
    K = naf_metric_blocked(ov_block, blocks)
    U, lam_kept, lam_all = naf_basis(K, naf_thresh)
    Bt = naf_project_blocked(ov_block, blocks, U, n_virt)
    Bt_tgt = np.stack([naf_project(B_tgt[t][:, n_frozen:], U) for t in range(len(targets))])
    out = solve_projected(eps, Bt, Bt_tgt, targets, shift, n_occ, n_virt, n_frozen, n_omega, omega0, spin,
                          tau_x, tau_w, return_all)
    if return_all:
        out[3].update(K=K, U=U, lam=lam_all, n_naf=U.shape[1])
    return out


# ----------------------------------------------------------------------------
# Eigenvalue-self-consistent GW (Sec. 3, computational details; the evGW
# timings table of Sec. 4)
# ----------------------------------------------------------------------------
def evgw_energies(eps_ks, targets, e_qp, n_frozen: int = 0) -> np.ndarray:
    """Orbital energies for the next evGW cycle: the quasi-particle energies for
    the target states; every other active orbital shifted by the shift
    (E_QP - eps) of the target nearest to it by orbital index (ties: the lower
    one), which below and above the window is the shift of the lowest and of
    the highest target; frozen-core orbitals unchanged."""
    eps_ks = np.asarray(eps_ks, dtype=np.float64)
    tg = np.asarray(targets)
    order = np.argsort(tg)
    tg = tg[order]
    sh = (np.asarray(e_qp, dtype=np.float64) - eps_ks[np.asarray(targets)])[order]
    out = eps_ks.copy()
    for p in range(n_frozen, len(eps_ks)):
        k = int(np.searchsorted(tg, p))
        if k < len(tg) and tg[k] == p:
            out[p] = eps_ks[p] + sh[k]
            continue
        cand = []
        if k - 1 >= 0:
            cand.append((p - tg[k - 1], 0, k - 1))
        if k < len(tg):
            cand.append((tg[k] - p, 1, k))
        out[p] = eps_ks[p] + sh[min(cand)[2]]
    return out


def evgw(eps, B_ov, B_tgt, targets, shift, n_occ, n_virt, n_frozen=0, n_cycles=5, gap_tol=0.0, **solve_kw):
    """evGW: cycle 0 is G0W0 on the input energies; each of up to n_cycles further
    cycles recomputes Pi, W and Sigma with evgw_energies of the previous cycle,
    keeping the input eps_n + (Sigma_x - V_xc)_n as the quasi-particle equation's
    reference.  With gap_tol > 0 and both HOMO and LUMO among the targets, it
    stops once the quasi-particle HOMO/LUMO gap changes by less than gap_tol.
    Returns (sigma, e_qp, status, cycles after G0W0)."""
    eps0 = np.asarray(eps, dtype=np.float64)
    targets = np.asarray(targets)
    sig, e, st = solve(eps0, B_ov, B_tgt, targets, shift, n_occ, n_virt, n_frozen, eps_qp_ref=eps0, **solve_kw)
    ih = np.where(targets == n_occ - 1)[0]
    il = np.where(targets == n_occ)[0]
    done = 0
    for _ in range(n_cycles):
        cur = evgw_energies(eps0, targets, e, n_frozen)
        sig, e_new, st = solve(cur, B_ov, B_tgt, targets, shift, n_occ, n_virt, n_frozen, eps_qp_ref=eps0,
                               **solve_kw)
        done += 1
        conv = (gap_tol > 0 and len(ih) and len(il) and
                abs((e_new[il[0]] - e_new[ih[0]]) - (e[il[0]] - e[ih[0]])) < gap_tol)
        e = e_new
        if conv:
            break
    return sig, e, st, done
