"""Seeded synthetic G0W0 inputs (orbital energies, RI tensor blocks, shifts).

This module generates workloads only; it contains none of the GW method's
arithmetic, so both the CPU oracle and the CUDA path can consume its arrays.

The law (one fixed reading, used for every workload):

* orbital energies, ascending: ``n_frozen`` core levels uniform in [-20, -10] Ha,
  ``n_occ - n_frozen`` valence levels uniform in [-1, -0.25] Ha, ``n_virt``
  virtual levels uniform in [0.02, 3.0] Ha, each group sorted;
* RI tensor ``B[Q, p, q] = sum_r U[Q, r] sigma_r Z[r, p, q] / sqrt(n_occ n_virt)``
  with ``U`` the orthogonal factor of the QR decomposition of a Gaussian
  ``n_aux x n_aux`` matrix (sign fixed so that diag(R) > 0),
  ``sigma_r = 0.5 exp(-6 r / n_aux)`` and ``Z[r, p, q]`` a standard normal drawn
  by Philox4x32-10 at counter ``(r, min(p, q), max(p, q))``, so ``B`` is
  symmetric in ``p, q``;
* a diagonal exchange-minus-xc shift per target, uniform in [-0.05, 0.05] Ha.

Random streams (the Philox key's high word is offset by the stream tag):
0 = pair normals Z, 1 = the Gaussian behind U, 2 = energies, 3 = shifts.

Layouts handed to the solver:
* ``B_ov[Q, i * n_virt + a] = B[Q, i, n_occ + a]`` for all occupied ``i``
  (frozen rows included; the solver slices them away);
* ``B_tgt[t, Q, m] = B[Q, targets[t], m]`` for all orbitals ``m``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "philox_gen.c")
_LIB_PATH = os.path.join(_HERE, "_philox_gen.so")
_lib = None

STREAM_Z, STREAM_U, STREAM_EPS, STREAM_SHIFT = 0, 1, 2, 3


def build_generator(force: bool = False) -> str:
    """Compile the host generator with gcc (OpenMP) into this directory."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_generator())
        u64, u32, i64, dp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64, ctypes.c_void_p
        lib.synth_philox4x32_10.argtypes = [dp, dp, dp]
        lib.synth_uniform.argtypes = [u64, u32, i64, ctypes.c_double, ctypes.c_double, u32, dp]
        lib.synth_normal_matrix.argtypes = [u64, u32, i64, i64, dp]
        lib.synth_pair_normals_ov.argtypes = [u64, u32, i64, i64, i64, i64, i64, dp]
        lib.synth_pair_normals_row.argtypes = [u64, u32, i64, i64, i64, dp]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def philox4x32_10(counter, key) -> np.ndarray:
    """Raw Philox4x32-10 block for a 4-word counter and 2-word key."""
    c = np.ascontiguousarray(counter, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().synth_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def uniform(seed: int, stream: int, n: int, lo: float, hi: float, group: int = 0) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    if n:
        _load().synth_uniform(seed, stream, n, lo, hi, group, _ptr(out))
    return out


def normal_matrix(seed: int, stream: int, rows: int, cols: int) -> np.ndarray:
    out = np.empty((rows, cols), dtype=np.float64)
    _load().synth_normal_matrix(seed, stream, rows, cols, _ptr(out))
    return out


def pair_normals_ov(seed: int, n_aux: int, n_occ: int, n_virt: int, i0: int = 0, i1: int | None = None) -> np.ndarray:
    i1 = n_occ if i1 is None else i1
    out = np.empty((n_aux, (i1 - i0) * n_virt), dtype=np.float64)
    _load().synth_pair_normals_ov(seed, STREAM_Z, n_aux, n_occ, n_virt, i0, i1, _ptr(out))
    return out


def pair_normals_row(seed: int, n_aux: int, n_orb: int, p: int) -> np.ndarray:
    out = np.empty((n_aux, n_orb), dtype=np.float64)
    _load().synth_pair_normals_row(seed, STREAM_Z, n_aux, n_orb, p, _ptr(out))
    return out


def aux_rotation(seed: int, n_aux: int) -> np.ndarray:
    """Orthogonal U from the QR decomposition of a seeded Gaussian, diag(R) > 0."""
    g = normal_matrix(seed, STREAM_U, n_aux, n_aux)
    q, r = np.linalg.qr(g)
    s = np.sign(np.diag(r))
    s[s == 0] = 1.0
    return np.ascontiguousarray(q * s[None, :])


def aux_loading(seed: int, n_aux: int, n_occ: int, n_virt: int) -> np.ndarray:
    """L[Q, r] = U[Q, r] sigma_r / sqrt(n_occ n_virt), so that B = L Z."""
    u = aux_rotation(seed, n_aux)
    sigma = 0.5 * np.exp(-6.0 * np.arange(n_aux) / n_aux)
    return np.ascontiguousarray(u * (sigma / np.sqrt(n_occ * n_virt))[None, :])


def orbital_energies(seed: int, n_occ: int, n_virt: int, n_frozen: int) -> np.ndarray:
    core = np.sort(uniform(seed, STREAM_EPS, n_frozen, -20.0, -10.0, group=0))
    val = np.sort(uniform(seed, STREAM_EPS, n_occ - n_frozen, -1.0, -0.25, group=1))
    virt = np.sort(uniform(seed, STREAM_EPS, n_virt, 0.02, 3.0, group=2))
    return np.concatenate([core, val, virt])


def gap_targets(n_occ: int, n_targets: int) -> np.ndarray:
    """The n_targets states around the gap: half occupied, half virtual."""
    h = n_targets // 2
    return np.arange(n_occ - h, n_occ - h + n_targets, dtype=np.int32)


@dataclass
class Problem:
    """One synthetic G0W0 request in the layouts the solver takes."""
    n_occ: int
    n_virt: int
    n_frozen: int
    n_aux: int
    seed: int
    eps: np.ndarray
    B_ov: np.ndarray
    B_tgt: np.ndarray
    targets: np.ndarray
    shift: np.ndarray
    meta: dict = field(default_factory=dict)


def make_problem(n_occ: int, n_virt: int, n_aux: int, n_frozen: int = 0, seed: int = 20230710,
                 n_targets: int = 2, targets=None, with_ov: bool = True) -> Problem:
    eps = orbital_energies(seed, n_occ, n_virt, n_frozen)
    tg = gap_targets(n_occ, n_targets) if targets is None else np.asarray(targets, dtype=np.int32)
    load = aux_loading(seed, n_aux, n_occ, n_virt)
    n_orb = n_occ + n_virt
    if with_ov:
        B_ov = np.ascontiguousarray(load @ pair_normals_ov(seed, n_aux, n_occ, n_virt))
    else:
        B_ov = np.empty((n_aux, 0))
    B_tgt = np.empty((len(tg), n_aux, n_orb), dtype=np.float64)
    for t, p in enumerate(tg):
        B_tgt[t] = load @ pair_normals_row(seed, n_aux, n_orb, int(p))
    shift = uniform(seed, STREAM_SHIFT, len(tg), -0.05, 0.05)
    return Problem(n_occ, n_virt, n_frozen, n_aux, seed, eps, B_ov, B_tgt, tg, shift)


# The workloads, by size.  Seeds: tiny 20230710, mid +1, large +2.
TINY = dict(n_occ=4, n_virt=16, n_aux=48, n_frozen=0, seed=20230710, n_targets=2,
            n_omega=24, n_tau=6, naf_thresh=-1.0)
MID = dict(n_occ=60, n_virt=540, n_aux=1800, n_frozen=10, seed=20230711, n_targets=10,
           n_omega=32, n_tau=8, naf_thresh=1e-2)
LARGE = dict(n_occ=320, n_virt=3500, n_aux=9000, n_frozen=60, seed=20230712, n_targets=20,
             n_omega=32, n_tau=10, naf_thresh=1e-2)


def make_workload(cfg: dict, **over) -> Problem:
    c = dict(cfg)
    c.update(over)
    return make_problem(c["n_occ"], c["n_virt"], c["n_aux"], c["n_frozen"], c["seed"], c["n_targets"])


STREAM_SERVING = 4


def serving_stream(n_requests: int = 512, rate_hz: float = 2.0, seed: int = 20230720, n_occ_min: int = 8,
                   n_occ_max: int = 200):
    """The serving workload: n_occ log-uniform in [n_occ_min, n_occ_max], frozen
    core n_occ // 6, n_virt = round(u n_occ) with u uniform in [8, 12],
    N_aux = 3 (n_occ + n_virt), 4 target states, request seed = seed + 1 + index,
    Poisson arrivals at rate_hz (exponential gaps).  Draws come from Philox
    stream 4 at counters (index, 0..2)."""
    u0 = uniform(seed, STREAM_SERVING, n_requests, 0.0, 1.0, group=0)
    u1 = uniform(seed, STREAM_SERVING, n_requests, 8.0, 12.0, group=1)
    u2 = uniform(seed, STREAM_SERVING, n_requests, 0.0, 1.0, group=2)
    lo, hi = np.log(n_occ_min), np.log(n_occ_max)
    t = 0.0
    out = []
    for i in range(n_requests):
        n_occ = int(round(np.exp(lo + (hi - lo) * u0[i])))
        n_virt = int(round(u1[i] * n_occ))
        t += -np.log(1.0 - u2[i]) / rate_hz
        out.append(dict(index=i, n_occ=n_occ, n_frozen=n_occ // 6, n_virt=n_virt, n_aux=3 * (n_occ + n_virt),
                        n_targets=4, seed=seed + 1 + i, t_arrival=t))
    return out
