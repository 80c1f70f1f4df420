"""Device-side synthetic inputs, for workloads too large to generate on the host.

Same law, keys and counters as the host generator in ``__init__.py`` (Philox
normals from ``philox_dev.cu``; the rotation U from a QR factorisation and the
loading GEMM B = L Z done with torch on the GPU).  Holds no GW arithmetic.

The loading GEMM can run in FP32 (``gemm="fp32"``): the result is then the
input, shared by every form that consumes it.  Results agree with the host
generator to rounding (log/cos/GEMM order), not bit for bit.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess

import numpy as np

from . import STREAM_U, STREAM_Z, gap_targets, orbital_energies, uniform, STREAM_SHIFT

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "philox_dev.cu")
_LIB_PATH = os.path.join(_HERE, "_philox_dev.so")
_lib = None


def build_device_generator(force: bool = False) -> str:
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        nvcc = os.environ.get("NVCC") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc")
                                          else shutil.which("nvcc"))
        if not nvcc:
            raise RuntimeError("nvcc not found: the device input generator needs the CUDA toolkit")
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-shared",
                               "-Xcompiler", "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_device_generator())
        u64, u32, i64, vp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64, ctypes.c_void_p
        lib.synth_dev_pair_normals_ov.argtypes = [u64, u32, i64, i64, i64, i64, i64, vp, vp]
        lib.synth_dev_pair_normals_row.argtypes = [u64, u32, i64, i64, i64, vp, vp]
        lib.synth_dev_normal_matrix.argtypes = [u64, u32, i64, i64, vp, vp]
        _lib = lib
    return _lib


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _check(rc):
    if rc != 0:
        raise RuntimeError(f"device generator launch failed (cudaError {rc})")


def normal_matrix(seed: int, stream: int, rows: int, cols: int):
    import torch
    out = torch.empty((rows, cols), dtype=torch.float64, device="cuda")
    _check(_load().synth_dev_normal_matrix(seed, stream, rows, cols, out.data_ptr(), _stream()))
    return out


def pair_normals_ov(seed: int, rows: int, n_occ: int, n_virt: int, i0: int, i1: int, out=None):
    import torch
    if out is None:
        out = torch.empty((rows, (i1 - i0) * n_virt), dtype=torch.float64, device="cuda")
    _check(_load().synth_dev_pair_normals_ov(seed, STREAM_Z, rows, n_occ, n_virt, i0, i1, out.data_ptr(), _stream()))
    return out


def pair_normals_row(seed: int, rows: int, n_orb: int, p: int):
    import torch
    out = torch.empty((rows, n_orb), dtype=torch.float64, device="cuda")
    _check(_load().synth_dev_pair_normals_row(seed, STREAM_Z, rows, n_orb, p, out.data_ptr(), _stream()))
    return out


def aux_loading(seed: int, n_aux: int, n_occ: int, n_virt: int, qr_dtype=None, host_qr: bool = False):
    """L[Q, r] = U[Q, r] sigma_r / sqrt(n_occ n_virt) on the device (FP64 result;
    the QR factorisation runs in qr_dtype, FP64 by default).  host_qr: the
    host generator's L (numpy QR in FP64) copied to the device, for processes
    where the device QR's library cannot be loaded (under a profiler)."""
    import torch
    if host_qr:
        from . import aux_loading as host_aux_loading
        return torch.from_numpy(host_aux_loading(seed, n_aux, n_occ, n_virt)).cuda()
    g = normal_matrix(seed, STREAM_U, n_aux, n_aux)
    if qr_dtype is not None and qr_dtype != torch.float64:
        q, r = torch.linalg.qr(g.to(qr_dtype))
        q, r = q.double(), r.double()
    else:
        q, r = torch.linalg.qr(g)
    s = torch.sign(torch.diagonal(r))
    s[s == 0] = 1.0
    sigma = 0.5 * torch.exp(-6.0 * torch.arange(n_aux, dtype=torch.float64, device="cuda") / n_aux)
    return (q * s[None, :]) * (sigma / np.sqrt(n_occ * n_virt))[None, :]


class DeviceLaw:
    """One request's synthetic RI tensor, generated on the device on demand."""

    def __init__(self, n_occ, n_virt, n_aux, n_frozen=0, seed=20230710, n_targets=2, gemm="fp64", host_qr=False):
        """gemm: "fp64" (the exact law), "fp32" (QR and loading GEMM in FP32) or
        "tf32" (QR in FP32, loading GEMM on the TF32 tensor cores); host_qr
        (with "fp64"): the rotation from the host generator's QR."""
        import torch
        self.n_occ, self.n_virt, self.n_aux, self.n_frozen, self.seed = n_occ, n_virt, n_aux, n_frozen, seed
        self.gemm = gemm
        self.dtype = torch.float64 if gemm == "fp64" else torch.float32
        self.eps = orbital_energies(seed, n_occ, n_virt, n_frozen)
        self.targets = gap_targets(n_occ, n_targets)
        self.shift = uniform(seed, STREAM_SHIFT, len(self.targets), -0.05, 0.05)
        self.L = aux_loading(seed, n_aux, n_occ, n_virt, qr_dtype=self.dtype, host_qr=host_qr and gemm == "fp64")
        self._Lc = self.L.to(self.dtype)

    def _gemm(self, z):
        import torch
        prev = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = self.gemm == "tf32"
        try:
            if self.dtype == z.dtype:
                return self._Lc @ z
            return (self._Lc @ z.to(self.dtype)).to(z.dtype)
        finally:
            torch.backends.cuda.matmul.allow_tf32 = prev

    def b_ov_block(self, i0: int, i1: int, out=None, chunk_elems: int = 1 << 27):
        """B_ov columns of occupied orbitals i0..i1-1: [n_aux][(i1-i0) n_virt] FP64,
        generated through Z chunks of at most chunk_elems values."""
        import torch
        cols = (i1 - i0) * self.n_virt
        if out is None:
            out = torch.empty((self.n_aux, cols), dtype=torch.float64, device="cuda")
        step = max(1, chunk_elems // max(1, self.n_aux * self.n_virt))
        for a in range(i0, i1, step):
            b = min(i1, a + step)
            z = pair_normals_ov(self.seed, self.n_aux, self.n_occ, self.n_virt, a, b)
            out[:, (a - i0) * self.n_virt:(b - i0) * self.n_virt] = self._gemm(z)
            del z
        return out

    def b_ov(self):
        return self.b_ov_block(0, self.n_occ)

    def b_tgt(self):
        import torch
        n_orb = self.n_occ + self.n_virt
        out = torch.empty((len(self.targets), self.n_aux, n_orb), dtype=torch.float64, device="cuda")
        for t, p in enumerate(self.targets):
            out[t] = self._gemm(pair_normals_row(self.seed, self.n_aux, n_orb, int(p)))
        return out

    def fill_block(self, i0: int, i1: int, dst_ptr: int) -> int:
        """Block callback for ltgw_solve_streamed: B_ov columns of occupied
        orbitals [i0, i1) into the library's device buffer at dst_ptr."""
        import torch
        from ..ltgw import device_view
        dst = device_view(dst_ptr, (self.n_aux, (i1 - i0) * self.n_virt))
        self.b_ov_block(i0, i1, out=dst)
        torch.cuda.synchronize()
        return 0
