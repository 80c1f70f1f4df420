"""Python binding of the LT-GW C ABI (include/ltgw.h): argument marshalling only.

Every function here calls the CUDA library ``libltgw.so`` built in-tree by
``paper_2307_04508_gb300.build``; nothing is computed in Python.  Arrays may be
numpy arrays (host memory) or torch CUDA tensors (device memory); the library
detects which.  Loading fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libltgw.so")

LTGW_OK, LTGW_ERR_BAD_ARG, LTGW_ERR_NOMEM, LTGW_ERR_NOT_SPD = 0, 1, 2, 3
LTGW_ERR_NO_CONVERGE, LTGW_ERR_DEVICE, LTGW_ERR_EIG, LTGW_ERR_NO_NAF = 4, 5, 6, 7
LTGW_ERR_TIMEOUT = 8
LTGW_FP64, LTGW_BF16X3, LTGW_FP8, LTGW_FP8_PI, LTGW_FP64_EMU = 0, 1, 2, 3, 4


class Params(ctypes.Structure):
    _fields_ = [("n_occ", ctypes.c_int), ("n_virt", ctypes.c_int), ("n_frozen", ctypes.c_int),
                ("n_aux", ctypes.c_int), ("n_omega", ctypes.c_int), ("n_tau", ctypes.c_int),
                ("omega0", ctypes.c_double), ("naf_thresh", ctypes.c_double), ("spin", ctypes.c_int),
                ("use_laplace", ctypes.c_int), ("precision", ctypes.c_int), ("reserved", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("n_naf", ctypes.c_int), ("n_pade", ctypes.c_int), ("n_tau", ctypes.c_int),
                ("naf_near_threshold", ctypes.c_int), ("lt_max_rel_err", ctypes.c_double),
                ("ms_naf", ctypes.c_double), ("ms_pi", ctypes.c_double), ("ms_screen", ctypes.c_double),
                ("ms_wnm", ctypes.c_double), ("ms_sigma_qp", ctypes.c_double), ("ms_total", ctypes.c_double),
                ("ms_pi_kernel", ctypes.c_double), ("pi_kernel_launches", ctypes.c_int),
                ("kernel_launches", ctypes.c_int), ("ms_tridiag", ctypes.c_double),
                ("ms_generate", ctypes.c_double), ("tc_autotuned", ctypes.c_int),
                ("ms_naf_metric", ctypes.c_double), ("ms_eig_vectors", ctypes.c_double),
                ("ms_naf_project", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class Request(ctypes.Structure):
    _fields_ = [("p", Params), ("eps", ctypes.c_void_p), ("B_ov", ctypes.c_void_p), ("B_tgt", ctypes.c_void_p),
                ("targets", ctypes.c_void_p), ("n_tgt", ctypes.c_int), ("shift", ctypes.c_void_p),
                ("tau_x", ctypes.c_void_p), ("tau_w", ctypes.c_void_p), ("sigma_iw", ctypes.c_void_p),
                ("e_qp", ctypes.c_void_p), ("qp_status", ctypes.c_void_p)]


class Completion(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("status", ctypes.c_int), ("queue_ms", ctypes.c_double),
                ("service_ms", ctypes.c_double), ("latency_ms", ctypes.c_double), ("start_ms", ctypes.c_double),
                ("end_ms", ctypes.c_double), ("message", ctypes.c_char * 120)]


class LtgwError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"ltgw status {status}: {msg}")
        self.status = status


_lib = None

BLOCK_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                            ctypes.c_void_p)

# exported symbols and their ctypes signatures
_P, _I, _D, _I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
SIGNATURES = {
    "ltgw_create": (_I, [ctypes.POINTER(ctypes.c_void_p), _I]),
    "ltgw_destroy": (None, [_P]),
    "ltgw_status_string": (ctypes.c_char_p, [_I]),
    "ltgw_last_error": (ctypes.c_char_p, [_P]),
    "ltgw_set_timing": (_I, [_P, _I]),
    "ltgw_set_autotune": (_I, [_P, _I]),
    "ltgw_workspace_bytes": (ctypes.c_size_t, [_P]),
    "ltgw_trim": (_I, [_P]),
    "ltgw_get_stats": (_I, [_P, ctypes.POINTER(Stats)]),
    "ltgw_solve": (_I, [_P, ctypes.POINTER(Params), _P, _P, _P, _P, _I, _P, _P, _P, _P, _P, _P, _P]),
    "ltgw_solve_ev": (_I, [_P, ctypes.POINTER(Params), _P, _P, _P, _P, _I, _P, _P, _P, _I, _D, _P, _P, _P,
                           _P, _P]),
    "ltgw_solve_streamed": (_I, [_P, ctypes.POINTER(Params), _P, BLOCK_FN, _P, _I, _P, _P, _I, _P, _P, _P, _P, _P,
                                 _P, _P]),
    "ltgw_gl_grid": (_I, [_I, _D, _P, _P]),
    "ltgw_laplace_grid": (_I, [_I, _D, _D, _P, _P, _P]),
    "ltgw_cosine_grid": (_I, [_I, _D, _D, _I, _P, _D, _P, _P, _P, _P]),
    "ltgw_naf_basis": (_I, [_P, _I, _I64, _P, _I64, _D, _P, _P, ctypes.POINTER(ctypes.c_int), _P]),
    "ltgw_naf_basis_mixed": (_I, [_P, _I, _I64, _P, _I64, _D, _P, _P, ctypes.POINTER(ctypes.c_int), _P]),
    "ltgw_polarizability": (_I, [_P, _I, _I64, _P, _P, _I, _P, _I, _P, _P, _I, _P, _P]),
    "ltgw_polarizability_mixed": (_I, [_P, _I, _I64, _P, _P, _I, _P, _I, _P, _P, _I, _P, _P]),
    "ltgw_polarizability_fp8": (_I, [_P, _I, _I64, _P, _P, _I, _P, _I, _P, _P, _I, _P, _P]),
    "ltgw_polarizability_emulated": (_I, [_P, _I, _I64, _P, _P, _I, _P, _I, _P, _P, _I, _I, _P, _P]),
    "ltgw_polarizability_tau": (_I, [_P, _I, _I64, _P, _P, _I, _P, _I, _P, _P, _I, _I, _P, _P]),
    "ltgw_screen": (_I, [_P, _I, _I, _P, _P, _P]),
    "ltgw_gemm_emulated": (_I, [_P, _I, _I, _I64, _P, _I64, _P, _I64, _P, _I64, _I, _I, _P]),
    "ltgw_screen_static": (_I, [_I, _I, _P, _P, _P]),
    "ltgw_server_create": (_I, [ctypes.POINTER(ctypes.c_void_p), _I, _I, ctypes.c_size_t]),
    "ltgw_server_submit": (_I, [_P, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]),
    "ltgw_server_poll": (_I, [_P, ctypes.POINTER(Completion), _I]),
    "ltgw_server_wait_all": (_I, [_P, _D]),
    "ltgw_server_destroy": (None, [_P]),
    "ltgw_request_footprint": (ctypes.c_size_t, [ctypes.POINTER(Params), _I]),
}

SCREEN_STATIC_MAX_ELEMS = 1 << 19


def load():
    """Load libltgw.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"LT-GW CUDA library not built ({LIB_PATH} missing); "
                               "run `python -m paper_2307_04508_gb300.build`")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _ptr(a):
    """Data pointer of a numpy array or torch tensor (contiguous), or None."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


class _DeviceBuffer:
    """Zero-copy torch view of library-owned device memory (for block callbacks)."""

    def __init__(self, ptr: int, shape, typestr: str = "<f8"):
        self.__cuda_array_interface__ = {"data": (int(ptr), False), "shape": tuple(shape), "typestr": typestr,
                                         "version": 3, "strides": None}


def device_view(ptr: int, shape, dtype: str = "<f8"):
    import torch
    return torch.as_tensor(_DeviceBuffer(ptr, shape, dtype), device="cuda")


class BlockSource:
    """Block callback for Context.solve_streamed over blocks the caller already
    holds: blocks[b] is B_ov's columns for active occupied orbitals
    [n_frozen + b occ_block, n_frozen + (b + 1) occ_block) (the last block may
    be shorter), a torch tensor [n_aux][(i1 - i0) n_virt] on the device or in
    pinned host memory.  A requested block is copied into the library's buffer
    asynchronously (from pinned memory too) on a stream of torch's pool, and
    the stream the library passes waits for the copy, so the copy overlaps the
    library's work on the previous block.  The copy is not issued on the
    library's stream itself: torch would then tie the pinned block's release
    to that stream, which the library destroys with its context."""

    def __init__(self, blocks, n_frozen: int, occ_block: int, n_virt: int):
        self.blocks, self.n_frozen, self.occ_block, self.n_virt = list(blocks), n_frozen, occ_block, n_virt
        self.bytes_copied = 0
        self._stream = None

    def __call__(self, i0: int, i1: int, dst: int, strm: int) -> int:
        import torch
        b, r = divmod(i0 - self.n_frozen, self.occ_block)
        src = self.blocks[b]
        if r or src.shape[1] != (i1 - i0) * self.n_virt:
            raise ValueError(f"block [{i0}, {i1}) does not match the held block {b} of shape {tuple(src.shape)}")
        if self._stream is None:
            self._stream = torch.cuda.Stream()
        view = device_view(dst, tuple(src.shape))
        with torch.cuda.stream(self._stream):
            view.copy_(src, non_blocking=True)
        done = torch.cuda.Event()
        done.record(self._stream)
        torch.cuda.ExternalStream(strm).wait_event(done)
        self.bytes_copied += src.numel() * src.element_size()
        return 0


def status_string(st: int) -> str:
    return load().ltgw_status_string(st).decode()


def gl_grid(n: int, omega0: float = 0.5):
    om, wt = np.zeros(n), np.zeros(n)
    st = load().ltgw_gl_grid(n, omega0, om.ctypes.data, wt.ctypes.data)
    if st:
        raise LtgwError(st, status_string(st))
    return om, wt


def cosine_grid(n_tau: int, dmin: float, dmax: float, omegas, ridge: float = 1e-14):
    """ltgw_cosine_grid: (tau [n_tau], gamma [n_omega][n_tau], max scaled error, amplification)."""
    om = np.ascontiguousarray(omegas, dtype=np.float64)
    tau, gam, err, amp = np.zeros(n_tau), np.zeros((len(om), n_tau)), ctypes.c_double(), ctypes.c_double()
    st = load().ltgw_cosine_grid(n_tau, dmin, dmax, len(om), om.ctypes.data, ridge, tau.ctypes.data,
                                 gam.ctypes.data, ctypes.byref(err), ctypes.byref(amp))
    if st != 0:
        raise RuntimeError(f"ltgw_cosine_grid failed ({st})")
    return tau, gam, err.value, amp.value


def laplace_grid(n_tau: int, a: float, b: float):
    x, w, e = np.zeros(n_tau), np.zeros(n_tau), ctypes.c_double()
    st = load().ltgw_laplace_grid(n_tau, a, b, x.ctypes.data, w.ctypes.data, ctypes.byref(e))
    if st:
        raise LtgwError(st, status_string(st))
    return x, w, e.value


class Context:
    """One ltgw_ctx on a CUDA device (ltgw_create / ltgw_destroy)."""

    def __init__(self, device: int = 0):
        self._lib = load()
        h = ctypes.c_void_p()
        st = self._lib.ltgw_create(ctypes.byref(h), device)
        if st:
            raise LtgwError(st, f"ltgw_create failed: {status_string(st)}")
        self.handle = h
        self.device = device

    def close(self):
        if getattr(self, "handle", None):
            self._lib.ltgw_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int, allow=()):
        if st and st not in allow:
            raise LtgwError(st, self._lib.ltgw_last_error(self.handle).decode())
        return st

    def set_timing(self, on: bool):
        self._check(self._lib.ltgw_set_timing(self.handle, int(bool(on))))

    def set_autotune(self, on: bool):
        self._check(self._lib.ltgw_set_autotune(self.handle, int(bool(on))))

    def workspace_bytes(self) -> int:
        return int(self._lib.ltgw_workspace_bytes(self.handle))

    def trim(self):
        self._check(self._lib.ltgw_trim(self.handle))

    def stats(self) -> dict:
        s = Stats()
        self._check(self._lib.ltgw_get_stats(self.handle, ctypes.byref(s)))
        return s.as_dict()

    def solve(self, params: Params, eps, B_ov, B_tgt, targets, shift, sigma_out, e_qp_out,
              status_out, tau_x=None, tau_w=None, stream=None, allow_no_converge=True) -> int:
        """ltgw_solve on caller-provided buffers (numpy = host, torch CUDA = device)."""
        n_tgt = int(targets.shape[0])
        st = self._lib.ltgw_solve(self.handle, ctypes.byref(params), _ptr(eps), _ptr(B_ov), _ptr(B_tgt),
                                  _ptr(targets), n_tgt, _ptr(shift), _ptr(tau_x), _ptr(tau_w),
                                  _ptr(sigma_out), _ptr(e_qp_out), _ptr(status_out), _stream_ptr(stream))
        return self._check(st, allow=(LTGW_ERR_NO_CONVERGE,) if allow_no_converge else ())

    def solve_ev(self, params: Params, eps, B_ov, B_tgt, targets, shift, sigma_out, e_qp_out, status_out,
                 n_cycles: int = 5, gap_tol: float = 0.0, tau_x=None, tau_w=None, stream=None,
                 allow_no_converge=True) -> int:
        """ltgw_solve_ev (evGW); returns the number of cycles run after G0W0."""
        done = ctypes.c_int()
        st = self._lib.ltgw_solve_ev(self.handle, ctypes.byref(params), _ptr(eps), _ptr(B_ov), _ptr(B_tgt),
                                     _ptr(targets), int(targets.shape[0]), _ptr(shift), _ptr(tau_x), _ptr(tau_w),
                                     n_cycles, gap_tol, _ptr(sigma_out), _ptr(e_qp_out), _ptr(status_out),
                                     ctypes.byref(done), _stream_ptr(stream))
        self._check(st, allow=(LTGW_ERR_NO_CONVERGE,) if allow_no_converge else ())
        return done.value

    def solve_streamed(self, params: Params, eps, fill, occ_block: int, B_tgt, targets, shift, sigma_out,
                       e_qp_out, status_out, tau_x=None, tau_w=None, stream=None, allow_no_converge=True) -> int:
        """ltgw_solve_streamed; fill(i0, i1, dst_ptr, stream_ptr) writes the occupied block
        [i0, i1) into the device buffer at dst_ptr and returns 0."""
        errors = []

        def _cb(user, i0, i1, dst, strm):
            try:
                return int(fill(i0, i1, dst, strm) or 0)
            except Exception as ex:  # reported through the status, re-raised below
                errors.append(ex)
                return 1

        cb = BLOCK_FN(_cb)
        st = self._lib.ltgw_solve_streamed(self.handle, ctypes.byref(params), _ptr(eps), cb, None, occ_block,
                                           _ptr(B_tgt), _ptr(targets), int(targets.shape[0]), _ptr(shift),
                                           _ptr(tau_x), _ptr(tau_w), _ptr(sigma_out), _ptr(e_qp_out),
                                           _ptr(status_out), _stream_ptr(stream))
        if errors:
            raise errors[0]
        return self._check(st, allow=(LTGW_ERR_NO_CONVERGE,) if allow_no_converge else ())

    def naf_basis(self, B, n_pairs: int, ld: int, thresh: float, Ut, lam, stream=None, mixed: bool = False) -> int:
        k = ctypes.c_int()
        fn = self._lib.ltgw_naf_basis_mixed if mixed else self._lib.ltgw_naf_basis
        st = fn(self.handle, int(B.shape[0]), n_pairs, _ptr(B), ld, thresh, _ptr(Ut), _ptr(lam), ctypes.byref(k),
                _stream_ptr(stream))
        self._check(st)
        return k.value

    def polarizability(self, Bt, delta, omegas: np.ndarray, Pi, spin: int = 2, x=None, w=None, stream=None):
        N, n_pairs = int(Bt.shape[0]), int(Bt.shape[1])
        om = np.ascontiguousarray(omegas, dtype=np.float64)
        n_tau = 0 if x is None else len(x)
        xx = None if x is None else np.ascontiguousarray(x, dtype=np.float64)
        ww = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
        st = self._lib.ltgw_polarizability(self.handle, N, n_pairs, _ptr(Bt), _ptr(delta), len(om), _ptr(om),
                                           n_tau, _ptr(xx), _ptr(ww), spin, _ptr(Pi), _stream_ptr(stream))
        self._check(st)

    def polarizability_mixed(self, Bt, delta, omegas: np.ndarray, Pi, spin: int = 2, x=None, w=None,
                             stream=None, fp8: bool = False):
        """Split-BF16 form (ltgw_polarizability_mixed), or with fp8 the FP8 E4M3
        form (ltgw_polarizability_fp8)."""
        N, n_pairs = int(Bt.shape[0]), int(Bt.shape[1])
        om = np.ascontiguousarray(omegas, dtype=np.float64)
        n_tau = 0 if x is None else len(x)
        xx = None if x is None else np.ascontiguousarray(x, dtype=np.float64)
        ww = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
        fn = self._lib.ltgw_polarizability_fp8 if fp8 else self._lib.ltgw_polarizability_mixed
        st = fn(self.handle, N, n_pairs, _ptr(Bt), _ptr(delta), len(om), _ptr(om), n_tau, _ptr(xx), _ptr(ww), spin,
                _ptr(Pi), _stream_ptr(stream))
        self._check(st)

    def polarizability_tau(self, Bt, delta, omegas: np.ndarray, tau, gamma, Pi, spin: int = 2,
                           precision: int = 0, stream=None):
        """Imaginary-time form (ltgw_polarizability_tau): tau [n_tau], gamma [n_omega][n_tau] on the host."""
        N, n_pairs = int(Bt.shape[0]), int(Bt.shape[1])
        om = np.ascontiguousarray(omegas, dtype=np.float64)
        tt = np.ascontiguousarray(tau, dtype=np.float64)
        gg = np.ascontiguousarray(gamma, dtype=np.float64)
        assert gg.shape == (len(om), len(tt))
        st = self._lib.ltgw_polarizability_tau(self.handle, N, n_pairs, _ptr(Bt), _ptr(delta), len(om), _ptr(om),
                                               len(tt), _ptr(tt), _ptr(gg), spin, precision, _ptr(Pi),
                                               _stream_ptr(stream))
        self._check(st)

    def polarizability_fp8(self, Bt, delta, omegas: np.ndarray, Pi, spin: int = 2, x=None, w=None, stream=None):
        self.polarizability_mixed(Bt, delta, omegas, Pi, spin, x, w, stream, fp8=True)

    def polarizability_emulated(self, Bt, delta, omegas: np.ndarray, Pi, spin: int = 2, x=None, w=None,
                                n_slices: int = 6, stream=None):
        """FP64-accurate form from integer slices on the tensor cores (ltgw_polarizability_emulated)."""
        N, n_pairs = int(Bt.shape[0]), int(Bt.shape[1])
        om = np.ascontiguousarray(omegas, dtype=np.float64)
        n_tau = 0 if x is None else len(x)
        xx = None if x is None else np.ascontiguousarray(x, dtype=np.float64)
        ww = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
        st = self._lib.ltgw_polarizability_emulated(self.handle, N, n_pairs, _ptr(Bt), _ptr(delta), len(om),
                                                    _ptr(om), n_tau, _ptr(xx), _ptr(ww), spin, n_slices, _ptr(Pi),
                                                    _stream_ptr(stream))
        self._check(st)

    def gemm_emulated(self, A, B, C, n_slices: int = 6, sym: bool = False, stream=None):
        """ltgw_gemm_emulated: C = A B^T (torch CUDA FP64, rows with unit column
        stride, any row stride) from integer slices; sym: B is A (pass None) and
        C is symmetric."""
        m, k = int(A.shape[0]), int(A.shape[1])
        n = m if sym else int(B.shape[0])
        for t in (A, C) if sym else (A, B, C):
            if t.dim() != 2 or (t.shape[1] > 1 and t.stride(1) != 1):
                raise ValueError("gemm_emulated needs 2-D tensors with unit column stride")
        st = self._lib.ltgw_gemm_emulated(self.handle, m, n, k, A.data_ptr(), A.stride(0),
                                          None if sym else B.data_ptr(), k if sym else B.stride(0), C.data_ptr(),
                                          C.stride(0), int(bool(sym)), n_slices, _stream_ptr(stream))
        self._check(st)

    def screen(self, Pi, C, stream=None):
        n_omega, N = int(Pi.shape[0]), int(Pi.shape[1])
        self._check(self._lib.ltgw_screen(self.handle, N, n_omega, _ptr(Pi), _ptr(C), _stream_ptr(stream)))


class Server:
    """ltgw_server: continuous admission of solves onto worker slots."""

    def __init__(self, device: int = 0, n_slots: int = 4, hbm_budget_bytes: int = 64 << 30):
        self._lib = load()
        h = ctypes.c_void_p()
        st = self._lib.ltgw_server_create(ctypes.byref(h), device, n_slots, hbm_budget_bytes)
        if st:
            raise LtgwError(st, f"ltgw_server_create failed: {status_string(st)}")
        self.handle = h
        self._keep = {}

    def submit(self, params: Params, eps, B_ov, B_tgt, targets, shift, sigma_out, e_qp_out, status_out,
               tau_x=None, tau_w=None) -> int:
        req = Request(params, _ptr(eps), _ptr(B_ov), _ptr(B_tgt), _ptr(targets), int(targets.shape[0]),
                      _ptr(shift), _ptr(tau_x), _ptr(tau_w), _ptr(sigma_out), _ptr(e_qp_out), _ptr(status_out))
        t = ctypes.c_uint64()
        st = self._lib.ltgw_server_submit(self.handle, ctypes.byref(req), ctypes.byref(t))
        if st:
            raise LtgwError(st, status_string(st))
        # the server reads the buffers later: keep them alive until polled
        self._keep[t.value] = (eps, B_ov, B_tgt, targets, shift, tau_x, tau_w, sigma_out, e_qp_out, status_out)
        return t.value

    def poll(self, max_out: int = 256):
        buf = (Completion * max_out)()
        n = self._lib.ltgw_server_poll(self.handle, buf, max_out)
        out = []
        for i in range(n):
            c = buf[i]
            self._keep.pop(c.ticket, None)
            out.append({"ticket": c.ticket, "status": c.status, "queue_ms": c.queue_ms,
                        "service_ms": c.service_ms, "latency_ms": c.latency_ms, "start_ms": c.start_ms,
                        "end_ms": c.end_ms, "message": c.message.decode()})
        return out

    def wait_all(self, timeout_s: float = 600.0):
        st = self._lib.ltgw_server_wait_all(self.handle, timeout_s)
        if st:
            raise LtgwError(st, status_string(st))

    def close(self):
        if getattr(self, "handle", None):
            self._lib.ltgw_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def request_footprint(params: Params, n_tgt: int) -> int:
    return int(load().ltgw_request_footprint(ctypes.byref(params), n_tgt))


def screen_static(Pi, C, stream=None) -> int:
    """ltgw_screen_static: the screening step with library-held scratch (no
    allocation); returns the status code."""
    n_omega, N = int(Pi.shape[0]), int(Pi.shape[1])
    return load().ltgw_screen_static(N, n_omega, _ptr(Pi), _ptr(C), _stream_ptr(stream))


def make_params(n_occ, n_virt, n_aux, n_frozen=0, n_omega=32, n_tau=8, omega0=0.5, naf_thresh=-1.0,
                spin=2, use_laplace=False, precision=LTGW_FP64) -> Params:
    """use_laplace: False / 0 direct (Eq. Pi), True / 1 Eq. LT's moments, 2 imaginary time."""
    return Params(n_occ, n_virt, n_frozen, n_aux, n_omega, n_tau if use_laplace else 0, omega0,
                  naf_thresh, spin, int(use_laplace), precision, 0)


def solve_problem(ctx: Context, prob, n_omega=32, n_tau=8, naf_thresh=-1.0, use_laplace=False, spin=2,
                  omega0=0.5, tau=None, device_arrays=None, stream=None, precision=LTGW_FP64):
    """Solve a synthetic ``Problem`` (host numpy arrays) and return
    (sigma [T][n_omega] complex, e_qp [T], status [T]).  ``device_arrays``,
    if given, is a dict of torch CUDA tensors used instead of the host inputs."""
    p = make_params(prob.n_occ, prob.n_virt, prob.n_aux, prob.n_frozen, n_omega, n_tau, omega0, naf_thresh,
                    spin, use_laplace, precision)
    T = len(prob.targets)
    sig = np.zeros((T, n_omega, 2))
    e = np.zeros(T)
    st = np.zeros(T, dtype=np.int32)
    src = device_arrays or {}
    tx, tw = (None, None) if tau is None else (np.ascontiguousarray(tau[0]), np.ascontiguousarray(tau[1]))
    ctx.solve(p, src.get("eps", prob.eps), src.get("B_ov", prob.B_ov), src.get("B_tgt", prob.B_tgt),
              src.get("targets", np.ascontiguousarray(prob.targets, dtype=np.int32)), src.get("shift", prob.shift),
              sig, e, st, tau_x=tx, tau_w=tw, stream=stream)
    return sig[..., 0] + 1j * sig[..., 1], e, st
