"""Python binding of the C ABI in ``include/nrx.h`` (ctypes; argument
marshalling only).  Every step of both receivers runs in the CUDA kernels of
``libnrx.so``; there is no CPU fallback, and loading fails loudly when the
library has not been built.

Device buffers are torch tensors (torch supplies device memory and streams).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

# The library the binding loads: libnrx.so, or another build of the same
# sources named by NRX_LIBRARY (the bounds-checked libnrx_debug.so).
_LIB_PATH = os.environ.get("NRX_LIBRARY") or os.path.join(os.path.dirname(os.path.abspath(__file__)), "libnrx.so")

NRX_OK, NRX_EINVAL, NRX_ENOMEM, NRX_ECUDA, NRX_ETIMEDOUT, NRX_EUNSUPPORTED = range(6)
NRX_FP32, NRX_BF16, NRX_FP16, NRX_FP8 = 0, 1, 2, 3
PRECISIONS = {"fp32": NRX_FP32, "bf16": NRX_BF16, "fp16": NRX_FP16, "fp8": NRX_FP8}

EXPORTED = (
    "nrx_create", "nrx_destroy", "nrx_llr_count", "nrx_detect_batch", "nrx_detect", "lmmse_detect_batch",
    "lmmse_detect", "nrx_detect_batch_host", "nrx_copy_state", "nrx_get_net", "nrx_last_launch_count",
    "nrx_last_error", "nrx_status_string", "nrx_profile", "nrx_profile_read", "nrx_detect_noalloc",
    "nrx_check", "nrx_dmrs_gold", "nrx_expire_wait", "nrx_detect_batch_host_async", "nrx_host_drain",
    "lmmse_fp64_count", "nrx_debug_counters",
)
KERNEL_KINDS = 5


class nrx_slot_cfg(ctypes.Structure):
    _fields_ = [
        ("num_prb", ctypes.c_int32),
        ("num_users", ctypes.c_int32),
        ("num_dmrs_symbols", ctypes.c_int32),
        ("dmrs_symbols", ctypes.c_int32 * 2),
        ("iterations", ctypes.c_int32),
        ("noise_var", ctypes.c_float),
        ("dmrs_seq", ctypes.c_void_p),
    ]


class NrxError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_status_name(status)}: {msg}")
        self.status = status


_lib = None


def load() -> ctypes.CDLL:
    """Load ``libnrx.so`` (built by ``paper_2409_02912_b300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"{_LIB_PATH} is missing: build the CUDA library first "
                          "(python -m paper_2409_02912_b300.build)")
    lib = ctypes.CDLL(_LIB_PATH)
    P, I32, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_size_t
    CFG = ctypes.POINTER(nrx_slot_cfg)
    lib.nrx_create.argtypes = [P, SZ, I32, I32, I32, I32, ctypes.c_int, ctypes.POINTER(P)]
    lib.nrx_create.restype = ctypes.c_int
    lib.nrx_destroy.argtypes = [P]
    lib.nrx_destroy.restype = None
    lib.nrx_llr_count.argtypes = [CFG, P]
    lib.nrx_llr_count.restype = SZ
    for name in ("nrx_detect_batch", "lmmse_detect_batch", "nrx_detect_batch_host"):
        f = getattr(lib, name)
        f.argtypes = [P, I32, P, CFG, P, P, P]
        f.restype = ctypes.c_int
    for name in ("nrx_detect", "lmmse_detect"):
        f = getattr(lib, name)
        f.argtypes = [P, P, CFG, P, P, P]
        f.restype = ctypes.c_int
    lib.nrx_copy_state.argtypes = [P, I32, P, P]
    lib.nrx_copy_state.restype = ctypes.c_int
    lib.nrx_get_net.argtypes = [P] + [ctypes.POINTER(I32)] * 5
    lib.nrx_get_net.restype = ctypes.c_int
    lib.nrx_last_launch_count.argtypes = [P]
    lib.nrx_last_launch_count.restype = I32
    lib.nrx_last_error.argtypes = [P]
    lib.nrx_last_error.restype = ctypes.c_char_p
    lib.nrx_profile.argtypes = [P, I32]
    lib.nrx_profile.restype = ctypes.c_int
    lib.nrx_profile_read.argtypes = [P, I32, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_int64), I32]
    lib.nrx_profile_read.restype = ctypes.c_int
    lib.nrx_check.argtypes = [P, P]
    lib.nrx_check.restype = ctypes.c_int
    lib.nrx_expire_wait.argtypes = [P, I32, P]
    lib.nrx_detect_batch_host_async.argtypes = [P, I32, P, CFG, P, P]
    lib.nrx_detect_batch_host_async.restype = ctypes.c_int
    lib.nrx_host_drain.argtypes = [P]
    lib.nrx_host_drain.restype = ctypes.c_int
    lib.nrx_expire_wait.restype = ctypes.c_int
    lib.nrx_detect_noalloc.argtypes = [P, P, P, CFG, P, P, P]
    lib.nrx_detect_noalloc.restype = ctypes.c_int
    lib.nrx_dmrs_gold.argtypes = [I32, P, I32, I32, I32, I32, P, P, P]
    lib.nrx_dmrs_gold.restype = ctypes.c_int
    lib.nrx_debug_counters.argtypes = [ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(I32),
                                       ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64), I32]
    lib.nrx_debug_counters.restype = ctypes.c_int
    lib.lmmse_fp64_count.argtypes = [P, ctypes.POINTER(ctypes.c_int64), I32, P]
    lib.lmmse_fp64_count.restype = ctypes.c_int
    lib.nrx_status_string.argtypes = [ctypes.c_int]
    lib.nrx_status_string.restype = ctypes.c_char_p
    _lib = lib
    return lib


def debug_counters(reset: bool = False) -> dict:
    """Bounds-checked build only: {"violations", "site", "index", "extent"} of
    the indices found outside their arrays since the last reset (see nrx.h)."""
    n, site, idx, ext = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
    st = load().nrx_debug_counters(ctypes.byref(n), ctypes.byref(site), ctypes.byref(idx), ctypes.byref(ext),
                                   int(bool(reset)))
    if st != NRX_OK:
        raise NrxError(st, "nrx_debug_counters")
    return {"violations": n.value, "site": site.value, "index": idx.value, "extent": ext.value}


def _status_name(s: int) -> str:
    try:
        return load().nrx_status_string(s).decode()
    except Exception:  # library not loadable: plain number
        return str(s)


def make_cfgs(n_slots: int, num_prb: int, num_users: int, dmrs_symbols: Sequence[int],
              dmrs_ptrs: Sequence[int], noise_vars: Sequence[float], iterations: int = 0):
    """Array of ``nrx_slot_cfg`` (one per slot)."""
    arr = (nrx_slot_cfg * n_slots)()
    for i in range(n_slots):
        c = arr[i]
        c.num_prb = num_prb
        c.num_users = num_users
        c.num_dmrs_symbols = len(dmrs_symbols)
        c.dmrs_symbols[0] = dmrs_symbols[0]
        c.dmrs_symbols[1] = dmrs_symbols[-1]
        c.iterations = iterations
        c.noise_var = float(noise_vars[i])
        c.dmrs_seq = int(dmrs_ptrs[i])
    return arr


def _bits_array(bits) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(bits, dtype=np.int32))


def _stream_ptr(stream) -> Optional[int]:
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


class Receiver:
    """A context (``nrx_create``) plus the detect calls on torch tensors."""

    def __init__(self, weights_blob: bytes, num_rx_ant: int, max_users: int, max_prb: int,
                 max_slots: int = 1, precision: str = "fp32"):
        lib = load()
        self._lib = lib
        ctx = ctypes.c_void_p()
        self._blob = ctypes.create_string_buffer(weights_blob, len(weights_blob))
        st = lib.nrx_create(self._blob, len(weights_blob), num_rx_ant, max_users, max_prb, max_slots,
                            PRECISIONS[precision], ctypes.byref(ctx))
        if st != NRX_OK:
            raise NrxError(st, "nrx_create failed")
        self.ctx = ctx
        self.precision = precision
        vals = [ctypes.c_int32() for _ in range(5)]
        lib.nrx_get_net(ctx, *[ctypes.byref(v) for v in vals])
        self.num_rx_ant, self.channels, self.res_blocks, self.iterations, self.m_max = [v.value for v in vals]

    def close(self):
        if getattr(self, "ctx", None):
            self._lib.nrx_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int, what: str):
        if st != NRX_OK:
            raise NrxError(st, f"{what}: {self._lib.nrx_last_error(self.ctx).decode()}")

    def last_launch_count(self) -> int:
        return int(self._lib.nrx_last_launch_count(self.ctx))

    def nrx_check(self, stream=None):
        """Synchronise and raise on a device-side failure (e.g. NRX_ETIMEDOUT)."""
        self._check(self._lib.nrx_check(self.ctx, _stream_ptr(stream)), "nrx_check")

    def nrx_expire_wait(self, limit_us: int, stream=None):
        """Enqueue a bounded device wait that runs out (see nrx.h); the next
        ``nrx_check`` raises NRX_ETIMEDOUT."""
        self._check(self._lib.nrx_expire_wait(self.ctx, int(limit_us), _stream_ptr(stream)), "nrx_expire_wait")

    def lmmse_fp64_count(self, reset: bool = False, stream=None) -> int:
        """REs whose LMMSE solve ran in FP64 since creation or the last reset."""
        n = ctypes.c_int64()
        self._check(self._lib.lmmse_fp64_count(self.ctx, ctypes.byref(n), int(bool(reset)), _stream_ptr(stream)),
                    "lmmse_fp64_count")
        return int(n.value)

    def nrx_profile(self, enable: bool):
        self._check(self._lib.nrx_profile(self.ctx, int(bool(enable))), "nrx_profile")

    def nrx_profile_read(self, reset: bool = False) -> dict:
        """{kernel kind: (total_ms, launches)} accumulated while profiling."""
        out = {}
        for k in range(KERNEL_KINDS):
            name, ms, n = ctypes.c_char_p(), ctypes.c_double(), ctypes.c_int64()
            st = self._lib.nrx_profile_read(self.ctx, k, ctypes.byref(name), ctypes.byref(ms), ctypes.byref(n),
                                            int(reset and k == KERNEL_KINDS - 1))
            self._check(st, "nrx_profile_read")
            out[name.value.decode()] = (ms.value, n.value)
        return out

    def llr_count(self, cfg: nrx_slot_cfg, bits_row) -> int:
        b = _bits_array(bits_row)
        return int(self._lib.nrx_llr_count(ctypes.byref(cfg), b.ctypes.data))

    def _device_call(self, fn, y, dmrs, dmrs_symbols, bits, noise_vars, iterations, out, stream):
        import torch
        assert y.is_cuda and y.dtype == torch.complex64 and y.is_contiguous()
        n, B, T, S = y.shape
        bits = _bits_array(bits).reshape(n, -1)
        U = bits.shape[1]
        dmrs = dmrs.contiguous()
        assert dmrs.is_cuda and dmrs.dtype == torch.complex64 and dmrs.shape[0] == n
        ptrs = [dmrs[i].data_ptr() for i in range(n)]
        nv = noise_vars if noise_vars is not None else [1.0] * n
        cfgs = make_cfgs(n, S // 12, U, dmrs_symbols, ptrs, nv, iterations)
        total = sum(self.llr_count(cfgs[i], bits[i]) for i in range(n))
        if out is None:
            out = torch.empty(total, dtype=torch.float32, device=y.device)
        assert out.numel() >= total and out.dtype == torch.float32 and out.is_cuda
        st = fn(self.ctx, n, y.data_ptr(), cfgs, bits.ctypes.data, out.data_ptr(), _stream_ptr(stream))
        self._check(st, fn.__name__)
        return out

    def nrx_detect_batch(self, y, dmrs, dmrs_symbols, bits, iterations: int = 0, out=None, stream=None,
                         noise_vars=None):
        """y: complex64 cuda [n, B, 14, S]; dmrs: complex64 cuda [n, n_dmrs, S/2];
        bits: [n][U] modulation orders.  Returns the packed float32 LLRs."""
        return self._device_call(self._lib.nrx_detect_batch, y, dmrs, dmrs_symbols, bits, noise_vars,
                                 iterations, out, stream)

    def lmmse_detect_batch(self, y, dmrs, dmrs_symbols, bits, noise_vars, out=None, stream=None):
        return self._device_call(self._lib.lmmse_detect_batch, y, dmrs, dmrs_symbols, bits, noise_vars,
                                 0, out, stream)

    def nrx_detect_batch_host(self, y_host, dmrs_host, dmrs_symbols, bits, llr_host, iterations: int = 0,
                              stream=None):
        """Host-buffer variant: y_host complex64 [n, B, 14, S] and dmrs_host
        complex64 [n, n_dmrs, S/2] (numpy arrays or pinned CPU tensors),
        llr_host float32 output; synchronises before returning."""
        yp, dp, lp = (_host_ptr(a) for a in (y_host, dmrs_host, llr_host))
        n, B, T, S = tuple(y_host.shape)
        bits = _bits_array(bits).reshape(n, -1)
        U = bits.shape[1]
        per = len(dmrs_symbols) * (S // 2) * 8
        cfgs = make_cfgs(n, S // 12, U, dmrs_symbols, [dp + i * per for i in range(n)], [1.0] * n, iterations)
        st = self._lib.nrx_detect_batch_host(self.ctx, n, yp, cfgs, bits.ctypes.data, lp, _stream_ptr(stream))
        self._check(st, "nrx_detect_batch_host")
        return llr_host

    def nrx_detect_batch_host_async(self, y_host, dmrs_host, dmrs_symbols, bits, llr_host, iterations: int = 0):
        """Pipelined host-buffer call (see nrx.h): returns at once; y_host,
        dmrs_host and llr_host must stay alive and unchanged until
        ``nrx_host_drain``."""
        yp, dp, lp = (_host_ptr(a) for a in (y_host, dmrs_host, llr_host))
        n, B, T, S = tuple(y_host.shape)
        bits = _bits_array(bits).reshape(n, -1)
        U = bits.shape[1]
        per = len(dmrs_symbols) * (S // 2) * 8
        cfgs = make_cfgs(n, S // 12, U, dmrs_symbols, [dp + i * per for i in range(n)], [1.0] * n, iterations)
        self._check(self._lib.nrx_detect_batch_host_async(self.ctx, n, yp, cfgs, bits.ctypes.data, lp),
                    "nrx_detect_batch_host_async")
        return llr_host

    def nrx_host_drain(self):
        """Wait for every pipelined call; raise on a device-side failure."""
        self._check(self._lib.nrx_host_drain(self.ctx), "nrx_host_drain")

    def nrx_copy_state(self, slot: int, num_users: int, S: int, stream=None):
        import torch
        out = torch.empty((num_users, 14, S, self.channels), dtype=torch.float32, device="cuda")
        st = self._lib.nrx_copy_state(self.ctx, slot, out.data_ptr(), _stream_ptr(stream))
        self._check(st, "nrx_copy_state")
        return out


def _host_ptr(a) -> int:
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    assert not a.is_cuda and a.is_contiguous()
    return a.data_ptr()


def nrx_detect_noalloc(weights_blob: bytes, weights_dev, y, dmrs, dmrs_symbols, bits, iterations: int = 0,
                       out=None, stream=None):
    """One slot through the allocation-free entry point.  weights_dev: float32
    cuda tensor holding the blob's payload (bytes 32..); y: complex64 cuda
    [B, 14, S]; dmrs: complex64 cuda [n_dmrs, S/2]; bits: [U]."""
    import torch
    lib = load()
    hdr = ctypes.create_string_buffer(weights_blob[:32], 32)
    B, T, S = y.shape
    b = _bits_array(bits).reshape(-1)
    cfg = make_cfgs(1, S // 12, b.size, dmrs_symbols, [dmrs.data_ptr()], [1.0], iterations)
    n = int(lib.nrx_llr_count(cfg, b.ctypes.data))
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=y.device)
    st = lib.nrx_detect_noalloc(hdr, weights_dev.data_ptr(), y.data_ptr(), cfg, b.ctypes.data, out.data_ptr(),
                                _stream_ptr(stream))
    if st != NRX_OK:
        raise NrxError(st, "nrx_detect_noalloc")
    return out


def nrx_dmrs_gold(slot_numbers, n_id: int, num_prb: int, dmrs_symbols, n_scid: int = 0, out=None, stream=None):
    """TS 38.211 DMRS base sequences on the device: complex64 cuda
    [n_slots, n_dmrs, 6 num_prb] (the ``dmrs`` argument of the detect calls)."""
    import torch
    sn = _bits_array(slot_numbers).reshape(-1)
    ds = _bits_array(dmrs_symbols).reshape(-1)
    if out is None:
        out = torch.empty((sn.size, ds.size, 6 * num_prb), dtype=torch.complex64, device="cuda")
    st = load().nrx_dmrs_gold(sn.size, sn.ctypes.data, n_id, n_scid, num_prb, ds.size, ds.ctypes.data,
                              out.data_ptr(), _stream_ptr(stream))
    if st != NRX_OK:
        raise NrxError(st, "nrx_dmrs_gold")
    return out
