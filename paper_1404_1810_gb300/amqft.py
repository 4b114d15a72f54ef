"""Thin Python binding of libamqft.so: the C-ABI entry points under the same
names, plus a small torch convenience layer (argument marshalling only --
every step of the transform runs in the library's CUDA kernels).

There is no fallback: if the compiled library is missing the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

AMQFT_C64, AMQFT_CBF16, AMQFT_CF16, AMQFT_CI16 = 0, 1, 2, 3
ERRORS = {
    -1: "AMQFT_ERR_N", -2: "AMQFT_ERR_VARIANT", -3: "AMQFT_ERR_DTYPE", -4: "AMQFT_ERR_ALIGN",
    -5: "AMQFT_ERR_INPLACE", -6: "AMQFT_ERR_CUDA", -7: "AMQFT_ERR_DEVICE", -8: "AMQFT_ERR_ARG",
    -9: "AMQFT_ERR_NOMEM",
}
LIB_PATH = _build.LIB

_lock = threading.Lock()
_lib = None


class AmqftError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {ERRORS.get(code, code)}: {msg}")
        self.code = code


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libamqft.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libamqft.so not found at {p}: run paper_1404_1810_gb300.build.build() first")
        lib = ctypes.CDLL(p)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
        lib.amqft_plan.argtypes = [ctypes.POINTER(vp), i32, i32, i64, i32]
        lib.amqft_plan.restype = i32
        lib.amqft_exec_fwd.argtypes = [vp, vp, vp, vp, vp]
        lib.amqft_exec_fwd.restype = i32
        lib.amqft_exec_inv.argtypes = [vp, vp, vp, vp, vp, vp]
        lib.amqft_exec_inv.restype = i32
        lib.amqft_destroy.argtypes = [vp]
        lib.amqft_destroy.restype = i32
        lib.amqft_last_error.restype = ctypes.c_char_p
        lib.amqft_version.restype = ctypes.c_char_p
        lib.amqft_plan_ragged.argtypes = [ctypes.POINTER(vp), i32, i32, i32, i64, i64]
        lib.amqft_plan_ragged.restype = i32
        lib.amqft_exec_ragged.argtypes = [vp, i64, vp, vp, vp, vp, i32, vp]
        lib.amqft_exec_ragged.restype = i32
        lib.amqft_ragged_tune.argtypes = [vp, i32, i32]
        lib.amqft_ragged_tune.restype = i32
        lib.amqft_ragged_skipped.argtypes = [vp, ctypes.POINTER(i64)]
        lib.amqft_ragged_skipped.restype = i32
        lib.amqft_exec_rdft.argtypes = [vp, vp, vp, vp]
        lib.amqft_exec_rdft.restype = i32
        lib.amqft_exec_irdft.argtypes = [vp, vp, vp, vp]
        lib.amqft_exec_irdft.restype = i32
        lib.amqft_exec_dct_dst.argtypes = [vp, i64, vp, vp, vp, vp, vp]
        lib.amqft_exec_dct_dst.restype = i32
        lib.amqft_exec_host.argtypes = [vp, vp, vp, i32, i64, vp]
        lib.amqft_exec_host.restype = i32
        lib.amqft_exec_static.argtypes = [vp, i64, vp, vp, i32, vp]
        lib.amqft_exec_static.restype = i32
        lib.amqft_plan_info.argtypes = [vp] + [ctypes.POINTER(i32)] * 4
        lib.amqft_plan_info.restype = i32
        lib.amqft_plan_launches.argtypes = [vp]
        lib.amqft_plan_launches.restype = i64
        lib.amqft_plan_set_constants.argtypes = [vp, i32]
        lib.amqft_plan_set_constants.restype = i32
        lib.amqft_plan_get_constants.argtypes = [vp]
        lib.amqft_plan_get_constants.restype = i32
        lib.amqft_debug_bounds.argtypes = [ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_uint64), i32]
        lib.amqft_debug_bounds.restype = i32
        _lib = lib
        return lib


class use_library:
    """Context manager: every binding call inside uses the library at `path`
    (e.g. the bounds-checked build), the previous one again afterwards.
    Plans must not cross the boundary."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        self.saved = load()
        with _lock:
            _lib = None
        return load(self.path)

    def __exit__(self, *exc):
        global _lib
        with _lock:
            _lib = self.saved
        return False


def amqft_debug_bounds(clear: bool = False) -> tuple[bool, int, int]:
    """(checked build?, failures, first failure) of the loaded library."""
    c, f = ctypes.c_int64(0), ctypes.c_uint64(0)
    rc = int(load().amqft_debug_bounds(ctypes.byref(c), ctypes.byref(f), 1 if clear else 0))
    if rc < 0:
        _check(rc, "amqft_debug_bounds")
    return rc == 1, int(c.value), int(f.value)


def _check(rc: int, where: str) -> None:
    if rc != 0:
        raise AmqftError(rc, where, load().amqft_last_error().decode())


# --- the C-ABI entry points, same names, plain integers for pointers ------

def amqft_plan(log2n: int, variant: int, batch: int, dtype: int = AMQFT_C64) -> int:
    h = ctypes.c_void_p()
    _check(load().amqft_plan(ctypes.byref(h), int(log2n), int(variant), int(batch), int(dtype)), "amqft_plan")
    return int(h.value)


def amqft_exec_fwd(plan: int, d_in: int, d_out: int, exp_out: int = 0, stream: int = 0) -> None:
    _check(load().amqft_exec_fwd(plan, d_in, d_out, exp_out or None, stream or None), "amqft_exec_fwd")


def amqft_exec_inv(plan: int, d_in: int, exp_in: int, d_out: int, exp_out: int = 0, stream: int = 0) -> None:
    _check(load().amqft_exec_inv(plan, d_in, exp_in or None, d_out, exp_out or None, stream or None),
           "amqft_exec_inv")


def amqft_exec_static(plan: int, batch: int, d_in: int, d_out: int, inverse: int = 0, stream: int = 0) -> None:
    """Multi-pass transform (2^17..2^20) with the library's fixed device scratch:
    no allocation in the call; calls overlapping in time on one device race."""
    _check(load().amqft_exec_static(plan, int(batch), d_in, d_out, int(inverse), stream or None),
           "amqft_exec_static")


def amqft_exec_rdft(plan: int, d_in: int, d_out: int, stream: int = 0) -> None:
    _check(load().amqft_exec_rdft(plan, d_in, d_out, stream or None), "amqft_exec_rdft")


def amqft_exec_irdft(plan: int, d_in: int, d_out: int, stream: int = 0) -> None:
    _check(load().amqft_exec_irdft(plan, d_in, d_out, stream or None), "amqft_exec_irdft")


def amqft_exec_dct_dst(plan: int, count: int, dct_in: int, dct_out: int, dst_in: int, dst_out: int,
                       stream: int = 0) -> None:
    _check(load().amqft_exec_dct_dst(plan, int(count), dct_in or None, dct_out or None, dst_in or None,
                                     dst_out or None, stream or None), "amqft_exec_dct_dst")


def amqft_exec_host(plan: int, h_in: int, h_out: int, direction: int = 0, chunk: int = 0, stream: int = 0) -> None:
    _check(load().amqft_exec_host(plan, h_in, h_out, int(direction), int(chunk), stream or None), "amqft_exec_host")


def amqft_plan_ragged(max_log2n: int, variant: int, dtype: int, max_count: int, max_points: int) -> int:
    h = ctypes.c_void_p()
    _check(load().amqft_plan_ragged(ctypes.byref(h), int(max_log2n), int(variant), int(dtype), int(max_count),
                                    int(max_points)), "amqft_plan_ragged")
    return int(h.value)


def amqft_exec_ragged(plan: int, count: int, d_offsets: int, d_log2n: int, d_in: int, d_out: int,
                      direction: int = 0, stream: int = 0) -> None:
    _check(load().amqft_exec_ragged(plan, int(count), d_offsets, d_log2n, d_in, d_out, int(direction),
                                    stream or None), "amqft_exec_ragged")


def amqft_ragged_tune(plan: int, knob: int, value: int) -> None:
    _check(load().amqft_ragged_tune(plan, int(knob), int(value)), "amqft_ragged_tune")


def amqft_ragged_skipped(plan: int) -> int:
    v = ctypes.c_int64()
    _check(load().amqft_ragged_skipped(plan, ctypes.byref(v)), "amqft_ragged_skipped")
    return int(v.value)


def amqft_destroy(plan: int) -> None:
    _check(load().amqft_destroy(plan), "amqft_destroy")


def amqft_last_error() -> str:
    return load().amqft_last_error().decode()


def amqft_version() -> str:
    return load().amqft_version().decode()


def amqft_plan_info(plan: int) -> dict:
    vals = [ctypes.c_int() for _ in range(4)]
    _check(load().amqft_plan_info(plan, *[ctypes.byref(v) for v in vals]), "amqft_plan_info")
    return dict(zip(("cluster", "per_cta", "threads", "smem_bytes"), (v.value for v in vals)))


def amqft_plan_launches(plan: int) -> int:
    """Kernels the library has launched for exec calls on this plan so far."""
    n = int(load().amqft_plan_launches(plan))
    if n < 0:
        _check(n, "amqft_plan_launches")
    return n


AMQFT_CONST_TABLE, AMQFT_CONST_FLY = 0, 1


def amqft_plan_set_constants(plan: int, mode: int) -> None:
    """Band-level trig constants from the plan's table (AMQFT_CONST_TABLE) or
    evaluated on the fly in the kernels (AMQFT_CONST_FLY)."""
    _check(load().amqft_plan_set_constants(plan, int(mode)), "amqft_plan_set_constants")


def amqft_plan_get_constants(plan: int) -> int:
    m = int(load().amqft_plan_get_constants(plan))
    if m < 0:
        _check(m, "amqft_plan_get_constants")
    return m


# --- torch convenience layer ------------------------------------------------

def _stream_handle(stream) -> int:
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


_TORCH_16 = {AMQFT_CBF16: "bfloat16", AMQFT_CF16: "float16", AMQFT_CI16: "int16"}


class Plan:
    """Owns one amqft plan.

    complex64 plans: fwd/inv take and return contiguous complex64 CUDA
    tensors of shape (batch, N).  16-bit plans (AMQFT_CBF16, AMQFT_CF16,
    AMQFT_CI16): tensors of shape (batch, N, 2) in bfloat16 / float16 / int16
    (real, imaginary),
    plus one int32 exponent per transform: fwd(x) returns (y, exp_y) and
    inv(x, exp_x) returns (y, exp_y), the values being y * 2^exp_y."""

    def __init__(self, log2n: int, variant: int, batch: int, dtype: int = AMQFT_C64):
        self.log2n, self.variant, self.batch, self.dtype = int(log2n), int(variant), int(batch), int(dtype)
        self.n = 1 << self.log2n
        self.handle = amqft_plan(self.log2n, self.variant, self.batch, self.dtype)

    def info(self) -> dict:
        return amqft_plan_info(self.handle)

    def launches(self) -> int:
        """Kernels launched by this plan's exec calls so far."""
        return amqft_plan_launches(self.handle)

    @property
    def constants(self) -> str:
        """"table" or "fly": where the kernels take the band levels' constants."""
        return "fly" if amqft_plan_get_constants(self.handle) == AMQFT_CONST_FLY else "table"

    @constants.setter
    def constants(self, mode: str) -> None:
        if mode not in ("table", "fly"):
            raise ValueError(f"constants mode {mode!r} is not 'table' or 'fly'")
        amqft_plan_set_constants(self.handle, AMQFT_CONST_FLY if mode == "fly" else AMQFT_CONST_TABLE)

    def _check_tensor(self, t, name):
        import torch

        if self.dtype == AMQFT_C64:
            if t.dtype != torch.complex64 or not t.is_cuda or not t.is_contiguous():
                raise ValueError(f"{name} must be a contiguous complex64 CUDA tensor")
            if t.numel() != self.batch * self.n:
                raise ValueError(f"{name} has {t.numel()} elements, plan needs {self.batch * self.n}")
        else:
            want = getattr(torch, _TORCH_16[self.dtype])
            if t.dtype != want or not t.is_cuda or not t.is_contiguous() or t.shape[-1] != 2:
                raise ValueError(f"{name} must be a contiguous {want} CUDA tensor of shape (..., N, 2)")
            if t.numel() != 2 * self.batch * self.n:
                raise ValueError(f"{name} has {t.numel() // 2} elements, plan needs {self.batch * self.n}")

    def _check_exp(self, e, name):
        import torch

        if e.dtype != torch.int32 or not e.is_cuda or not e.is_contiguous() or e.numel() != self.batch:
            raise ValueError(f"{name} must be a contiguous int32 CUDA tensor of {self.batch} exponents")

    def fwd(self, x, out=None, stream=None, exp_out=None):
        import torch

        self._check_tensor(x, "x")
        if out is None:
            out = torch.empty_like(x)
        self._check_tensor(out, "out")
        if self.dtype == AMQFT_C64:
            amqft_exec_fwd(self.handle, x.data_ptr(), out.data_ptr(), 0, _stream_handle(stream))
            return out
        if exp_out is None:
            exp_out = torch.empty(self.batch, dtype=torch.int32, device=x.device)
        self._check_exp(exp_out, "exp_out")
        amqft_exec_fwd(self.handle, x.data_ptr(), out.data_ptr(), exp_out.data_ptr(), _stream_handle(stream))
        return out, exp_out

    def inv(self, x, out=None, stream=None, exp_in=None, exp_out=None):
        import torch

        self._check_tensor(x, "x")
        if out is None:
            out = torch.empty_like(x)
        self._check_tensor(out, "out")
        if self.dtype == AMQFT_C64:
            if exp_in is not None:
                raise ValueError("exp_in is only used with 16-bit storage")
            amqft_exec_inv(self.handle, x.data_ptr(), 0, out.data_ptr(), 0, _stream_handle(stream))
            return out
        if exp_in is not None:
            self._check_exp(exp_in, "exp_in")
        if exp_out is None:
            exp_out = torch.empty(self.batch, dtype=torch.int32, device=x.device)
        self._check_exp(exp_out, "exp_out")
        amqft_exec_inv(self.handle, x.data_ptr(), exp_in.data_ptr() if exp_in is not None else 0, out.data_ptr(),
                       exp_out.data_ptr(), _stream_handle(stream))
        return out, exp_out

    def rdft(self, x, out=None, stream=None):
        """Harmonics 0 .. N/2 of `batch` real float32 signals (batch, N) -> (batch, N/2 + 1) complex64."""
        import torch

        if self.dtype != AMQFT_C64:
            raise ValueError("rdft needs a complex64 plan")
        if x.dtype != torch.float32 or not x.is_cuda or not x.is_contiguous() or x.numel() != self.batch * self.n:
            raise ValueError(f"x must be a contiguous float32 CUDA tensor of {self.batch} x {self.n}")
        if out is None:
            out = torch.empty((self.batch, self.n // 2 + 1), dtype=torch.complex64, device=x.device)
        if out.dtype != torch.complex64 or not out.is_contiguous() or out.numel() != self.batch * (self.n // 2 + 1):
            raise ValueError("out must be a contiguous complex64 tensor of batch x (N/2 + 1)")
        amqft_exec_rdft(self.handle, x.data_ptr(), out.data_ptr(), _stream_handle(stream))
        return out

    def irdft(self, x, out=None, stream=None):
        """Unnormalised inverse of rdft: (batch, N/2 + 1) complex64 half spectra ->
        (batch, N) float32 signals N * x."""
        import torch

        if self.dtype != AMQFT_C64:
            raise ValueError("irdft needs a complex64 plan")
        h = self.n // 2 + 1
        if x.dtype != torch.complex64 or not x.is_cuda or not x.is_contiguous() or x.numel() != self.batch * h:
            raise ValueError(f"x must be a contiguous complex64 CUDA tensor of {self.batch} x {h}")
        if out is None:
            out = torch.empty((self.batch, self.n), dtype=torch.float32, device=x.device)
        if out.dtype != torch.float32 or not out.is_contiguous() or out.numel() != self.batch * self.n:
            raise ValueError("out must be a contiguous float32 tensor of batch x N")
        amqft_exec_irdft(self.handle, x.data_ptr(), out.data_ptr(), _stream_handle(stream))
        return out

    def dct_dst(self, dct=None, dst=None, dct_out=None, dst_out=None, stream=None):
        """DCT-0 (Eq. qft_0B) of the rows of `dct` (count x (N/2 + 1) float32) and
        DST-0 (Eq. qft_0C) of the rows of `dst` (count x (N/2 - 1), sample n at
        column n - 1), either may be None; returns (dct_out, dst_out)."""
        import torch

        if self.dtype != AMQFT_C64:
            raise ValueError("dct_dst needs a complex64 plan")
        count = None
        for t, w, name in ((dct, self.n // 2 + 1, "dct"), (dst, self.n // 2 - 1, "dst")):
            if t is None:
                continue
            if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous() or t.dim() != 2 or t.shape[1] != w:
                raise ValueError(f"{name} must be a contiguous float32 CUDA tensor of count x {w}")
            if count is not None and t.shape[0] != count:
                raise ValueError("dct and dst differ in count")
            count = t.shape[0]
        if count is None:
            return None, None
        if dct is not None and dct_out is None:
            dct_out = torch.empty_like(dct)
        if dst is not None and dst_out is None:
            dst_out = torch.empty_like(dst)
        ptr = lambda t: t.data_ptr() if t is not None else 0  # noqa: E731
        amqft_exec_dct_dst(self.handle, count, ptr(dct), ptr(dct_out), ptr(dst), ptr(dst_out),
                           _stream_handle(stream))
        return dct_out, dst_out

    def _host(self, x, out, inverse, chunk, stream):
        import torch

        for t, name in ((x, "x"), (out, "out")):
            if t is not None and (t.dtype != torch.complex64 or t.is_cuda or not t.is_contiguous()):
                raise ValueError(f"{name} must be a contiguous complex64 CPU tensor (pinned for overlap)")
        if x.numel() != self.batch * self.n:
            raise ValueError(f"x has {x.numel()} elements, plan needs {self.batch * self.n}")
        if out is None:
            out = torch.empty_like(x, pin_memory=x.is_pinned())
        amqft_exec_host(self.handle, x.data_ptr(), out.data_ptr(), 1 if inverse else 0, chunk,
                        _stream_handle(stream))
        return out

    def fwd_host(self, x, out=None, chunk: int = 0, stream=None):
        """DFT of a host batch into host memory (complete once `stream` is)."""
        return self._host(x, out, False, chunk, stream)

    def inv_host(self, x, out=None, chunk: int = 0, stream=None):
        """Unnormalised inverse of a host batch into host memory."""
        return self._host(x, out, True, chunk, stream)

    def close(self):
        if getattr(self, "handle", 0):
            amqft_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class RaggedPlan:
    """Owns a ragged plan: exec() transforms, in one call, `count` complex64
    transforms of lengths 2^log2n[i] at element offsets offsets[i] of flat
    complex64 CUDA tensors (log2n: uint8, offsets: int64, both on the device)."""

    KNOBS = ("schedule", "order", "small_ctas_per_sm", "cluster_mult")

    def __init__(self, max_log2n: int, variant: int, max_count: int, max_points: int):
        self.max_log2n, self.variant = int(max_log2n), int(variant)
        self.max_count, self.max_points = int(max_count), int(max_points)
        self.handle = amqft_plan_ragged(self.max_log2n, self.variant, AMQFT_C64, self.max_count, self.max_points)
        self.knobs = {"schedule": 1, "order": 0, "small_ctas_per_sm": 1, "cluster_mult": 1}

    def tune(self, **knobs) -> None:
        for k, v in knobs.items():
            amqft_ragged_tune(self.handle, self.KNOBS.index(k), int(v))
            self.knobs[k] = int(v)

    def exec(self, x, log2n, offsets, out=None, inverse: bool = False, stream=None):
        import torch

        for t, dt, name in ((x, torch.complex64, "x"), (log2n, torch.uint8, "log2n"), (offsets, torch.int64, "offsets")):
            if t.dtype != dt or not t.is_cuda or not t.is_contiguous():
                raise ValueError(f"{name} must be a contiguous {dt} CUDA tensor")
        if log2n.numel() != offsets.numel():
            raise ValueError("log2n and offsets differ in length")
        if out is None:
            out = torch.empty_like(x)
        amqft_exec_ragged(self.handle, log2n.numel(), offsets.data_ptr(), log2n.data_ptr(), x.data_ptr(),
                          out.data_ptr(), 1 if inverse else 0, _stream_handle(stream))
        return out

    def launches(self) -> int:
        """Kernels launched by this plan's exec calls so far."""
        return amqft_plan_launches(self.handle)

    def skipped(self) -> int:
        return amqft_ragged_skipped(self.handle)

    def close(self):
        if getattr(self, "handle", 0):
            amqft_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dequantize(values, exps):
    """complex128 tensor of values * 2^exp from 16-bit (batch, N, 2) storage
    and its (batch,) int32 exponents (on the tensors' device)."""
    import torch

    v = values.to(torch.float64)
    scale = torch.pow(torch.tensor(2.0, dtype=torch.float64, device=v.device), exps.to(torch.float64))
    v = v * scale.reshape((-1,) + (1,) * (v.dim() - 1))
    return torch.complex(v[..., 0], v[..., 1])


def fft(x, variant: int = 4, inverse: bool = False):
    """DFT (or unnormalised inverse) over the last axis of a complex64 CUDA tensor."""
    n = x.shape[-1]
    log2n = n.bit_length() - 1
    if n != 1 << log2n:
        raise ValueError("length must be a power of two")
    xc = x.reshape(-1, n).contiguous()
    p = Plan(log2n, variant, xc.shape[0])
    try:
        y = p.inv(xc) if inverse else p.fwd(xc)
    finally:
        p.close()
    return y.reshape(x.shape)
