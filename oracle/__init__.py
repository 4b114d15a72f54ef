"""CPU oracle for the AM-QFT complex DFT.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline legs of ``bench.py`` may import this package.  The product
(``paper_1404_1810_gb300`` and its CUDA library) never imports, links or runs
it, and the two share no code: the oracle is plain C (``amqft_oracle.c`` and
``amqft_rec.inc``) built with gcc into ``oracle/_build/liboracle.so``.

Functions (all take / return numpy float64 or complex128 arrays):

* ``naive_dft(x, sign=-1)`` -- Eq. qft_0A written out, long double sums.
* ``dft_bin(x, k, sign=-1)`` -- one bin of the same definition, O(N).
* ``amqft(x, variant, prec="f64", sign=-1)`` -- the AM-QFT recursion of the
  paper (Sect. 3-6) for one transform or a batch ``(..., N)``.
* ``amqft_batch(x, variant, threads)`` -- OpenMP over the batch (CPU baseline).
* ``tally(variant, log2n, kind)`` -- (sums, multiplications, halvings) the
  recursion performs (Sect. 7 conventions).
* ``sub(kind, variant, log2m, x)`` -- one function of the recursion.
* ``mv_time`` / ``mv_freq`` -- the two phases of M1..M8 (Tab. 5-6).
* ``angles(variant, log2n)`` -- trig-constant angles used (Sect. 7.1).
* ``fault(id)`` -- context manager planting a deliberate mistake.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRCS = [os.path.join(_HERE, "amqft_oracle.c"), os.path.join(_HERE, "amqft_rec.inc")]
_lock = threading.Lock()
_lib = None

PREC = {"f32": 0, "f64": 1, "f80": 2, "ld": 2}
KIND = {"rdft": 0, "dct": 1, "dst": 2, "dct_ot": 3, "dst_ot": 4, "dct_to": 5,
        "dst_to": 6, "dct_oo": 7, "dst_oo": 8}
FAULTS = {"dc_misprint": 1, "dr_sign": 2, "dk_drop": 3, "m4_neighbour": 4,
          "const_index": 5, "dn_sign": 6, "m1_halving": 7}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, IEEE semantics)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(s) for s in _SRCS)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=gnu11", "-ffp-contract=off",
           "-fno-fast-math", "-fopenmp", "-Wall", "-Wno-unused-function",
           "-Wno-maybe-uninitialized", _SRCS[0], "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        llp = ctypes.POINTER(ctypes.c_longlong)
        lib.orc_cdft.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int, llp]
        lib.orc_cdft_batch.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_longlong,
                                       dp, dp, ctypes.c_int, ctypes.c_int]
        lib.orc_sub.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, llp]
        lib.orc_mv_time.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp]
        lib.orc_mv_freq.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp]
        lib.orc_angles.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_ubyte)]
        lib.orc_naive_dft.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int]
        lib.orc_dft_bin.argtypes = [ctypes.c_int, dp, ctypes.c_longlong, dp, ctypes.c_int]
        lib.orc_set_fault.argtypes = [ctypes.c_int]
        _lib = lib
        return lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _log2(n: int) -> int:
    if n < 1 or n & (n - 1):
        raise ValueError(f"length {n} is not a power of two")
    return n.bit_length() - 1


def _as_ri(x) -> np.ndarray:
    """complex array (..., N) -> contiguous float64 (..., N, 2)."""
    x = np.asarray(x)
    if np.iscomplexobj(x):
        return np.ascontiguousarray(np.stack([x.real, x.imag], axis=-1), dtype=np.float64)
    return np.ascontiguousarray(np.stack([x, np.zeros_like(x)], axis=-1), dtype=np.float64)


def _from_ri(a: np.ndarray) -> np.ndarray:
    return a[..., 0] + 1j * a[..., 1]


def long_double_mantissa_bits() -> int:
    return int(_load().orc_long_double_digits())


def naive_dft(x, sign: int = -1) -> np.ndarray:
    """X(k) = sum_n x(n) exp(sign * 2*pi*i*n*k/N), Eq. qft_0A (sign -1)."""
    lib = _load()
    ri = _as_ri(x)
    n = ri.shape[-2]
    flat = ri.reshape(-1, n, 2)
    out = np.empty_like(flat)
    for b in range(flat.shape[0]):
        src = np.ascontiguousarray(flat[b])
        dst = np.empty_like(src)
        rc = lib.orc_naive_dft(_log2(n), _dp(src), _dp(dst), sign)
        if rc:
            raise ValueError(f"orc_naive_dft rc={rc}")
        out[b] = dst
    return _from_ri(out.reshape(ri.shape))


def dft_bin(x, k: int, sign: int = -1) -> complex:
    """One bin of Eq. qft_0A in long double, O(N)."""
    lib = _load()
    ri = np.ascontiguousarray(_as_ri(x).reshape(-1, 2))
    out = np.empty(2)
    rc = lib.orc_dft_bin(_log2(ri.shape[0]), _dp(ri), int(k), _dp(out), sign)
    if rc:
        raise ValueError(f"orc_dft_bin rc={rc}")
    return complex(out[0], out[1])


def amqft(x, variant: int, prec: str = "f64", sign: int = -1) -> np.ndarray:
    """AM-QFT complex DFT (variant 1..8) of x with shape (..., N)."""
    lib = _load()
    ri = _as_ri(x)
    n = ri.shape[-2]
    flat = ri.reshape(-1, n, 2)
    out = np.empty_like(flat)
    for b in range(flat.shape[0]):
        src = np.ascontiguousarray(flat[b])
        dst = np.empty_like(src)
        rc = lib.orc_cdft(PREC[prec], int(variant), _log2(n), _dp(src), _dp(dst), sign, None)
        if rc:
            raise ValueError(f"orc_cdft rc={rc}")
        out[b] = dst
    return _from_ri(out.reshape(ri.shape))


def amqft_batch(x, variant: int, threads: int = 0, prec: str = "f64", sign: int = -1):
    """Batch (B, N) with OpenMP over B; returns (result, threads_used)."""
    lib = _load()
    ri = _as_ri(x)
    b, n = ri.shape[0], ri.shape[1]
    out = np.empty_like(ri)
    used = lib.orc_cdft_batch(PREC[prec], int(variant), _log2(n), b, _dp(ri), _dp(out), sign, threads)
    if used < 0:
        raise ValueError(f"orc_cdft_batch rc={used}")
    return _from_ri(out), int(used)


def tally(variant: int, log2n: int, kind: str = "cdft"):
    """(sums, mults, halvings) of one transform of length 2^log2n."""
    lib = _load()
    t = (ctypes.c_longlong * 3)()
    n = 1 << log2n
    if kind == "cdft":
        src = np.zeros((n, 2))
        dst = np.empty_like(src)
        rc = lib.orc_cdft(1, int(variant), log2n, _dp(src), _dp(dst), -1, t)
    else:
        src = np.zeros(n + 2)
        dst = np.zeros(n + 2)
        rc = lib.orc_sub(1, int(variant), KIND[kind], log2n, _dp(src), _dp(dst), t)
    if rc:
        raise ValueError(f"tally rc={rc}")
    return int(t[0]), int(t[1]), int(t[2])


def sub_sizes(kind: str, m: int):
    if kind == "rdft":
        return m, m
    if kind == "dct":
        return m // 2 + 1, m // 2 + 1
    if kind == "dst":
        return m // 2 - 1, m // 2 - 1
    if kind in ("dct_ot", "dst_ot", "dct_to", "dst_to"):
        return m // 4, m // 4
    return m // 8, m // 8


def sub(kind: str, variant: int, log2m: int, x, prec: str = "f64") -> np.ndarray:
    """One function of the recursion on its input array (Tab. 2 storage)."""
    lib = _load()
    nin, nout = sub_sizes(kind, 1 << log2m)
    src = np.zeros(max(nin, 1) + 1)
    src[:nin] = np.asarray(x, dtype=np.float64)
    dst = np.zeros(max(nout, 1) + 1)
    rc = lib.orc_sub(PREC[prec], int(variant), KIND[kind], log2m, _dp(src), _dp(dst), None)
    if rc:
        raise ValueError(f"orc_sub rc={rc}")
    return dst[:nout].copy()


def mv_time(variant: int, ctx: int, log2m: int, x) -> np.ndarray:
    lib = _load()
    src = np.ascontiguousarray(x, dtype=np.float64)
    dst = np.zeros_like(src)
    if lib.orc_mv_time(variant, ctx, log2m, _dp(src), _dp(dst)):
        raise ValueError("orc_mv_time")
    return dst


def mv_freq(variant: int, ctx: int, log2m: int, e) -> np.ndarray:
    lib = _load()
    src = np.ascontiguousarray(e, dtype=np.float64)
    dst = np.zeros_like(src)
    if lib.orc_mv_freq(variant, ctx, log2m, _dp(src), _dp(dst)):
        raise ValueError("orc_mv_freq")
    return dst


def angles(variant: int, log2n: int) -> np.ndarray:
    """Sorted q (0 < q < N) such that the transform reads a constant at 2*pi*q/N."""
    lib = _load()
    n = 1 << log2n
    used = np.zeros(n, dtype=np.uint8)
    if lib.orc_angles(variant, log2n, used.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))):
        raise ValueError("orc_angles")
    return np.nonzero(used)[0]


@contextlib.contextmanager
def fault(name: str):
    """Plant one deliberate mistake in the oracle for the duration of a block."""
    lib = _load()
    lib.orc_set_fault(FAULTS[name])
    try:
        yield
    finally:
        lib.orc_set_fault(0)


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
