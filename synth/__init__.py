"""Seeded synthetic workloads for the AM-QFT transform.

Shared by the tests, the bench and the smoke check; imported by neither the
oracle nor the CUDA library (both receive arrays).  This module holds no
transform arithmetic: only random draws, the definitions of the test
signals, and size lists.

Every generator is counter-based (numpy Philox, or torch's Philox on the
device) keyed by ``SEED_BASE + config`` so the same call always returns the
same data.  Config ids follow the workload list:

  1  single complex DFT N=1024, Re/Im iid U[-1, 1)
  2  batched complex64, N=2^16 x 4096 (and the 2^28-point size sweep), N(0, 1)
  3  16-bit storage: N(0, 1) and sparse multi-tone (8 tones, 60 dB spread)
  4  ragged batch: 20000 transforms, log2 N ~ U{4..18}, U[-1, 1)
  5  autograd: 512 real signals N=2^14 lifted to complex, spectral mask U[0, 1)
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 1404_1810


def rng(config: int, stream: int = 0) -> np.random.Generator:
    """Philox generator for (config, stream)."""
    return np.random.Generator(np.random.Philox(key=[SEED_BASE + int(config), int(stream)]))


def uniform_complex(n: int, batch: int = 1, config: int = 1, stream: int = 0) -> np.ndarray:
    """(batch, n) complex128, Re and Im iid U[-1, 1)."""
    g = rng(config, stream)
    re = g.uniform(-1.0, 1.0, size=(batch, n))
    im = g.uniform(-1.0, 1.0, size=(batch, n))
    return re + 1j * im


def normal_complex(n: int, batch: int = 1, config: int = 2, stream: int = 0) -> np.ndarray:
    """(batch, n) complex128, Re and Im iid N(0, 1)."""
    g = rng(config, stream)
    re = g.standard_normal(size=(batch, n))
    im = g.standard_normal(size=(batch, n))
    return re + 1j * im


def multitone(n: int, batch: int = 1, config: int = 3, stream: int = 0, tones: int = 8,
              spread_db: float = 60.0, floor_std: float = 1e-6) -> np.ndarray:
    """(batch, n) complex128: a sum of `tones` complex exponentials at random
    integer bins with uniform random phases and amplitudes 10^(-u*spread/20),
    u ~ U[0, 1), plus an iid complex N(0, floor_std^2) floor."""
    g = rng(config, stream)
    t = np.arange(n, dtype=np.float64)
    out = np.empty((batch, n), dtype=np.complex128)
    for b in range(batch):
        bins = g.integers(0, n, size=tones)
        phase = g.uniform(0.0, 2.0 * np.pi, size=tones)
        amp = 10.0 ** (-g.uniform(0.0, 1.0, size=tones) * spread_db / 20.0)
        sig = np.zeros(n, dtype=np.complex128)
        for f, p, a in zip(bins, phase, amp):
            # the turn fraction f*t/n is reduced mod 1 exactly before scaling by 2*pi
            frac = np.mod(f * t, n) / n
            sig += a * np.exp(1j * (2.0 * np.pi * frac + p))
        sig += floor_std * (g.standard_normal(n) + 1j * g.standard_normal(n))
        out[b] = sig
    return out


def ragged_log2n(count: int = 20000, lo: int = 4, hi: int = 18, config: int = 4) -> np.ndarray:
    """log2 N of each transform, uniform over {lo..hi}."""
    return rng(config, 1).integers(lo, hi + 1, size=count).astype(np.uint8)


def ragged_offsets(log2n: np.ndarray) -> np.ndarray:
    """Packed element offsets (int64) of each transform: transform i occupies
    [off[i], off[i] + 2^log2n[i]) complex elements.  Every N >= 2 is even, so
    every offset is even and a complex64 transform starts 16-byte aligned."""
    sizes = (np.int64(1) << log2n.astype(np.int64))
    off = np.zeros(len(sizes), dtype=np.int64)
    if len(sizes) > 1:
        off[1:] = np.cumsum(sizes[:-1])
    return off


def ragged_data(log2n: np.ndarray, config: int = 4, stream: int = 0) -> np.ndarray:
    """Packed complex128 data, Re/Im iid U[-1, 1), total sum(2^log2n) points."""
    total = int((np.int64(1) << log2n.astype(np.int64)).sum())
    g = rng(config, stream)
    return g.uniform(-1.0, 1.0, size=total) + 1j * g.uniform(-1.0, 1.0, size=total)


def real_signals(n: int, batch: int, config: int = 5, stream: int = 0) -> np.ndarray:
    """(batch, n) float64, iid U[-1, 1): real signals to lift to complex."""
    return rng(config, stream).uniform(-1.0, 1.0, size=(batch, n))


def spectral_mask(n: int, config: int = 5, stream: int = 1) -> np.ndarray:
    """(n,) float64 weights w_k ~ U[0, 1)."""
    return rng(config, stream).uniform(0.0, 1.0, size=n)


def device_normal_complex64(n: int, batch: int, device, seed_offset: int = 0):
    """(batch, n) torch.complex64 on `device`, Re/Im iid N(0, 1), drawn with
    torch's counter-based generator seeded from SEED_BASE + 2.  Used for the
    2^28-point bench buffers, which are too large to draw on the host quickly."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(SEED_BASE + 2 + seed_offset)
    ri = torch.randn((batch, n, 2), generator=g, device=device, dtype=torch.float32)
    return torch.view_as_complex(ri)
