"""Host-side logic that needs no GPU: the autotuner's cache and batch
signature, 16-bit dequantisation, and that the library refuses to run without
a CUDA device (there is no CPU fallback)."""
import os

import numpy as np
import pytest
import torch

import synth


def test_batch_signature_counts_lengths():
    from paper_1404_1810_gb300.autotune import batch_signature

    lg = torch.tensor([4, 4, 18, 0, 4], dtype=torch.uint8)
    sig = batch_signature(lg).split(",")
    assert len(sig) == 32
    assert sig[4] == "3" and sig[18] == "1" and sig[0] == "1" and sig[5] == "0"


def test_autotune_cache_roundtrip(tmp_path):
    from paper_1404_1810_gb300.autotune import _load_cache, _save_cache

    path = str(tmp_path / "sub" / "tune.json")
    assert _load_cache(path) == {}
    _save_cache(path, {"k": {"knobs": {"schedule": 1}, "ms": 1.5}})
    assert _load_cache(path)["k"]["knobs"]["schedule"] == 1
    with open(path, "w") as f:
        f.write("not json")
    assert _load_cache(path) == {}      # a damaged cache is ignored, not fatal


@pytest.mark.parametrize("dt", [torch.bfloat16, torch.float16])
def test_dequantize_scales_by_two_to_the_exponent(dt):
    from paper_1404_1810_gb300 import dequantize

    x = synth.normal_complex(64, 3, config=3)
    v = torch.view_as_real(torch.from_numpy(x)).to(dt)
    e = torch.tensor([0, 5, -7], dtype=torch.int32)
    got = dequantize(v, e).numpy()
    want = torch.view_as_complex(v.double()).numpy() * (2.0 ** e.numpy().astype(np.float64))[:, None]
    assert np.array_equal(got, want)


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the behaviour without a GPU")
def test_no_cpu_fallback():
    from paper_1404_1810_gb300 import AmqftError, Plan, build

    build.build()
    with pytest.raises(AmqftError):
        Plan(10, 4, 1)                  # no CUDA device: the plan cannot be made


def test_expected_exponent_puts_the_maximum_in_range():
    """16-bit storage reading: the exponent is the one power of two that scales
    the largest component magnitude into [2^13, 2^14), clamped to [-100, 100],
    and 0 for an all-zero or non-finite transform.  Checked against a direct
    search over exponents, not against the helper's own formula."""
    from gpu_util import expected_exponent

    rng = np.random.default_rng(14041810)
    for _ in range(2000):
        mag = np.float32(10.0 ** rng.uniform(-25, 30))
        v = (rng.standard_normal(16) + 1j * rng.standard_normal(16)).astype(np.complex64)
        v = (v / np.max(np.abs(np.stack([v.real, v.imag]))) * mag).astype(np.complex64)
        m = float(np.max(np.abs(np.stack([v.real, v.imag]))))
        want = next(e for e in range(-200, 200) if 2.0 ** 13 <= m * 2.0 ** -e < 2.0 ** 14)
        assert expected_exponent(v) == min(100, max(-100, want))
    # boundaries: exactly 2^13 and just below 2^14 keep exponent 0
    assert expected_exponent(np.array([2.0 ** 13], np.complex64)) == 0
    assert expected_exponent(np.array([np.nextafter(np.float32(2.0 ** 14), np.float32(0))], np.complex64)) == 0
    assert expected_exponent(np.array([2.0 ** 14], np.complex64)) == 1
    assert expected_exponent(np.array([1j * -3.0 * 2.0 ** 20], np.complex64)) == 8
    assert expected_exponent(np.zeros(4, np.complex64)) == 0
    assert expected_exponent(np.array([np.inf, 1.0], np.complex64)) == 0


def test_sine_scan_check_rejects_mismatches():
    """The check used for variants 5 and 7 beyond 2^9 fails on a non-finite
    pattern that differs from the float32 recursion and on an error far from
    the recursion's own; it passes on the recursion itself."""
    import numpy as np
    import pytest

    from gpu_util import sine_scan_check

    rng = np.random.default_rng(3)
    r64 = rng.standard_normal(256) + 1j * rng.standard_normal(256)
    r32 = r64 + 1e-3 * (rng.standard_normal(256) + 1j * rng.standard_normal(256))
    sine_scan_check(r32.copy(), r32, r64, "same")
    bad = r32.copy()
    bad[7] = np.nan
    with pytest.raises(AssertionError):
        sine_scan_check(bad, r32, r64, "nan")
    with pytest.raises(AssertionError):
        sine_scan_check(r64 + 10.0 * (r32 - r64), r32, r64, "x10")


def test_autograd_plan_cache_is_bounded(monkeypatch):
    """The autograd plan cache keeps the most recently used plans and closes
    the least recently used one beyond its bound (fake plans, no GPU)."""
    import contextlib

    import torch

    from paper_1404_1810_gb300 import autograd

    closed = []

    class FakePlan:
        def __init__(self, log2n, variant, batch):
            self.key = (log2n, variant, batch)

        def close(self):
            closed.append(self.key)

    monkeypatch.setattr(autograd, "Plan", FakePlan)
    monkeypatch.setattr(torch.cuda, "device", lambda i: contextlib.nullcontext())
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    autograd._plans.clear()
    try:
        first = autograd.plan_for(10, 4, 1, 0)
        for b in range(2, 2 + autograd.MAX_CACHED_PLANS):
            autograd.plan_for(10, 4, b, 0)
            if b == 3:
                assert autograd.plan_for(10, 4, 1, 0) is first   # reuse refreshes the entry
        assert len(autograd._plans) == autograd.MAX_CACHED_PLANS
        assert closed == [(10, 4, 2)]                             # least recently used went first
        assert autograd.plan_for(10, 4, 1, 0) is first
    finally:
        autograd._plans.clear()


def _umulhi(a, b):
    return (int(a) * int(b)) >> 32


def _div_model(n, d):
    """The kernels' Div helper: a multiply-high by ceil(2^32 / d) and one
    correction step, all in 32-bit unsigned arithmetic."""
    m = (0xFFFFFFFF // d + 1) & 0xFFFFFFFF if d > 1 else 0
    q = _umulhi(n, m) if d > 1 else n
    r = (n - q * d) & 0xFFFFFFFF
    r = r - (1 << 32) if r >= 1 << 31 else r
    if r < 0:
        q -= 1
    elif r >= d:
        q += 1
    return q


def test_multipass_word_index_fits_32_bits():
    """The multi-pass gather passes split a word index w into (region,
    word) with the 32-bit Div helper, valid while a chunk's words stay below
    2^32.  The plan sizes chunks to a 2 GiB workspace of two buffers of four
    regions per transform (one transform's buffers if larger); check the
    bound at every multi-pass length and the split at the region edges."""
    import re

    src = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            "paper_1404_1810_gb300", "csrc", "amqft_api.cu")).read()
    m = re.search(r"kWorkspaceBytes\s*=\s*(\d+)LL\s*<<\s*(\d+)", src)
    assert m, "workspace size not found"
    ws = int(m.group(1)) << int(m.group(2))
    rng = np.random.default_rng(5)
    for log2n in range(17, 29):
        half = 1 << (log2n - 1)
        rsg = ((half + 2 + 31) // 32) * 32
        per_t = 2 * 4 * rsg * 4
        chunk = max(1, ws // per_t)
        words = chunk * 4 * rsg
        assert words < 1 << 32, log2n
        probes = [0, words - 1] + [k * rsg + d for k in range(1, 4 * chunk, max(1, 4 * chunk // 64))
                                   for d in (-1, 0, 1)]
        probes += [int(x) for x in rng.integers(0, words, 200)]
        for w in probes:
            assert _div_model(w, rsg) == w // rsg, (log2n, w)
