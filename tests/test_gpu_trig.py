"""DCT-0 / DST-0 (Eq. qft_0B-0C) and the inverse real transform.

amqft_exec_dct_dst feeds the caller's signals straight into the regions of
the recursion (no D_c, D_r) and returns the regions' results, so for the
variants without recurrences (2, 4, 6, 8) it must equal the oracle's dct(N)
and dst(N) evaluated in float32 bit for bit; variants 1 and 3 are held to the
derived tolerance against the float64 oracle, 5 and 7 to the float32
recursion's own error.  The oracle's functions are pinned against the pruned
DCT-0 / DST-0 definitions in the CPU tests.  amqft_exec_irdft is the complex
inverse of Z = X_a + i X_b (Hermitian extension of two half spectra): equal,
for 2/4/6/8, to the oracle's float32 inverse of the same Z, and irdft(rdft(x))
= N x.  Covered: single-CTA, cluster (2^14..2^16) and multi-pass sizes, an
odd count, one kind absent, in place.
"""
import numpy as np
import pytest

import synth
from gpu_util import derived_tol, rel, sine_scan_check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch

    from paper_1404_1810_gb300 import build, load

    assert torch.cuda.is_available()
    build.build()
    return load()


def _signals(count, width, stream):
    return synth.real_signals(width, count, stream=stream).astype(np.float32)


def _check(got, x, kind, v, log2n, orc, tag):
    for i in range(x.shape[0]):
        r32 = orc.sub(kind, v, log2n, x[i].astype(np.float64), prec="f32")
        if v in (2, 4, 6, 8):
            assert np.array_equal(got[i], r32.astype(np.float32), equal_nan=True), (tag, i)
        else:
            r64 = orc.sub(kind, v, log2n, x[i].astype(np.float64))
            if v in (1, 3):
                assert rel(got[i], r64) <= derived_tol(rel(r32, r64), log2n), (tag, i)
            else:
                sine_scan_check(got[i].astype(np.float64), r32, r64, f"{tag} {i}")


CASES = [(2, 4, 3), (3, 2, 2), (6, 8, 5), (10, 4, 7), (10, 1, 4), (12, 6, 3), (13, 3, 3), (14, 4, 3), (14, 2, 3),
         (15, 8, 2), (16, 4, 3), (16, 5, 2), (17, 4, 3), (17, 3, 2), (18, 2, 2)]


@pytest.mark.parametrize("log2n,v,count", CASES)
def test_dct_dst_against_oracle(orc, log2n, v, count):
    import torch

    from paper_1404_1810_gb300 import Plan

    n = 1 << log2n
    c = _signals(count, n // 2 + 1, 800 + log2n)
    s = _signals(count, n // 2 - 1, 900 + log2n)
    p = Plan(log2n, v, count)
    try:
        co, so = p.dct_dst(torch.from_numpy(c).cuda(), torch.from_numpy(s).cuda())
        torch.cuda.synchronize()
    finally:
        p.close()
    _check(co.cpu().numpy(), c, "dct", v, log2n, orc, f"dct v{v} 2^{log2n}")
    _check(so.cpu().numpy(), s, "dst", v, log2n, orc, f"dst v{v} 2^{log2n}")


def test_dct_dst_one_kind_and_in_place(orc):
    import torch

    from paper_1404_1810_gb300 import AmqftError, Plan, amqft_exec_dct_dst

    log2n, v, count = 14, 4, 3
    n = 1 << log2n
    c = _signals(count, n // 2 + 1, 811)
    s = _signals(count, n // 2 - 1, 911)
    p = Plan(log2n, v, count)
    try:
        co, so = p.dct_dst(dct=torch.from_numpy(c).cuda())            # DCT-0 only
        assert so is None
        _check(co.cpu().numpy(), c, "dct", v, log2n, orc, "dct only")
        sd = torch.from_numpy(s).cuda()
        p.dct_dst(dst=sd, dst_out=sd)                                 # DST-0 in place
        torch.cuda.synchronize()
        _check(sd.cpu().numpy(), s, "dst", v, log2n, orc, "dst in place")
        cd = torch.from_numpy(c).cuda()
        with pytest.raises(AmqftError) as e:                          # partial overlap
            amqft_exec_dct_dst(p.handle, 2, cd.data_ptr(), cd.data_ptr() + 4, 0, 0)
        assert e.value.code == -5
        with pytest.raises(AmqftError) as e:                          # count above the plan's batch
            amqft_exec_dct_dst(p.handle, 4, cd.data_ptr(), cd.data_ptr(), 0, 0)
        assert e.value.code == -8
    finally:
        p.close()


# (the sine family only where its float32 spectra are still finite)
IR_CASES = [(1, 4, 2), (2, 4, 3), (5, 2, 3), (10, 4, 5), (10, 1, 2), (12, 6, 2), (13, 8, 3), (14, 4, 2), (15, 2, 3),
            (16, 4, 3), (17, 4, 2), (18, 2, 3), (17, 3, 2)]


@pytest.mark.parametrize("log2n,v,b", IR_CASES)
def test_irdft(orc, log2n, v, b):
    import torch

    from paper_1404_1810_gb300 import Plan

    n = 1 << log2n
    x = synth.real_signals(n, b, stream=950 + log2n).astype(np.float32)
    p = Plan(log2n, v, b)
    try:
        X = p.rdft(torch.from_numpy(x).cuda())
        y = p.irdft(X)
        torch.cuda.synchronize()
        X, y = X.cpu().numpy(), y.cpu().numpy()
    finally:
        p.close()
    for j in range(0, b, 2):
        # the oracle's inverse of the same float32 Z = X_a + i X_b (Hermitian extension)
        xa = X[j]
        xb = X[j + 1] if j + 1 < b else np.zeros_like(xa)
        full = lambda h: np.concatenate([h, np.conj(h[1:-1][::-1])]) if n > 1 else h[:1]  # noqa: E731
        fa, fb = full(xa), full(xb)
        zr = (fa.real.astype(np.float32) - fb.imag.astype(np.float32))
        zi = (fa.imag.astype(np.float32) + fb.real.astype(np.float32))
        z = zr.astype(np.float64) + 1j * zi.astype(np.float64)
        r32 = orc.amqft(z, v, prec="f32", sign=+1)
        r64 = orc.amqft(z, v, sign=+1)
        got = y[j].astype(np.float64) + 1j * (y[j + 1].astype(np.float64) if j + 1 < b else 0.0)
        if v in (2, 4, 6, 8):
            assert np.array_equal(y[j], r32.real.astype(np.float32), equal_nan=True), (log2n, v, j)
            if j + 1 < b:
                assert np.array_equal(y[j + 1], r32.imag.astype(np.float32), equal_nan=True), (log2n, v, j + 1)
        elif j + 1 < b:
            assert rel(got, r64) <= derived_tol(rel(r32, r64), log2n), (log2n, v, j)
    # irdft(rdft(x)) = N x for variants 1-4, within twice the derived bound of
    # one transform (the float32 recursion's error on this input)
    if v <= 4:
        x0 = x[0].astype(np.complex128)
        e32 = rel(orc.amqft(x0, v, prec="f32"), orc.amqft(x0, v))
        assert rel(y, n * x) <= 2 * derived_tol(e32, log2n), (log2n, v, rel(y, n * x), e32)
