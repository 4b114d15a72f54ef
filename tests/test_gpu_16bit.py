"""16-bit storage (bf16 / fp16 / int16 pairs with one power-of-two exponent
per transform, float32 arithmetic; int16 is the block-floating-point form)
against the oracle.

Variants 2, 4, 6, 8 compute the same float32 values as the oracle's float32
recursion, so their 16-bit output is pinned bit for bit: the exponent from
the largest component magnitude, the values scaled by 2^-exp and rounded to
nearest even.  Every variant is also held to rel-L2 <= 4e-3 (plus twice the
float32 recursion's own error) against the float64 oracle run on the
16-bit-rounded input.
"""
import numpy as np
import pytest

import synth
from gpu_util import expected_exponent, rel

pytestmark = pytest.mark.gpu

AMQFT_CBF16, AMQFT_CF16, AMQFT_CI16 = 1, 2, 3
DTYPES = [AMQFT_CBF16, AMQFT_CF16, AMQFT_CI16]


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch

    from paper_1404_1810_gb300 import build, load

    assert torch.cuda.is_available()
    build.build()
    return load()


def _tdt(dt):
    import torch

    return {AMQFT_CBF16: torch.bfloat16, AMQFT_CF16: torch.float16, AMQFT_CI16: torch.int16}[dt]


def _to16(t, dt):
    """float tensor -> the 16-bit type: round to nearest even (int16: to the
    nearest integer, ties to even, as the kernels store it)."""
    return t.round().to(_tdt(dt)) if dt == AMQFT_CI16 else t.to(_tdt(dt))


def quantize_input(x, dt):
    """(b, n) complex128 -> (b, n, 2) 16-bit CPU tensor (round to nearest even;
    int16 holds the signal times 2^12, exponent 0)."""
    import torch

    t = torch.view_as_real(torch.from_numpy(np.ascontiguousarray(x)))
    return _to16(t * 4096.0 if dt == AMQFT_CI16 else t, dt).contiguous()


def run16(x16, log2n, v, dt, inverse=False, exp_in=None):
    import torch

    from paper_1404_1810_gb300 import Plan

    b = x16.shape[0]
    p = Plan(log2n, v, b, dt)
    try:
        xd = x16.cuda()
        if inverse:
            y, e = p.inv(xd, exp_in=exp_in.cuda() if exp_in is not None else None)
        else:
            y, e = p.fwd(xd)
        torch.cuda.synchronize()
    finally:
        p.close()
    return y.cpu(), e.cpu()


CASES = [(0, 4), (1, 4), (2, 2), (3, 8), (10, 4), (10, 2), (13, 6), (14, 4), (15, 8), (16, 2), (16, 4), (17, 4),
         (17, 6)]


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("log2n,v", CASES)
def test_16bit_bit_exact(orc, dt, log2n, v):
    import torch

    n = 1 << log2n
    b = 5 if log2n <= 14 else 2
    x = synth.normal_complex(n, b, config=3, stream=log2n)
    x16 = quantize_input(x, dt)
    y16, e = run16(x16, log2n, v, dt)
    xin = torch.view_as_complex(x16.double()).numpy()
    for i in range(b):
        r32 = orc.amqft(xin[i], v, prec="f32").astype(np.complex64)
        ee = expected_exponent(r32)
        assert int(e[i]) == ee, (i, int(e[i]), ee)
        scaled = (r32 * np.float32(2.0 ** -ee)).astype(np.complex64)
        want = _to16(torch.view_as_real(torch.from_numpy(scaled)), dt)
        assert torch.equal(y16[i].view(torch.int16), want.view(torch.int16)), (log2n, v, i)


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("family", ["gauss", "multitone"])
@pytest.mark.parametrize("log2n,v", [(10, 1), (10, 3), (10, 5), (10, 7), (10, 2), (14, 1), (14, 3), (16, 4), (16, 1),
                                     (18, 2)])
def test_16bit_accuracy(orc, dt, family, log2n, v):
    import torch

    from paper_1404_1810_gb300 import dequantize

    n, b = 1 << log2n, 2
    if family == "gauss":
        x = synth.normal_complex(n, b, config=3, stream=100 + log2n)
    else:
        x = synth.multitone(n, b, config=3, stream=200 + log2n)
    x16 = quantize_input(x, dt)
    y16, e = run16(x16, log2n, v, dt)
    y = dequantize(y16, e).numpy()
    xin = torch.view_as_complex(x16.double()).numpy()
    for i in range(b):
        r64 = orc.amqft(xin[i], v)
        r32 = orc.amqft(xin[i], v, prec="f32")
        tol = 4e-3 + 2.0 * rel(r32, r64)
        assert rel(y[i], r64) <= tol, (v, log2n, family, rel(y[i], r64), tol)


@pytest.mark.parametrize("dt", DTYPES)
@pytest.mark.parametrize("log2n", [6, 14, 17])
def test_16bit_roundtrip_with_exponents(dt, log2n):
    """inv(fwd(x)) with the forward's exponents as exp_in gives N x."""
    import torch

    from paper_1404_1810_gb300 import dequantize

    n, b = 1 << log2n, 3
    x = synth.normal_complex(n, b, config=3, stream=300 + log2n)
    x16 = quantize_input(x, dt)
    y16, e = run16(x16, log2n, 4, dt)
    z16, ez = run16(y16, log2n, 4, dt, inverse=True, exp_in=e)
    z = dequantize(z16, ez).numpy()
    xin = torch.view_as_complex(x16.double()).numpy()
    assert rel(z, n * xin) < (8e-3 if dt == AMQFT_CBF16 else 2e-3)


def test_16bit_zero_transform_and_errors():
    import torch

    from paper_1404_1810_gb300 import AmqftError, Plan, amqft_exec_fwd

    n, b = 1 << 12, 2
    x = torch.zeros((b, n, 2), dtype=torch.bfloat16, device="cuda")
    p = Plan(12, 4, b, AMQFT_CBF16)
    try:
        y, e = p.fwd(x)
        torch.cuda.synchronize()
        assert int(e.abs().sum()) == 0 and int(y.view(torch.int16).abs().sum()) == 0
        out = torch.empty_like(x)
        with pytest.raises(AmqftError) as err:   # exp_out is required
            amqft_exec_fwd(p.handle, x.data_ptr(), out.data_ptr(), 0, 0)
        assert err.value.code == -8
    finally:
        p.close()
    pc = Plan(12, 4, b)
    try:
        xc = torch.zeros((b, n), dtype=torch.complex64, device="cuda")
        e = torch.zeros(b, dtype=torch.int32, device="cuda")
        with pytest.raises(AmqftError) as err:   # exponents with complex64
            amqft_exec_fwd(pc.handle, xc.data_ptr(), torch.empty_like(xc).data_ptr(), e.data_ptr(), 0)
        assert err.value.code == -3
    finally:
        pc.close()
