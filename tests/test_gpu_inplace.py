"""In-place execution (in == out).

Every kernel reads a transform's whole input before it writes any of that
transform's output, and no transform's output overlaps another transform's
input, so the in-place call must give the out-of-place result bit for bit:
on the single-CTA kernels (N <= 2^13), the cluster kernels (2^14..2^16), the
paired-region kernel (variant 4, 2^14..2^16), the multi-pass path (2^17 and
up, a time-first and a recurrence variant), 16-bit storage (values and
exponents in place), the host-memory path, the ragged path and the
allocation-free entry point.  An overlap that is not equality stays an error.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch

    from paper_1404_1810_gb300 import build, load

    assert torch.cuda.is_available()
    build.build()
    return load()


# (log2n, variant, batch)
CASES = [(0, 4, 5), (10, 4, 37), (10, 1, 33), (13, 7, 5), (14, 2, 9), (15, 8, 6), (16, 4, 40), (16, 5, 7),
         (17, 4, 3), (17, 3, 2), (18, 6, 2)]


@pytest.mark.parametrize("log2n,v,b", CASES)
def test_inplace_matches_out_of_place(log2n, v, b):
    import torch

    from paper_1404_1810_gb300 import Plan

    x = synth.device_normal_complex64(1 << log2n, b, "cuda")
    p = Plan(log2n, v, b)
    try:
        for inverse in (False, True):
            ref = p.inv(x) if inverse else p.fwd(x)
            z = x.clone()
            r = p.inv(z, out=z) if inverse else p.fwd(z, out=z)
            torch.cuda.synchronize()
            assert r.data_ptr() == z.data_ptr()
            assert torch.equal(z, ref), (log2n, v, inverse)
    finally:
        p.close()


@pytest.mark.parametrize("dt", [1, 2])
@pytest.mark.parametrize("log2n", [12, 16, 17])
def test_inplace_16bit(dt, log2n):
    import torch

    from paper_1404_1810_gb300 import Plan

    b = 3
    tdt = torch.bfloat16 if dt == 1 else torch.float16
    x = synth.device_normal_complex64(1 << log2n, b, "cuda")
    x16 = torch.view_as_real(x).to(tdt).contiguous()
    p = Plan(log2n, 4, b, dt)
    try:
        y, e = p.fwd(x16)
        zi, ze = p.inv(y, exp_in=e)
        y2 = x16.clone()
        e2 = torch.empty(b, dtype=torch.int32, device="cuda")
        p.fwd(y2, out=y2, exp_out=e2)
        p.inv(y2, out=y2, exp_in=e2, exp_out=e2)     # exponents in place too
        torch.cuda.synchronize()
        assert torch.equal(y2.view(torch.int16), zi.view(torch.int16))
        assert torch.equal(e2, ze)
    finally:
        p.close()


def test_inplace_host():
    import torch

    from paper_1404_1810_gb300 import Plan

    log2n, b = 12, 20
    x = torch.from_numpy(synth.normal_complex(1 << log2n, b, stream=31).astype(np.complex64)).pin_memory()
    p = Plan(log2n, 4, b)
    try:
        ref = p.fwd_host(x, chunk=3)
        torch.cuda.synchronize()
        z = x.clone().pin_memory()
        p.fwd_host(z, out=z, chunk=3)
        torch.cuda.synchronize()
        assert torch.equal(z, ref)
    finally:
        p.close()


def test_inplace_ragged():
    import torch

    from paper_1404_1810_gb300 import RaggedPlan

    lg = synth.ragged_log2n(120, 0, 17)
    off = synth.ragged_offsets(lg)
    x = torch.from_numpy(synth.ragged_data(lg, stream=12).astype(np.complex64)).cuda()
    lgd, offd = torch.from_numpy(lg).cuda(), torch.from_numpy(off).cuda()
    p = RaggedPlan(17, 4, 120, int(x.numel()))
    try:
        ref = p.exec(x, lgd, offd)
        z = x.clone()
        p.exec(z, lgd, offd, out=z)
        torch.cuda.synchronize()
        assert p.skipped() == 0
        assert torch.equal(z, ref)
    finally:
        p.close()


def test_inplace_static():
    import torch

    from paper_1404_1810_gb300 import amqft_destroy, amqft_exec_static, amqft_plan

    log2n, b = 17, 4
    x = synth.device_normal_complex64(1 << log2n, b, "cuda")
    h = amqft_plan(log2n, 1, 0)
    try:
        ref = torch.empty_like(x)
        amqft_exec_static(h, b, x.data_ptr(), ref.data_ptr(), 0, 0)
        z = x.clone()
        amqft_exec_static(h, b, z.data_ptr(), z.data_ptr(), 0, 0)
        torch.cuda.synchronize()
        assert torch.equal(z, ref)
    finally:
        amqft_destroy(h)


def test_partial_overlap_rejected():
    import torch

    from paper_1404_1810_gb300 import AmqftError, Plan, amqft_exec_fwd

    p = Plan(10, 4, 2)
    buf = torch.zeros(4 * 1024, dtype=torch.complex64, device="cuda")
    try:
        with pytest.raises(AmqftError) as e:
            amqft_exec_fwd(p.handle, buf.data_ptr(), buf.data_ptr() + 8 * 8, 0, 0)
        assert e.value.code == -5
        amqft_exec_fwd(p.handle, buf.data_ptr(), buf.data_ptr(), 0, 0)   # equal: in place
        torch.cuda.synchronize()
    finally:
        p.close()
