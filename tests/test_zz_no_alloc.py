"""amqft_exec_static: the multi-pass transform with the library's fixed device
scratch instead of a plan workspace.  It must give the same results as
amqft_exec_fwd/inv of an ordinary plan, on repeated calls (the scratch then
holds the previous call's data), and reject lengths it cannot hold."""
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch

    from paper_1404_1810_gb300 import build, load

    assert torch.cuda.is_available()
    build.build()
    return load()


def _ref(log2n, variant, x, inverse):
    import torch

    from paper_1404_1810_gb300 import Plan

    p = Plan(log2n, variant, x.shape[0])
    try:
        y = p.inv(x) if inverse else p.fwd(x)
        torch.cuda.synchronize()
    finally:
        p.close()
    return y


# (log2n, variant, batch): 20 transforms of 2^17 take two chunks (15 + 5);
# 3 of 2^20 take two (2 + 1)
CASES = [(17, 4, 20), (18, 8, 3), (20, 2, 3), (19, 6, 2), (17, 1, 20), (18, 3, 3)]


@pytest.mark.parametrize("log2n,variant,batch", CASES)
def test_static_matches_plan_exec(lib, log2n, variant, batch):
    import torch

    from paper_1404_1810_gb300 import amqft_destroy, amqft_exec_static, amqft_plan

    n = 1 << log2n
    x = synth.device_normal_complex64(n, batch, "cuda", seed_offset=log2n * 10 + variant)
    h = amqft_plan(log2n, variant, 0)   # constant table only, no workspace
    try:
        for inverse in (0, 1):
            ref = _ref(log2n, variant, x, inverse)
            for _ in range(2):          # two calls in a row on the same scratch
                out = torch.full_like(x, complex(float("nan"), float("nan")))
                amqft_exec_static(h, batch, x.data_ptr(), out.data_ptr(), inverse,
                                  torch.cuda.current_stream().cuda_stream)
                torch.cuda.synchronize()
                # same kernels and operations: bit-identical (tolerance 0)
                torch.testing.assert_close(torch.view_as_real(out), torch.view_as_real(ref), rtol=0, atol=0,
                                           equal_nan=True)
    finally:
        amqft_destroy(h)


def test_static_allocates_nothing(lib):
    """A batch-0 plan holds its constant table only, and calls of
    amqft_exec_static take no device memory (free memory measured by the
    driver before and after, once a warm-up call has loaded the module)."""
    import torch

    from paper_1404_1810_gb300 import amqft_destroy, amqft_exec_static, amqft_plan

    log2n, batch = 18, 4
    n = 1 << log2n
    x = synth.device_normal_complex64(n, batch, "cuda", seed_offset=5)
    out = torch.empty_like(x)
    st = torch.cuda.current_stream().cuda_stream
    h = amqft_plan(log2n, 4, 0)
    try:
        amqft_exec_static(h, batch, x.data_ptr(), out.data_ptr(), 0, st)   # warm-up: module loaded
        torch.cuda.synchronize()
    finally:
        amqft_destroy(h)
    free0 = torch.cuda.mem_get_info()[0]
    h = amqft_plan(log2n, 4, 0)
    try:
        table = (n // 4 - 2) * 4
        free1 = torch.cuda.mem_get_info()[0]
        assert free0 - free1 <= table + (4 << 20), "a batch-0 plan holds more than its constant table"
        for inverse in (0, 1, 0):
            amqft_exec_static(h, batch, x.data_ptr(), out.data_ptr(), inverse, st)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free1, "amqft_exec_static took device memory"
    finally:
        amqft_destroy(h)


def test_static_rejects_what_it_cannot_hold(lib):
    import torch

    from paper_1404_1810_gb300 import AmqftError, amqft_destroy, amqft_exec_static, amqft_plan

    x = torch.zeros(1 << 17, dtype=torch.complex64, device="cuda")
    y = torch.zeros_like(x)
    for log2n, code in ((21, -1), (16, -1)):
        h = amqft_plan(log2n, 4, 0)
        try:
            with pytest.raises(AmqftError) as e:
                amqft_exec_static(h, 1, x.data_ptr(), y.data_ptr())
            assert e.value.code == code
            assert "static scratch" in str(e.value)
        finally:
            amqft_destroy(h)
    h = amqft_plan(17, 4, 0)
    try:
        with pytest.raises(AmqftError) as e:
            amqft_exec_static(h, -1, x.data_ptr(), y.data_ptr())
        assert e.value.code == -8
        amqft_exec_static(h, 0, 0, 0)          # empty batch: nothing to do
        with pytest.raises(AmqftError) as e:   # in and out overlap without being equal
            amqft_exec_static(h, 1, x.data_ptr(), x.data_ptr() + 8 * 64)
        assert e.value.code == -5
    finally:
        amqft_destroy(h)
