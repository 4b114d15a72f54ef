"""Constants mode "fly" (Sect. 7.1): the kernels evaluate the band levels'
trig constants themselves instead of reading the plan's table.

The constants then differ from the table's (long double, rounded once) in the
last bits, so the results are no longer bit-identical to the float32
recursion; they are held to the same bounds as the recurrence variants:
variants 1-4 to the derived float32 tolerance against the float64 oracle,
variants 5-8 (no float32 accuracy beyond ~2^9, Sect. 7.3) to the float32
recursion's own error and non-finite pattern.  Every kernel family is covered:
single-CTA (2^10, 2^13), cluster (2^14, 2^15), paired (variant 4, 2^14..2^16),
multi-pass (2^17, 2^18: solve staging and the per-use evaluation of the levels
above 2^13), 16-bit storage and the ragged path.  Table mode stays the
default and bit-exact (the other parity tests).
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


def run_mode(x, v, mode, inverse=False):
    import torch

    from paper_1404_1810_gb300 import Plan

    xb = np.ascontiguousarray(np.atleast_2d(x).astype(np.complex64))
    b, n = xb.shape
    p = Plan(n.bit_length() - 1, v, b)
    try:
        p.constants = mode
        assert p.constants == mode
        xt = torch.from_numpy(xb).cuda()
        y = p.inv(xt) if inverse else p.fwd(xt)
        torch.cuda.synchronize()
    finally:
        p.close()
    return y.cpu().numpy().astype(np.complex128)


def check(y, xr, v, log2n, orc, sign, tag):
    r32 = orc.amqft(xr, v, prec="f32", sign=sign)
    r64 = orc.amqft(xr, v, sign=sign)
    if v <= 4:
        assert np.all(np.isfinite(y)), tag
        assert rel(y, r64) <= derived_tol(rel(r32, r64), log2n), (tag, rel(y, r64), rel(r32, r64))
    else:
        sine_scan_check(y, r32, r64, tag)


@pytest.mark.parametrize("v", range(1, 9))
@pytest.mark.parametrize("log2n", [8, 10, 13, 14, 15, 16])
def test_fly_single_pass(orc, v, log2n):
    if v >= 5 and log2n > 14:
        pytest.skip("sine family: overflow patterns at 2^15+ are covered by the multi-pass case")
    n = 1 << log2n
    x = synth.normal_complex(n, 3, config=2, stream=600 + 10 * v + log2n)
    for inverse in (False, True):
        y = run_mode(x, v, "fly", inverse)
        for row in (0, 2):
            xr = x[row].astype(np.complex64).astype(np.complex128)
            check(y[row], xr, v, log2n, orc, +1 if inverse else -1, f"v{v} 2^{log2n} inv={inverse} row {row}")


@pytest.mark.parametrize("v", [4, 1, 2, 3])
def test_fly_close_to_table(v):
    """The two modes differ only by the constants' last bits: their results
    agree to well within the float32 recursion's own error."""
    log2n = 16
    x = synth.normal_complex(1 << log2n, 2, config=2, stream=650 + v)
    yt = run_mode(x, v, "table")
    yf = run_mode(x, v, "fly")
    assert rel(yf, yt) < 1e-5


@pytest.mark.parametrize("v", [4, 1, 3, 2])
@pytest.mark.parametrize("log2n", [17, 18])
def test_fly_multipass(orc, v, log2n):
    x = synth.normal_complex(1 << log2n, 1, config=2, stream=660 + log2n)
    y = run_mode(x, v, "fly")
    check(y[0], x[0].astype(np.complex64).astype(np.complex128), v, log2n, orc, -1, f"v{v} 2^{log2n}")


def test_fly_16bit_and_ragged():
    import torch

    from paper_1404_1810_gb300 import Plan, RaggedPlan, amqft_plan_set_constants

    # 16-bit storage: the fly-mode float32 transform rounded as 16-bit output
    log2n, b = 14, 2
    x = synth.device_normal_complex64(1 << log2n, b, "cuda")
    p32, p16 = Plan(log2n, 4, b), Plan(log2n, 4, b, 1)
    try:
        p32.constants = p16.constants = "fly"
        y32 = p32.fwd(x)
        y16, e = p16.fwd(torch.view_as_real(x).to(torch.bfloat16).contiguous())
        torch.cuda.synchronize()
        deq = torch.view_as_complex(y16.float().contiguous()) * torch.pow(2.0, e.float())[:, None]
        assert rel(deq.cpu().numpy(), y32.cpu().numpy()) < 4e-3
    finally:
        p32.close()
        p16.close()
    # ragged: each transform equals the batched fly-mode call of its length
    lg = synth.ragged_log2n(60, 8, 17)
    off = synth.ragged_offsets(lg)
    xr = torch.from_numpy(synth.ragged_data(lg, stream=14).astype(np.complex64)).cuda()
    rp = RaggedPlan(17, 2, 60, int(xr.numel()))
    try:
        amqft_plan_set_constants(rp.handle, 1)
        yr = rp.exec(xr, torch.from_numpy(lg).cuda(), torch.from_numpy(off).cuda())
        torch.cuda.synchronize()
        for i in (0, 7, int(np.argmax(lg))):
            n = 1 << int(lg[i])
            p = Plan(int(lg[i]), 2, 1)
            try:
                p.constants = "fly"
                yi = p.fwd(xr[int(off[i]):int(off[i]) + n].reshape(1, n).contiguous())
                torch.cuda.synchronize()
            finally:
                p.close()
            assert torch.equal(yr[int(off[i]):int(off[i]) + n], yi[0]), i
    finally:
        rp.close()


def test_mode_errors():
    from paper_1404_1810_gb300 import AmqftError, Plan, amqft_plan_set_constants

    p = Plan(10, 4, 1)
    try:
        assert p.constants == "table"
        with pytest.raises(AmqftError):
            amqft_plan_set_constants(p.handle, 2)
        with pytest.raises(ValueError):
            p.constants = "disk"
    finally:
        p.close()


def test_constants_autotuner(tmp_path):
    import torch

    from paper_1404_1810_gb300 import Plan
    from paper_1404_1810_gb300.autotune import tune_constants

    x = synth.device_normal_complex64(1 << 12, 64, "cuda")
    p = Plan(12, 1, 64)
    try:
        cache = str(tmp_path / "tune.json")
        r = tune_constants(p, x, reps=2, cache_path=cache)
        assert r["mode"] in ("table", "fly") and p.constants == r["mode"]
        assert r["table_ms"] > 0 and r["fly_ms"] > 0
        assert r["mode"] == ("fly" if r["fly_ms"] < r["table_ms"] else "table")
        p.constants = "table" if r["mode"] == "fly" else "fly"
        again = tune_constants(p, x, reps=2, cache_path=cache)     # served from the cache
        assert again["mode"] == r["mode"] and p.constants == r["mode"]
        torch.cuda.synchronize()
    finally:
        p.close()
