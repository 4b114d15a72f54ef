"""Ragged batches: every transform of a mixed-length batch equals, bit for
bit, the batched entry point of its own length (both run the same kernels),
for every launch-knob setting, under CUDA-graph capture and replay, with
skipped entries counted; sampled transforms also against the oracle."""
import numpy as np
import pytest

import synth
from gpu_util import derived_tol, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    import torch

    from paper_1404_1810_gb300 import build, load

    assert torch.cuda.is_available()
    build.build()
    return load()


def make_batch(count, lo, hi, stream=0):
    import torch

    lg = synth.ragged_log2n(count, lo, hi)
    off = synth.ragged_offsets(lg)
    x = synth.ragged_data(lg, stream=stream).astype(np.complex64)
    return (torch.from_numpy(x).cuda(), torch.from_numpy(lg).cuda(), torch.from_numpy(off).cuda(), lg, off)


def batched_reference(x, lg, off, variant, inverse):
    """Per-length batched calls on the same data (the standard entry point)."""
    import torch

    from paper_1404_1810_gb300 import Plan

    out = torch.zeros_like(x)
    for c in np.unique(lg):
        idx = np.nonzero(lg == c)[0]
        n = 1 << int(c)
        rows = torch.stack([x[int(off[i]):int(off[i]) + n] for i in idx]).contiguous()
        p = Plan(int(c), variant, len(idx))
        y = p.inv(rows) if inverse else p.fwd(rows)
        torch.cuda.synchronize()
        p.close()
        for j, i in enumerate(idx):
            out[int(off[i]):int(off[i]) + n] = y[j]
    return out


@pytest.mark.parametrize("v,hi", [(4, 18), (2, 17), (1, 16), (8, 16), (3, 14), (1, 17), (7, 17)])
def test_ragged_matches_batched(v, hi):
    import torch

    from paper_1404_1810_gb300 import RaggedPlan

    x, lgd, offd, lg, off = make_batch(240, 0, hi, stream=v)
    total = int(x.numel())
    p = RaggedPlan(hi, v, 240, total)
    try:
        for inverse in (False, True):
            y = p.exec(x, lgd, offd, inverse=inverse)
            torch.cuda.synchronize()
            assert p.skipped() == 0
            ref = batched_reference(x, lg, off, v, inverse)
            assert torch.equal(y, ref), (v, inverse)
    finally:
        p.close()


def test_ragged_against_oracle(orc):
    import torch

    from paper_1404_1810_gb300 import RaggedPlan

    x, lgd, offd, lg, off = make_batch(60, 4, 17, stream=9)
    p = RaggedPlan(17, 4, 60, int(x.numel()))
    try:
        y = p.exec(x, lgd, offd).cpu().numpy()
    finally:
        p.close()
    xh = x.cpu().numpy().astype(np.complex128)
    for i in list(np.argsort(lg)[-3:]) + [0, 1, 2]:
        n = 1 << int(lg[i])
        s = slice(int(off[i]), int(off[i]) + n)
        r32 = orc.amqft(xh[s], 4, prec="f32")
        assert np.array_equal(y[s], r32.astype(np.complex64)), i


def test_ragged_knobs_agree():
    import itertools

    import torch

    from paper_1404_1810_gb300 import RaggedPlan

    x, lgd, offd, lg, off = make_batch(500, 1, 16, stream=3)
    p = RaggedPlan(16, 2, 500, int(x.numel()))
    try:
        ref = p.exec(x, lgd, offd).clone()
        for sched, order, spm, cm in itertools.product((0, 1), (0, 1), (1, 2), (1, 2)):
            p.tune(schedule=sched, order=order, small_ctas_per_sm=spm, cluster_mult=cm)
            y = p.exec(x, lgd, offd)
            torch.cuda.synchronize()
            assert torch.equal(y, ref), (sched, order, spm, cm)
    finally:
        p.close()


def test_ragged_cuda_graph():
    """Captured once, replayed on new data in the same buffers."""
    import torch

    from paper_1404_1810_gb300 import RaggedPlan

    x, lgd, offd, lg, off = make_batch(300, 4, 18, stream=5)
    x2 = make_batch(300, 4, 18, stream=6)[0]
    p = RaggedPlan(18, 4, 300, int(x.numel()))
    try:
        xin = x.clone()
        y = torch.empty_like(x)
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            p.exec(xin, lgd, offd, y, stream=s)   # eager call first (kernel attributes)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            p.exec(xin, lgd, offd, y)
        for data in (x, x2):
            xin.copy_(data)
            g.replay()
            torch.cuda.synchronize()
            assert torch.equal(y, p.exec(data, lgd, offd))
    finally:
        p.close()


def test_ragged_skips_and_errors():
    import torch

    from paper_1404_1810_gb300 import AmqftError, Plan, RaggedPlan, amqft_exec_ragged

    lg = np.array([3, 12, 15, 5, 14], dtype=np.uint8)
    off = synth.ragged_offsets(lg)
    total = int((1 << lg.astype(np.int64)).sum())
    x = torch.from_numpy(synth.ragged_data(lg, stream=7).astype(np.complex64)).cuda()
    p = RaggedPlan(12, 4, 5, total)
    try:
        y = torch.zeros_like(x)
        p.exec(x, torch.from_numpy(lg).cuda(), torch.from_numpy(off).cuda(), y)
        torch.cuda.synchronize()
        assert p.skipped() == 2                       # 2^15 and 2^14 exceed the plan
        n12 = 1 << 12
        q = Plan(12, 4, 1)
        ref = q.fwd(x[int(off[1]):int(off[1]) + n12].reshape(1, -1).contiguous())
        q.close()
        assert torch.equal(y[int(off[1]):int(off[1]) + n12], ref[0])
        with pytest.raises(AmqftError) as e:          # count above max_count
            amqft_exec_ragged(p.handle, 6, off.ctypes.data, lg.ctypes.data, x.data_ptr(), y.data_ptr())
        assert e.value.code == -8
    finally:
        p.close()
    # multi-pass capacity: max_points admits one transform of 2^17 only
    lg2 = np.array([17, 17, 4], dtype=np.uint8)
    off2 = synth.ragged_offsets(lg2)
    x2 = torch.from_numpy(synth.ragged_data(lg2, stream=8).astype(np.complex64)).cuda()
    p2 = RaggedPlan(17, 4, 3, (1 << 17) + 16)
    try:
        p2.exec(x2, torch.from_numpy(lg2).cuda(), torch.from_numpy(off2).cuda())
        torch.cuda.synchronize()
        assert p2.skipped() == 1
    finally:
        p2.close()
    q = Plan(10, 4, 1)
    try:
        with pytest.raises(AmqftError) as e:          # not a ragged plan
            amqft_exec_ragged(q.handle, 1, off.ctypes.data, lg.ctypes.data, x.data_ptr(), x.data_ptr())
        assert e.value.code == -8
    finally:
        q.close()
    with pytest.raises(AmqftError) as e:
        from paper_1404_1810_gb300 import amqft_plan_ragged
        amqft_plan_ragged(10, 4, 1, 10, 1000)        # 16-bit storage
    assert e.value.code == -3


def test_autotuner_picks_a_valid_setting(tmp_path):
    import torch

    from paper_1404_1810_gb300 import RaggedPlan
    from paper_1404_1810_gb300.autotune import GRID, tune_ragged

    x, lgd, offd, lg, off = make_batch(400, 4, 16, stream=11)
    p = RaggedPlan(16, 4, 400, int(x.numel()))
    try:
        cache = str(tmp_path / "tune.json")
        best = tune_ragged(p, x, lgd, offd, reps=2, cache_path=cache)
        assert all(best[k] in GRID[k] for k in GRID)
        again = tune_ragged(p, x, lgd, offd, reps=2, cache_path=cache)   # served from the cache
        assert again == best
        y = p.exec(x, lgd, offd)
        torch.cuda.synchronize()
        assert torch.equal(y, batched_reference(x, lg, off, 4, False))
    finally:
        p.close()


@pytest.mark.parametrize("shift", [0, 1])
def test_ragged_unaligned_offsets(shift):
    """Variant 4 runs the 2^14..2^16 transforms of a ragged batch on the
    paired-region kernel when their data is 16-byte aligned and on the fused
    cluster kernel otherwise (odd element offsets, or in and out at different
    16-byte phases): every transform still equals the per-length batched call."""
    import torch

    from paper_1404_1810_gb300 import RaggedPlan

    lg = np.array([14, 15, 16, 14, 16, 15, 3, 14], dtype=np.uint8)
    n = 1 << lg.astype(np.int64)
    gaps = np.array([1, 0, 1, 1, 0, 0, 1, 0])               # one-element gaps make odd offsets
    off = np.cumsum(n + gaps) - n
    total = int(off[-1] + n[-1]) + 2
    data = synth.normal_complex(total, 1, config=4, stream=77)[0].astype(np.complex64)
    base = torch.zeros(total + 2, dtype=torch.complex64, device="cuda")
    x = base[shift:shift + total]                            # shift 1: the buffer at an odd 8-byte phase
    x.copy_(torch.from_numpy(data))
    lgd, offd = torch.from_numpy(lg).cuda(), torch.from_numpy(off.astype(np.int64)).cuda()
    p = RaggedPlan(16, 4, len(lg), total)
    try:
        for inverse in (False, True):
            for out_shift in (0, 1):
                ob = torch.zeros(total + 2, dtype=torch.complex64, device="cuda")
                out = ob[out_shift:out_shift + total]
                p.exec(x, lgd, offd, out=out, inverse=inverse)
                torch.cuda.synchronize()
                assert p.skipped() == 0
                ref = batched_reference(x, lg, off, 4, inverse)
                for i in range(len(lg)):
                    a, b = int(off[i]), int(off[i] + n[i])
                    assert torch.equal(out[a:b], ref[a:b]), (shift, out_shift, inverse, i)
    finally:
        p.close()
