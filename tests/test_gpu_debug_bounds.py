"""The bounds-checked debug library (AMQFT_BOUNDS_CHECK) on small cases of
every launch shape: single-CTA, the 4-CTA cluster kernels at 2^14/2^15/2^16,
the paired kernel, the ragged path (small, cluster and multi-pass lengths),
every multi-pass kernel (load, fold bands, solve, neighbour and recurrence
passes, chain, store, the 16-bit maximum and store), the real-input,
inverse-real and DCT-0 / DST-0 forms and the on-the-fly constants.  Every
region, distributed-shared-memory and HBM-element index is checked; the
failure count must stay 0, and the checked build computes the same bits as
the release build."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def debug_lib():
    import torch

    from paper_1404_1810_gb300 import build

    assert torch.cuda.is_available()
    build.build()
    return build.build(debug=True)


def _cases(torch):
    """(name, callable) pairs, each returning output tensors."""
    from paper_1404_1810_gb300 import Plan, RaggedPlan

    def cplx(log2n, v, b, inverse=False, fly=False):
        def run():
            x = synth.device_normal_complex64(1 << log2n, b, "cuda", seed_offset=log2n + v)
            p = Plan(log2n, v, b)
            try:
                if fly:
                    p.constants = "fly"
                y = p.inv(x) if inverse else p.fwd(x)
                torch.cuda.synchronize()
                return [y]
            finally:
                p.close()
        return run

    def b16(log2n, v, b):
        def run():
            x = synth.device_normal_complex64(1 << log2n, b, "cuda", seed_offset=3)
            p = Plan(log2n, v, b, 1)
            try:
                y, e = p.fwd(torch.view_as_real(x).to(torch.bfloat16).contiguous())
                torch.cuda.synchronize()
                return [y.view(torch.int16), e]
            finally:
                p.close()
        return run

    def ragged():
        lg = synth.ragged_log2n(40, 0, 17)
        off = synth.ragged_offsets(lg)
        x = torch.from_numpy(synth.ragged_data(lg, stream=21).astype(np.complex64)).cuda()
        p = RaggedPlan(17, 2, 40, int(x.numel()))
        try:
            y = p.exec(x, torch.from_numpy(lg).cuda(), torch.from_numpy(off).cuda())
            torch.cuda.synchronize()
            assert p.skipped() == 0
            return [y]
        finally:
            p.close()

    def special(log2n, v):
        def run():
            n, b = 1 << log2n, 3
            xr = torch.from_numpy(synth.real_signals(n, b, stream=5).astype(np.float32)).cuda()
            c = torch.from_numpy(synth.real_signals(n // 2 + 1, b, stream=6).astype(np.float32)).cuda()
            s = torch.from_numpy(synth.real_signals(n // 2 - 1, b, stream=7).astype(np.float32)).cuda()
            p = Plan(log2n, v, b)
            try:
                X = p.rdft(xr)
                y = p.irdft(X)
                co, so = p.dct_dst(c, s)
                torch.cuda.synchronize()
                return [X, y, co, so]
            finally:
                p.close()
        return run

    return [
        ("single-CTA 2^10 v1", cplx(10, 1, 33)), ("single-CTA 2^13 v2 inverse", cplx(13, 2, 5, True)),
        ("single-CTA 2^12 v8 fly", cplx(12, 8, 4, fly=True)), ("16-bit 2^12 v4", b16(12, 4, 3)),
        ("cluster 2^14 v2", cplx(14, 2, 3)), ("cluster 2^15 v8", cplx(15, 8, 2)), ("cluster 2^16 v1", cplx(16, 1, 2)),
        ("cluster 2^16 v4 16-bit", b16(16, 4, 2)), ("paired 2^14", cplx(14, 4, 5)), ("paired 2^15", cplx(15, 4, 3)),
        ("paired 2^16", cplx(16, 4, 40)), ("paired 2^16 inverse fly", cplx(16, 4, 3, True, True)),
        ("ragged", ragged), ("multi-pass 2^17 v4", cplx(17, 4, 2)), ("multi-pass 2^17 v1", cplx(17, 1, 2)),
        ("multi-pass 2^18 v3 fly", cplx(18, 3, 1, fly=True)), ("multi-pass 2^17 16-bit", b16(17, 4, 2)),
        ("real / DCT-DST 2^10", special(10, 2)), ("real / DCT-DST 2^14", special(14, 4)),
        ("real / DCT-DST 2^17", special(17, 4)),
    ]


def test_debug_build_checks_every_shape(debug_lib):
    import torch

    from paper_1404_1810_gb300.amqft import amqft_debug_bounds, use_library

    checked = {}
    with use_library(debug_lib):
        is_checked, c0, _ = amqft_debug_bounds(clear=True)
        assert is_checked and c0 == 0
        for name, run in _cases(torch):
            out = run()
            ok, count, first = amqft_debug_bounds(clear=True)
            assert count == 0, f"{name}: {count} out-of-bounds accesses, first site {first >> 48} index {first & ((1 << 48) - 1)}"
            checked[name] = [t.clone() for t in out]
    # the release library: no checks, the same bits
    is_checked, c, _ = amqft_debug_bounds()
    assert not is_checked and c == 0
    for name, run in _cases(torch):
        for a, b in zip(run(), checked[name]):
            assert torch.equal(a, b), name
