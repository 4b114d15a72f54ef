"""Real input (amqft_exec_rdft): pairs of real signals share one complex
transform, on the fused kernels and (above 2^16) the multi-pass path.  Every harmonic 0 .. N/2 must equal the complex transform of the
signal with a zero imaginary part (same kernels, same float32 operations),
and the float64 reference within the float32 recursion's error."""
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


CASES = [(0, 4, 3), (1, 4, 2), (2, 2, 5), (3, 1, 4), (5, 8, 7), (10, 4, 9), (10, 3, 6), (12, 6, 3), (13, 4, 4),
         (14, 4, 3), (14, 2, 2), (15, 1, 5), (16, 4, 3), (16, 7, 2)]


@pytest.mark.parametrize("log2n,v,b", CASES)
def test_rdft_equals_complex_path(log2n, v, b):
    import torch

    from paper_1404_1810_gb300 import Plan

    n = 1 << log2n
    xr = torch.from_numpy(synth.real_signals(n, b, stream=log2n + 10 * v).astype(np.float32)).cuda()
    p = Plan(log2n, v, b)
    try:
        r = p.rdft(xr)
        full = p.fwd(torch.complex(xr, torch.zeros_like(xr)).contiguous())
        torch.cuda.synchronize()
        assert torch.equal(r, full[:, : n // 2 + 1]), (log2n, v, b)
    finally:
        p.close()


@pytest.mark.parametrize("log2n,v", [(10, 4), (13, 2), (16, 4)])
def test_rdft_against_float64(orc, log2n, v):
    import torch

    from paper_1404_1810_gb300 import Plan

    n, b = 1 << log2n, 3
    x = synth.real_signals(n, b, stream=77).astype(np.float32)
    p = Plan(log2n, v, b)
    try:
        r = p.rdft(torch.from_numpy(x).cuda()).cpu().numpy()
    finally:
        p.close()
    for i in range(b):
        ref = np.fft.rfft(x[i].astype(np.float64))
        r32 = orc.amqft(x[i].astype(np.complex128), v, prec="f32")[: n // 2 + 1]
        assert rel(r[i], ref) <= derived_tol(rel(r32, ref), log2n)


@pytest.mark.parametrize("log2n,v", [(17, 4), (18, 1), (17, 6)])
def test_rdft_multipass_equals_complex_path(log2n, v):
    """Above 2^16 the real input runs on the multi-pass path: still every
    harmonic of the complex transform of the zero-imaginary signal."""
    import torch

    from paper_1404_1810_gb300 import Plan

    n, b = 1 << log2n, 3
    xr = torch.from_numpy(synth.real_signals(n, b, stream=log2n + 10 * v).astype(np.float32)).cuda()
    p = Plan(log2n, v, b)
    try:
        r = p.rdft(xr)
        full = p.fwd(torch.complex(xr, torch.zeros_like(xr)).contiguous())
        torch.cuda.synchronize()
        assert torch.equal(r, full[:, : n // 2 + 1]), (log2n, v)
    finally:
        p.close()
