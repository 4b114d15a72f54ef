"""The paired-region kernel's index logic on the CPU: its stages (written
against a context, amqft_paired.cuh) run in a host emulation of one cluster,
every GPU thread a host thread, built with AddressSanitizer.  The result must
be bit-identical to the oracle's float32 recursion (variant 4), and no access
may leave a region, a constant table or a buffer.  This covers the kernel's
indexing without a GPU; the GPU parity tests cover the kernel itself."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import synth

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1404_1810_gb300", "csrc")


def _cuda_include():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return os.path.join(os.path.dirname(os.path.dirname(nvcc)), "include")


@pytest.fixture(scope="module")
def emu_binary(tmp_path_factory):
    def build(log2n):
        out = str(tmp_path_factory.mktemp("emu") / f"paired_emu_{log2n}")
        cmd = ["g++", "-std=c++20", "-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
               "-ffp-contract=off", f"-DPAIRED_LN={log2n}", "-I" + _cuda_include(), "-I" + CSRC,
               "-I" + os.path.join(ROOT, "include"), os.path.join(HERE, "paired_emu.cpp"), "-o", out, "-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            pytest.skip(f"host compiler could not build the emulation: {r.stderr[-400:]}")
        return out
    return build


def _run(orc, binary, log2n, batch, inverse, tmp_path, listed=False):
    n = 1 << log2n
    x = synth.normal_complex(n, batch, config=2, stream=700 + log2n).astype(np.complex64)
    fi, fo = str(tmp_path / "in.bin"), str(tmp_path / "out.bin")
    x.tofile(fi)
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=0:detect_stack_use_after_return=0")
    r = subprocess.run([binary, str(int(inverse)), str(-batch if listed else batch), fi, fo], capture_output=True,
                       text=True, env=env, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    y = np.fromfile(fo, dtype=np.complex64).reshape(batch, n)
    sign = +1 if inverse else -1
    for b in range(batch):
        ref = orc.amqft(x[b].astype(np.complex128), 4, prec="f32", sign=sign).astype(np.complex64)
        assert np.array_equal(y[b], ref), (log2n, inverse, b)


@pytest.mark.parametrize("inverse", [False, True])
def test_paired_emulation_2e14(orc, emu_binary, inverse, tmp_path):
    _run(orc, emu_binary(14), 14, 3, inverse, tmp_path)


@pytest.mark.slow
@pytest.mark.parametrize("log2n", [15, 16])
def test_paired_emulation_larger(orc, emu_binary, log2n, tmp_path):
    _run(orc, emu_binary(log2n), log2n, 2, log2n == 16, tmp_path)


def _run16(orc, binary, log2n, batch, dt, tmp_path):
    """16-bit storage (dt 1 bf16, 3 int16): forward from exponent-0 input,
    then the inverse of that output with its exponents; every value and
    exponent must equal the oracle's float32 recursion rounded the same way."""
    import torch

    from gpu_util import expected_exponent

    n = 1 << log2n
    x = synth.normal_complex(n, batch, config=2, stream=720 + log2n)
    t = torch.view_as_real(torch.from_numpy(np.ascontiguousarray(x)))
    to16 = (lambda v: (v * 4096.0).round().to(torch.int16)) if dt == 3 else (lambda v: v.to(torch.bfloat16))
    x16 = to16(t).contiguous()
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=0:detect_stack_use_after_return=0")
    e_in = np.zeros(batch, dtype=np.int32)
    for inverse in (False, True):
        fi, fo = str(tmp_path / "in16.bin"), str(tmp_path / "out16.bin")
        ei, eo = str(tmp_path / "ein.bin"), str(tmp_path / "eout.bin")
        x16.view(torch.int16).numpy().tofile(fi)
        e_in.tofile(ei)
        r = subprocess.run([binary, str(int(inverse)), str(batch), fi, fo, str(dt), ei, eo], capture_output=True,
                           text=True, env=env, timeout=900)
        assert r.returncode == 0, r.stderr[-2000:]
        y16 = torch.from_numpy(np.fromfile(fo, dtype=np.int16).reshape(batch, n, 2).copy())
        e_out = np.fromfile(eo, dtype=np.int32)
        xin = torch.view_as_complex(x16.double().contiguous()).numpy() * (2.0 ** e_in)[:, None]
        for b in range(batch):
            r32 = orc.amqft(xin[b], 4, prec="f32", sign=+1 if inverse else -1).astype(np.complex64)
            ee = expected_exponent(r32)
            assert int(e_out[b]) == ee, (dt, inverse, b, int(e_out[b]), ee)
            scaled = torch.view_as_real(torch.from_numpy((r32 * np.float32(2.0 ** -ee)).astype(np.complex64)))
            want = (scaled.round().to(torch.int16) if dt == 3 else scaled.to(torch.bfloat16)).view(torch.int16)
            assert torch.equal(y16[b], want), (dt, inverse, b)
        x16 = y16.view(torch.bfloat16) if dt == 1 else y16
        e_in = e_out.astype(np.int32)


@pytest.mark.parametrize("dt", [1, 3])
def test_paired_emulation_16bit(orc, emu_binary, dt, tmp_path):
    _run16(orc, emu_binary(14), 14, 2, dt, tmp_path)


def test_paired_emulation_transform_list(orc, emu_binary, tmp_path):
    """The ragged form: transforms taken through a list (reversed order,
    a capacity above the count read from device memory)."""
    _run(orc, emu_binary(14), 14, 3, False, tmp_path, listed=True)
