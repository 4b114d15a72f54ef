"""Pins of the CPU oracle against what the paper and the mathematics fix.

The oracle (``oracle/``) is the reference the CUDA path is compared with, so
it is checked here against things other than itself:
  * the textbook DFT (numpy's FFT as a library special case, closed forms),
  * the pruned DCT-0 / DST-0 definitions (Eq. qft_0B-0C) on every function
    of the recursion and every signal type of Tab. 1,
  * the defining identity of every M_v elaboration (Tab. 5-6) by brute force,
  * the exact operation counts the paper prints (Tab. 7-11),
  * the trig-constant budget (Sect. 7.1),
and deliberately planted mistakes must make these pins fail.
"""
import os

import numpy as np
import pytest

import synth

VARIANTS = list(range(1, 9))
COS_FAMILY = [1, 2, 3, 4]
SIN_FAMILY = [5, 6, 7, 8]
HERE = os.path.dirname(os.path.abspath(__file__))


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def turn_cos(q, m):
    """cos(2*pi*q/m) with q reduced mod m first (integer arrays)."""
    return np.cos(2.0 * np.pi * (np.mod(q, m) / m))


def turn_sin(q, m):
    return np.sin(2.0 * np.pi * (np.mod(q, m) / m))


# ---------------------------------------------------------------- textbook DFT

@pytest.mark.parametrize("log2n", range(0, 13))
def test_naive_dft_matches_library_fft(orc, log2n):
    n = 1 << log2n
    x = synth.uniform_complex(n, 1, config=1, stream=log2n)[0]
    assert rel(orc.naive_dft(x), np.fft.fft(x)) < 2e-15
    assert rel(orc.naive_dft(x, sign=+1), n * np.fft.ifft(x)) < 2e-15


@pytest.mark.parametrize("log2n", [3, 6, 10])
def test_naive_dft_closed_forms(orc, log2n):
    n = 1 << log2n
    k = np.arange(n)
    for n0 in (0, 1, n // 2 - 1, n - 1):
        x = np.zeros(n, complex)
        x[n0] = 1.0
        want = np.exp(-2j * np.pi * np.mod(n0 * k, n) / n)
        assert np.max(np.abs(orc.naive_dft(x) - want)) < 1e-15
    k0 = 3 % n
    tone = np.exp(2j * np.pi * np.mod(k0 * k, n) / n)
    want = np.zeros(n, complex)
    want[k0] = n
    assert np.max(np.abs(orc.naive_dft(tone) - want)) < 1e-12 * n


def test_dft_bin_matches_naive(orc):
    x = synth.uniform_complex(512, 1, stream=7)[0]
    full = orc.naive_dft(x)
    for k in (0, 1, 17, 255, 256, 511):
        assert abs(orc.dft_bin(x, k) - full[k]) < 1e-13


# ------------------------------------------------------------ whole transform

def fp64_bound(v, log2n):
    """Error bound of the fp64 recursion against the exact DFT.  Variants 5-8
    lose accuracy far faster (Sect. 7.3); the bound follows that growth."""
    if v in COS_FAMILY:
        return 5e-15 * max(1, log2n)
    return 1e-14 * 16.0 ** max(0, log2n - 6)


@pytest.mark.parametrize("v", VARIANTS)
@pytest.mark.parametrize("log2n", range(1, 11))
def test_amqft_f64_matches_naive(orc, v, log2n):
    n = 1 << log2n
    x = synth.uniform_complex(n, 1, config=1, stream=100 + log2n)[0]
    ref = orc.naive_dft(x)
    assert rel(orc.amqft(x, v), ref) < fp64_bound(v, log2n)
    assert rel(orc.amqft(x, v, sign=+1), orc.naive_dft(x, sign=+1)) < fp64_bound(v, log2n)


@pytest.mark.parametrize("v", COS_FAMILY)
def test_amqft_f64_matches_naive_4096(orc, v):
    x = synth.uniform_complex(4096, 1, stream=5)[0]
    assert rel(orc.amqft(x, v), orc.naive_dft(x)) < 1e-14


@pytest.mark.parametrize("v", [2, 4])
def test_amqft_spot_bins_large(orc, v):
    n = 1 << 15
    x = synth.normal_complex(n, 1, stream=3)[0]
    y = orc.amqft(x, v)
    scale = np.sqrt(n)
    for k in (0, 1, 2, 3, n // 4, n // 2, n // 2 + 1, n - 1, 12345):
        assert abs(y[k] - orc.dft_bin(x, k)) < 1e-12 * scale


@pytest.mark.parametrize("v", VARIANTS)
@pytest.mark.parametrize("log2n", [2, 5, 8])
def test_amqft_closed_forms(orc, v, log2n):
    n = 1 << log2n
    k = np.arange(n)
    tol = 1e-13 if v in COS_FAMILY else 1e-11
    for n0 in (0, 1, n - 1):
        x = np.zeros(n, complex)
        x[n0] = 1.0
        want = np.exp(-2j * np.pi * np.mod(n0 * k, n) / n)
        assert np.max(np.abs(orc.amqft(x, v) - want)) < tol, ("impulse", n0)
    assert np.max(np.abs(orc.amqft(np.ones(n, complex), v) - n * (k == 0))) < tol * n
    for k0 in (1, n // 2 - 1 if n > 2 else 1, n - 1):
        tone = np.exp(2j * np.pi * np.mod(k0 * k, n) / n)
        assert np.max(np.abs(orc.amqft(tone, v) - n * (k == k0))) < tol * n, ("tone", k0)


@pytest.mark.parametrize("v", VARIANTS)
def test_amqft_parseval_linearity_inverse(orc, v):
    n = 256
    x = synth.normal_complex(n, 2, stream=11)
    a, b = 0.75 - 0.5j, -1.25 + 2.0j
    tol = 1e-13 if v in COS_FAMILY else 1e-10
    X0, X1 = orc.amqft(x[0], v), orc.amqft(x[1], v)
    assert abs(np.sum(np.abs(X0) ** 2) - n * np.sum(np.abs(x[0]) ** 2)) < tol * n * np.sum(np.abs(x[0]) ** 2)
    assert rel(orc.amqft(a * x[0] + b * x[1], v), a * X0 + b * X1) < tol
    assert rel(orc.amqft(X0, v, sign=+1), n * x[0]) < tol


@pytest.mark.parametrize("v", VARIANTS)
def test_long_double_instantiation(orc, v):
    n = 256
    x = synth.uniform_complex(n, 1, stream=21)[0]
    ref = orc.naive_dft(x)
    e_ld = rel(orc.amqft(x, v, prec="ld"), ref)
    e_64 = rel(orc.amqft(x, v, prec="f64"), ref)
    assert e_ld <= max(e_64, 2e-16)
    assert e_ld < (5e-16 if v in COS_FAMILY else 1e-14)


@pytest.mark.parametrize("v", VARIANTS)
def test_f32_instantiation_small(orc, v):
    n = 64
    x = synth.uniform_complex(n, 1, stream=31)[0].astype(np.complex64).astype(np.complex128)
    assert rel(orc.amqft(x, v, prec="f32"), orc.naive_dft(x)) < 1e-6


# ---------------------------------------------- single functions, Tab. 1 types

def pruned(kind, m, s):
    """Brute-force DCT-0 / DST-0 (Eq. qft_0B-0C) restricted to the sto_n and
    sto_k sets of Tab. 1 for the signal type each function takes."""
    q = m // 4
    tables = {
        "dct": (np.arange(0, m // 2 + 1), np.arange(0, m // 2 + 1), "c"),
        "dst": (np.arange(1, m // 2), np.arange(1, m // 2), "s"),
        "dct_ot": (np.arange(1, m // 2, 2), np.arange(0, q), "c"),
        "dst_ot": (np.arange(1, m // 2, 2), np.arange(1, q + 1), "s"),
        "dct_to": (np.arange(0, q), np.arange(1, m // 2, 2), "c"),
        "dst_to": (np.arange(1, q + 1), np.arange(1, m // 2, 2), "s"),
        "dct_oo": (np.arange(1, q, 2), np.arange(1, q, 2), "c"),
        "dst_oo": (np.arange(1, q, 2), np.arange(1, q, 2), "s"),
    }
    ns, ks, f = tables[kind]
    trig = turn_cos if f == "c" else turn_sin
    return np.array([np.sum(s * trig(ns * k, m)) for k in ks])


OT_KINDS = ["dct", "dst", "dct_ot", "dst_ot", "dct_oo", "dst_oo"]
TO_KINDS = ["dct", "dst", "dct_to", "dst_to", "dct_oo", "dst_oo"]


@pytest.mark.parametrize("v", VARIANTS)
@pytest.mark.parametrize("log2m", range(2, 9))
def test_functions_against_pruned_definitions(orc, v, log2m):
    m = 1 << log2m
    kinds = OT_KINDS if v in (1, 4, 5, 8) else TO_KINDS
    tol = 1e-13 if v in COS_FAMILY else 1e-11
    for kind in kinds:
        if kind.endswith("_oo") and m < 8:
            continue
        if kind == "dst" and m < 4:
            continue
        nin, _ = orc.sub_sizes(kind, m)
        x = synth.uniform_complex(nin, 1, stream=log2m * 10 + v)[0].real
        got = orc.sub(kind, v, log2m, x)
        want = pruned(kind, m, x)
        assert np.max(np.abs(got - want)) < tol * max(1.0, np.max(np.abs(want))), kind


@pytest.mark.parametrize("log2m", range(1, 9))
def test_rdft_against_library(orc, log2m):
    m = 1 << log2m
    x = synth.uniform_complex(m, 1, stream=40 + log2m)[0].real
    r = np.fft.rfft(x)
    for v in VARIANTS:
        tol = 1e-12 if v in COS_FAMILY else 1e-12 * 16.0 ** max(0, log2m - 6)
        got = orc.sub("rdft", v, log2m, x)
        assert np.max(np.abs(got[: m // 2 + 1] - r.real)) < tol
        if m >= 4:
            assert np.max(np.abs(got[m // 2 + 1:] - r.imag[1: m // 2])) < tol


# --------------------------------------------------- M_v identities (Tab. 5-6)

def child_type(v, ctx):
    """(transform of the child, child sto_n, child sto_k) of M_v (Tab. 5-6)."""
    child_ctx = ctx if v <= 4 else 1 - ctx
    oe = v in (1, 4, 5, 8)
    return child_ctx, oe


@pytest.mark.parametrize("v", VARIANTS)
@pytest.mark.parametrize("ctx", [0, 1])
@pytest.mark.parametrize("log2m", range(4, 10))
def test_mv_identities_by_brute_force(orc, v, ctx, log2m):
    m = 1 << log2m
    q = m // 4
    x = synth.uniform_complex(m // 8, 1, stream=1000 + 16 * v + log2m + 8 * ctx)[0].real
    n_x = np.arange(1, q, 2)
    k_odd = np.arange(1, q, 2)
    trig_x = turn_cos if ctx == 0 else turn_sin
    o_true = np.array([np.sum(x * trig_x(n_x * k, m)) for k in k_odd])
    y = orc.mv_time(v, ctx, log2m, x)
    child_ctx, oe = child_type(v, ctx)
    if oe:                       # s_oe: n odd < M/4; even harmonics
        n_y = np.arange(1, q, 2)
        k_y = np.arange(0, q - 1, 2) if child_ctx == 0 else np.arange(2, q + 1, 2)
    else:                        # s_eo: even n; odd harmonics
        n_y = np.arange(0, q - 1, 2) if child_ctx == 0 else np.arange(2, q + 1, 2)
        k_y = np.arange(1, q, 2)
    trig_y = turn_cos if child_ctx == 0 else turn_sin
    e_true = np.array([np.sum(y * trig_y(n_y * k, m)) for k in k_y])
    o = orc.mv_freq(v, ctx, log2m, e_true)
    assert np.max(np.abs(o - o_true)) < 1e-11 * max(1.0, np.max(np.abs(o_true))) * (1 if v <= 4 else m)


# ----------------------------------------------------- operation counts (Sect. 7)

def tab7(kind, n):
    lg = n.bit_length() - 1
    f = {
        "cdft": (n * lg - 3 * n + 4, 3 * n * lg - 3 * n + 4, n - 4 * lg + 4),
        "rdft": (n * lg // 2 - 3 * n // 2 + 2, 3 * n * lg // 2 - 5 * n // 2 + 4, n // 2 - 2 * lg + 2),
        "dct": (n * lg // 4 - 3 * n // 4 + 1, 3 * n * lg // 4 - 7 * n // 4 + lg + 3, n // 4 - lg + 1),
        "dst": (n * lg // 4 - 3 * n // 4 + 1, 3 * n * lg // 4 - 7 * n // 4 - lg + 3, n // 4 - lg + 1),
    }[kind]
    return {"mults": f[0], "sums": f[1], "halvings": f[2]}


@pytest.mark.parametrize("v", VARIANTS)
@pytest.mark.parametrize("kind", ["cdft", "rdft", "dct", "dst"])
def test_tally_matches_tab7(orc, v, kind):
    for log2n in range(2, 15):
        n = 1 << log2n
        sums, mults, halvings = orc.tally(v, log2n, kind)
        want = tab7(kind, n)
        assert sums == want["sums"], (n, "sums")
        assert mults == want["mults"], (n, "mults")
        assert halvings == (want["halvings"] if v in (1, 3, 5, 7) else 0), (n, "halvings")


def load_golden_counts():
    rows = []
    with open(os.path.join(HERE, "golden", "cdft_counts_var_qft.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(tuple(int(t) for t in line.split()))
    return rows


@pytest.mark.parametrize("v", VARIANTS)
def test_tally_matches_tab9_to_tab11(orc, v):
    rows = load_golden_counts()
    assert len(rows) == 10
    for n, sums, mults, flop_a, flop_b in rows:
        s, m, h = orc.tally(v, n.bit_length() - 1)
        assert (s, m) == (sums, mults), n
        assert s + m == flop_a, n
        if v in (1, 3, 5, 7):
            assert s + m + h == flop_b, n


@pytest.mark.parametrize("v", VARIANTS)
@pytest.mark.parametrize("log2n", [3, 4, 6, 10, 13])
def test_constant_budget(orc, v, log2n):
    n = 1 << log2n
    q = orc.angles(v, log2n)
    # N/4 - 1 stored angles (p = 1..N/4-1) plus the common cos(pi/4), which is
    # the p = N/8 angle, Sect. 7.1: N/4 - 1 distinct angles in total
    assert list(q) == list(range(1, n // 4))


# ------------------------------------------------------- planted mistakes

@pytest.mark.parametrize("fault,v,log2n", [
    ("dc_misprint", 4, 4), ("dr_sign", 2, 4), ("dk_drop", 4, 5), ("m4_neighbour", 4, 6),
    ("const_index", 2, 6), ("dn_sign", 4, 4), ("m1_halving", 1, 4),
])
def test_planted_mistakes_are_caught(orc, fault, v, log2n):
    n = 1 << log2n
    x = synth.uniform_complex(n, 1, stream=77)[0]
    ref = orc.naive_dft(x)
    assert rel(orc.amqft(x, v), ref) < 1e-14
    with orc.fault(fault):
        bad = orc.amqft(x, v)
    assert rel(bad, ref) > 1e-3
    assert rel(orc.amqft(x, v), ref) < 1e-14


def test_accuracy_ordering_sine_family_worse(orc):
    """Sect. 7.3 reports that the sine variants (5-8) lose accuracy far
    faster than the cosine ones (1-4).  Measured here in fp64 at N = 1024."""
    n = 1024
    x = synth.uniform_complex(n, 1, stream=123)[0]
    ref = orc.naive_dft(x)
    err = {v: rel(orc.amqft(x, v), ref) for v in VARIANTS}
    assert max(err[v] for v in COS_FAMILY) * 100 < min(err[v] for v in SIN_FAMILY)
