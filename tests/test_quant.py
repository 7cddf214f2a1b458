"""The host rounding of weights to E4M3 and BF16 (tensor-core weight images),
checked exhaustively on the CPU against the formats' definitions: E4M3 has a
sign bit, 4 exponent bits (bias 7) and 3 mantissa bits, subnormals below
2^-6, largest finite value 448 and no infinities; rounding is to nearest with
ties to the even code, saturating."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2508_12117_gb300", "csrc")


@pytest.fixture(scope="module")
def q(tmp_path_factory):
    d = tmp_path_factory.mktemp("quant")
    so = str(d / "quant_harness.so")
    subprocess.run(["g++", "-O2", "-fPIC", "-shared", "-std=c++17", "-I", CSRC,
                    os.path.join(ROOT, "tests", "host", "quant_harness.cpp"), "-o", so],
                   check=True, capture_output=True)
    L = C.CDLL(so)
    L.quant_e4m3.restype = C.c_uint8
    L.quant_e4m3.argtypes = [C.c_float]
    L.quant_bf16.restype = C.c_uint16
    L.quant_bf16.argtypes = [C.c_float]
    return L


def e4m3_value(b):
    s = -1.0 if b & 0x80 else 1.0
    e, m = (b >> 3) & 15, b & 7
    if e == 15 and m == 7:
        return float("nan")
    if e == 0:
        return s * m * 2.0 ** -9
    return s * (1 + m / 8.0) * 2.0 ** (e - 7)


def test_e4m3_roundtrip_every_code(q):
    for b in range(256):
        v = e4m3_value(b)
        if np.isnan(v):
            continue
        assert q.quant_e4m3(v) == b, (b, v)


def test_e4m3_ties_to_even_and_between(q):
    pos = sorted({e4m3_value(b) for b in range(128) if not np.isnan(e4m3_value(b))})
    assert pos[0] == 0.0 and pos[-1] == 448.0 and len(pos) == 127
    for lo, hi in zip(pos[:-1], pos[1:]):
        blo, bhi = q.quant_e4m3(lo), q.quant_e4m3(hi)
        mid = np.float32((lo + hi) / 2)
        if float(mid) == (lo + hi) / 2:       # exact tie in FP32
            want = blo if (blo & 1) == 0 else bhi
            assert q.quant_e4m3(float(mid)) == want, (lo, hi)
        below = float(np.nextafter(np.float32((lo + hi) / 2), np.float32(-1)))
        above = float(np.nextafter(np.float32((lo + hi) / 2), np.float32(1e9)))
        if lo < below < (lo + hi) / 2:
            assert q.quant_e4m3(below) == blo
        if (lo + hi) / 2 < above < hi:
            assert q.quant_e4m3(above) == bhi
        assert q.quant_e4m3(-hi) == bhi | 0x80


def test_e4m3_saturates_and_nan(q):
    for v in (448.0, 449.0, 464.0, 500.0, 1e6, float("inf")):
        assert q.quant_e4m3(v) == 0x7E
        assert q.quant_e4m3(-v) == 0xFE
    assert q.quant_e4m3(float("nan")) & 0x7F == 0x7F
    assert q.quant_e4m3(2.0 ** -10) == 0          # tie between 0 and 2^-9: even code 0
    assert q.quant_e4m3(1.5 * 2.0 ** -10) == 1


def test_bf16_round_to_nearest_even(q):
    rng = np.random.default_rng(1)
    x = rng.standard_normal(20000).astype(np.float32) * np.float32(10.0) ** rng.integers(-8, 8, 20000)
    for v in x[:2000]:
        b = q.quant_bf16(float(v))
        got = np.array([b << 16], np.uint32).view(np.float32)[0]
        # the BF16 neighbours of v
        u = np.array([v], np.float32).view(np.uint32)[0]
        lo = np.array([u & 0xFFFF0000], np.uint32).view(np.float32)[0]
        hi = np.array([(u & 0xFFFF0000) + 0x10000], np.uint32).view(np.float32)[0]
        dlo, dhi = abs(float(v) - float(lo)), abs(float(hi) - float(v))
        if dlo < dhi:
            assert got == lo
        elif dhi < dlo:
            assert got == hi
        else:
            assert (np.array([got], np.float32).view(np.uint32)[0] >> 16) & 1 == 0


def _bf16_value(q, v):
    b = int(q.quant_bf16(float(v)))
    return float(np.frombuffer(np.array([b << 16], np.uint32).tobytes(), np.float32)[0])


def test_bf16_split_first_layer_bound(q):
    """The BF16 tensor-core form's first layer: each FP32 operand v is split into
    BF16 values v_hi = bf16(v), v_lo = bf16(v - v_hi), and the K = 18 product
    [x_hi, x_lo, x_hi] . [W_hi, W_hi, W_lo] stands for W1 x.  With round to
    nearest, |v - v_hi - v_lo| <= 2^-18 |v| and the dropped x_lo W_lo is at most
    2^-18 |x W|, so every term is within 3 * 2^-18 < 2^-15 of x W (products of
    BF16 values are exact in FP32).  Checked on the network inputs of the
    synthetic catalogs (coordinates in km) and the seeded first-layer weights."""
    from paper_2508_12117_gb300 import synth
    net = synth.mlp_weights(256, 811)
    W = net["W"][0]                                      # (H, 6), FP32
    rng = np.random.default_rng(5)
    n = 400
    src = np.c_[rng.uniform(0, 60, n), rng.uniform(0, 60, n), rng.uniform(2, 16, n)]
    rcv = np.c_[rng.uniform(-10, 70, n), rng.uniform(-10, 70, n), np.zeros(n)]
    x = np.c_[src, rcv].astype(np.float32)

    def split(a):
        hi = np.vectorize(lambda v: _bf16_value(q, v))(a).astype(np.float32)
        lo = np.vectorize(lambda v: _bf16_value(q, v))((a - hi).astype(np.float32)).astype(np.float32)
        return hi.astype(np.float64), lo.astype(np.float64)

    xh, xl = split(x)
    wh, wl = split(W)
    exact = x.astype(np.float64) @ W.T.astype(np.float64)
    approx = xh @ wh.T + xl @ wh.T + xh @ wl.T
    scale = np.abs(x.astype(np.float64)) @ np.abs(W.T.astype(np.float64))
    assert np.all(np.abs(approx - exact) <= 2.0 ** -15 * scale)
    # and a plain BF16 product (no split) would not meet it
    assert np.max(np.abs(xh @ wh.T - exact) / scale) > 2.0 ** -12
