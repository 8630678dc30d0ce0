"""The double-float arithmetic of the CUDA pointwise step (paper_1711_04060_gb300/csrc/pf_df.cuh), built for
the host with g++ and checked against exact decimal arithmetic: the error-free transformations give sums
and products to about 2^-46 relative, and the table-driven exponential to about 1e-14 over the range the
Fermi step uses (arguments from -87 to +2)."""
import os
import struct
import subprocess
from decimal import Decimal, getcontext

import numpy as np
import pytest

from paper_1711_04060_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
getcontext().prec = 50


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    exe = tmp_path_factory.mktemp("df") / "df_harness"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-o", str(exe),
                           os.path.join(HERE, "df_harness.cpp"), "-lm"])
    return str(exe)


def _bits(x):
    return struct.unpack("<I", struct.pack("<f", x))[0]


def _f(u):
    return struct.unpack("<f", struct.pack("<I", int(u, 16)))[0]


def _split(v):
    """A double-float pair for the double v: hi = nearest float, lo = nearest float to the rest."""
    hi = struct.unpack("<f", struct.pack("<f", v))[0]
    lo = struct.unpack("<f", struct.pack("<f", v - hi))[0]
    return hi, lo


def _run(exe, rows):
    inp = "".join(f"{op} {_bits(a):08x} {_bits(b):08x} {_bits(c):08x} {_bits(d):08x}\n" for op, a, b, c, d in rows)
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    res = []
    for line in out:
        if line.strip():
            h, l = line.split()
            res.append(Decimal(_f(h)) + Decimal(_f(l)))
    return res


def test_df_exp_matches_exact_exponential(harness):
    xs = np.concatenate([W.uniform(W.substream(5, 1), 3000, -70.0, 2.0), W.uniform(W.substream(5, 2), 1000, -1.0, 1.0),
                         np.array([0.0, 1e-9, -1e-9, 0.0054, -0.0054, np.log(2.0) / 128, 1.0, -1.0, -69.9, 50.0])])
    rows = []
    exact = []
    for x in xs:
        hi, lo = _split(float(x) * (1.0 + 1e-9))  # a nonzero lo part as well
        rows.append(("exp", hi, lo, 0.0, 0.0))
        exact.append((Decimal(hi) + Decimal(lo)).exp())
    got = _run(harness, rows)
    rel = max(abs(g - e) / e for g, e in zip(got, exact))
    assert rel < 2e-14, float(rel)
    # below -70 the low part is subnormal: absolute accuracy far below the terms' resolution; 0 below -87
    xs = W.uniform(W.substream(5, 3), 500, -90.0, -70.0)
    rows = [("exp",) + _split(float(x)) + (0.0, 0.0) for x in xs]
    got = _run(harness, rows)
    for (op, hi, lo, _, __), g in zip(rows, got):
        e = (Decimal(hi) + Decimal(lo)).exp()
        assert abs(g - e) < Decimal(2) ** -125 and (g == 0 or hi >= -87.0)


def test_df_add_mul_error_free_enough(harness):
    a = W.uniform(W.substream(6, 1), 2000, -50.0, 50.0)
    b = W.uniform(W.substream(6, 2), 2000, -50.0, 50.0)
    rows, exact = [], []
    for x, y in zip(a, b):
        xh, xl = _split(float(x))
        yh, yl = _split(float(y) * 1.000001)
        X, Y = Decimal(xh) + Decimal(xl), Decimal(yh) + Decimal(yl)
        rows += [("add", xh, xl, yh, yl), ("mul", xh, xl, yh, yl), ("addf", xh, xl, yh, 0.0), ("mulf", xh, xl, yh, 0.0)]
        exact += [(X + Y, abs(X) + abs(Y)), (X * Y, abs(X * Y)), (X + Decimal(yh), abs(X) + abs(Decimal(yh))),
                  (X * Decimal(yh), abs(X * Decimal(yh)))]
    got = _run(harness, rows)
    worst = max(abs(g - e) / s for g, (e, s) in zip(got, exact) if s > 0)
    assert worst < 2 ** -44, float(worst)
    # cancellation: (x + y) - y recovers x to double-float accuracy
    xh, xl = _split(1.0 + 2 ** -30)
    s = _run(harness, [("add", xh, xl, -1.0, 0.0)])[0]
    assert abs(s - Decimal(2) ** -30) < Decimal(2) ** -70
