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


def _run_d(exe, lines):
    """Harness lines with doubles; returns each result's hi + lo exactly and the pair."""
    out = subprocess.run([exe], input="".join(l + "\n" for l in lines), capture_output=True, text=True,
                         check=True).stdout.split("\n")
    res = []
    for line in out:
        if line.strip():
            h, l = line.split()
            hi, lo = _f(h), _f(l)
            res.append((Decimal(hi) + Decimal(lo) if np.isfinite(hi) and np.isfinite(lo) else None, hi, lo))
    return res


def _hx(v):
    return f"{struct.unpack('<Q', struct.pack('<d', float(v)))[0]:016x}"


def test_split_of_a_double_by_its_bits(harness):
    """df_from_double_bits: hi + lo equals the double to 2^-48 relative over the exponents it keeps, hi is the
    double rounded to FP32 up to one unit, and the edge cases (zeros, tiny, huge, infinities, NaN) map as stated."""
    rng = np.random.default_rng(11)
    n = 3000
    mant = 1.0 + rng.random(n)
    expo = rng.integers(-97, 128, n)
    sgn = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    vals = [float(s * m * 2.0 ** int(e)) for s, m, e in zip(sgn, mant, expo)]
    vals += [1.0 + 2.0 ** -52, 1.0 - 2.0 ** -53, 2.0 ** -97, 3.0e38, -2.0 ** 127 * (2 - 2.0 ** -23), 78.5 / 0.0625]
    got = _run_d(harness, [f"split {_hx(v)}" for v in vals])
    for v, (s, hi, lo) in zip(vals, got):
        V = Decimal(v)
        assert abs(s - V) <= abs(V) * Decimal(2) ** -48, v
        assert abs(Decimal(lo)) <= abs(Decimal(hi)) * Decimal(2) ** -24, v  # |lo| <= ulp(hi) / 2
        f32 = struct.unpack("<f", struct.pack("<f", v))[0]
        assert abs(Decimal(hi) - Decimal(f32)) <= abs(Decimal(f32)) * Decimal(2) ** -23, v
    # between 2^-126 and 2^-97 lo loses bits, within 2^-149 absolute
    small = [2.0 ** -100 * (1 + 2.0 ** -40), -2.0 ** -120 * 1.3, 2.0 ** -126]
    for v, (s, hi, lo) in zip(small, _run_d(harness, [f"split {_hx(v)}" for v in small])):
        assert abs(s - Decimal(v)) <= Decimal(2) ** -149, v
    edge = [0.0, -0.0, 5e-324, -1e-40, 1e39, -1e300, float("inf"), -float("inf"), float("nan"),
            -2.0 ** 127 * (2 - 2.0 ** -24)]
    got = _run_d(harness, [f"split {_hx(v)}" for v in edge])
    his = [hi for _, hi, _ in got]
    los = [lo for _, _, lo in got]
    assert his[:4] == [0.0, 0.0, 0.0, 0.0] and all(l == 0.0 for l in los[:8])
    assert np.copysign(1.0, his[1]) == -1.0 and np.copysign(1.0, his[3]) == -1.0  # signed zeros
    assert his[4] == float("inf") and his[5] == -float("inf") and his[6] == float("inf") and his[7] == -float("inf")
    assert np.isnan(his[8])
    assert his[9] == -float("inf")  # above the largest float plus half its unit, as the FP32 conversion rounds


def test_residual_row_in_double_float(harness):
    """df_residual_row against the exact residual of the FP64 inputs, on rows like the PF2 operator's near
    convergence (faces eps/h^2 of the two dielectrics, diagonal = sum of faces + kappa, b within 1e-6 of A x, so
    the sum cancels by six decades or more): error within 2^-43 of |b| + sum |f q| + |d x|."""
    rng = np.random.default_rng(12)
    lines, rows = [], []
    for i in range(2000):
        nk = 6 if i % 10 else int(rng.integers(0, 6))
        eps = np.where(rng.random(nk) < 0.8, 78.5, 2.0) * (1 + 1e-3 * rng.random(nk))
        f = eps / 0.0625 / (1 + rng.random(nk))
        x = float(rng.uniform(-8, 8))
        q = x + rng.normal(0, 0.05, nk)
        kap = float(rng.uniform(0, 50)) if i % 3 else 0.0
        d = float(f.sum() + kap)
        ax = d * x - float((f * q).sum())
        b = ax * (1 + float(rng.normal(0, 1e-6))) + float(rng.normal(0, 1e-9))
        rows.append((b, d, x, f, q))
        lines.append(f"row {nk} {_hx(b)} {_hx(d)} {_hx(x)} " + " ".join(f"{_hx(a)} {_hx(c)}" for a, c in zip(f, q)))
    got = _run_d(harness, lines)
    worst = Decimal(0)
    for (b, d, x, f, q), (s, _, _) in zip(rows, got):
        exact = Decimal(b) + sum(Decimal(float(a)) * Decimal(float(c)) for a, c in zip(f, q)) - Decimal(d) * Decimal(x)
        scale = abs(Decimal(b)) + sum(abs(Decimal(float(a)) * Decimal(float(c))) for a, c in zip(f, q)) + \
            abs(Decimal(d) * Decimal(x))
        worst = max(worst, abs(s - exact) / scale)
    assert worst < Decimal(2) ** -43, float(worst)
    # the cancellation these rows have: the residual is 1e-6..1e-10 of the scale, so FP32 alone would lose it
    # all while double-float keeps 3-7 significant digits of it
    b, d, x, f, q = rows[1]
    assert abs(Decimal(b) + sum(Decimal(float(a)) * Decimal(float(c)) for a, c in zip(f, q)) - Decimal(d) * Decimal(x)) \
        < Decimal(1e-5) * (abs(Decimal(d) * Decimal(x)))
