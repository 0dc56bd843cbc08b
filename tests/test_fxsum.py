"""The fixed-point neighbour sums of csrc/fxsum.cuh (host build of the same
header the kernels include), against exact rational arithmetic: the
(2D+1)-point operator's sum of the 2D face neighbours (Eq. 5, Sec. 3.1) and
the same sum less 2D times the centre value.

Pins: (1) terms whose exponents lie within the guard bits of the largest
are aligned without loss, so the result equals the correctly rounded exact
sum (Python's Fraction -> float rounds to nearest-even); (2) in general the
error is at most half an ulp of the result plus the truncation bound, one
unit of 2^-G ulp(largest term) per unit of weight; (3) zeros and subnormals
beside normal terms contribute exactly nothing beyond their value; (4) the
unhandled range (all terms tiny, near overflow, inf, NaN) is reported, not
computed."""
import math
import os
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fxhost(tmp_path_factory):
    d = tmp_path_factory.mktemp("fx")
    exe = str(d / "fxsum_host")
    subprocess.run(["g++", "-O2", "-std=c++17", "-o", exe, os.path.join(ROOT, "tests", "fxsum_host.cpp")],
                   check=True)

    def run(x, K, C):
        x = np.ascontiguousarray(x, dtype=np.float64)
        assert x.shape[1] == K + 1
        fin, fout = str(d / "in.bin"), str(d / "out.bin")
        x.tofile(fin)
        subprocess.run([exe, str(K), str(C), fin, fout], check=True)
        raw = open(fout, "rb").read()
        n = x.shape[0]
        return np.frombuffer(raw[:8 * n], np.float64), np.frombuffer(raw[8 * n:], np.uint8).astype(bool)
    return run


def headroom(w):
    return 1 if w <= 2 else 2 if w <= 4 else 3 if w <= 8 else 4 if w <= 16 else 5


def exact(row, K, C):
    return sum(Fraction(float(v)) for v in row[:K]) - C * Fraction(float(row[K]))


def ulp(v):
    return math.ulp(v) if v != 0 else 0.0


def trunc_bound(row, K, C):
    G = 63 - headroom(K + C) - 53
    terms = list(row[:K]) + ([row[K]] if C else [])
    E = max((np.float64(t).view(np.uint64) >> np.uint64(52)) & np.uint64(0x7FF) for t in terms)
    return Fraction(K + C) * Fraction(2) ** (int(E) - 1075 - G)


CASES = [(2, 0), (3, 0), (4, 0), (6, 0), (4, 4), (6, 6)]


@pytest.mark.parametrize("K,C", CASES)
def test_close_exponents_are_correctly_rounded(fxhost, K, C):
    rng = np.random.default_rng(11 + K + C)
    n = 4000
    # terms within a factor 2^G of one another: no bit leaves the window
    G = 63 - headroom(K + C) - 53
    mant = rng.uniform(1.0, 2.0, size=(n, K + 1))
    expo = rng.integers(0, G, size=(n, K + 1)) + rng.integers(-40, 40, size=(n, 1))
    sign = rng.choice([-1.0, 1.0], size=(n, K + 1))
    x = sign * np.ldexp(mant, expo)
    s, ok = fxhost(x, K, C)
    assert ok.all()
    for i in range(n):
        assert s[i] == float(exact(x[i], K, C)), (x[i], s[i])


@pytest.mark.parametrize("K,C", CASES)
def test_wide_exponents_within_bound(fxhost, K, C):
    rng = np.random.default_rng(21 + K + C)
    n = 4000
    mant = rng.uniform(1.0, 2.0, size=(n, K + 1))
    expo = rng.integers(-70, 70, size=(n, K + 1))
    sign = rng.choice([-1.0, 1.0], size=(n, K + 1))
    x = sign * np.ldexp(mant, expo)
    # exact cancellation in some rows: the result may be tiny or zero
    x[::7, 1] = -x[::7, 0]
    s, ok = fxhost(x, K, C)
    assert ok.all()
    worst = worst64 = 0.0
    for i in range(n):
        ex = exact(x[i], K, C)
        err = abs(Fraction(float(s[i])) - ex)
        bound = Fraction(ulp(float(ex))) / 2 + trunc_bound(x[i], K, C)
        assert err <= bound, (x[i], s[i], float(ex))
        big = max(abs(float(v)) for v in list(x[i, :K]) + [C * x[i, K]])
        worst = max(worst, float(err) / big)
        acc = float(x[i, 0])                 # recursive FP64 summation of the same terms
        for k in range(1, K):
            acc += float(x[i, k])
        if C:
            acc -= C * float(x[i, K])
        worst64 = max(worst64, float(abs(Fraction(acc) - ex)) / big)
    # relative to the largest term, no worse than adding in FP64 (both include
    # the final rounding of a result up to K + C times the largest term)
    assert worst <= worst64


@pytest.mark.parametrize("K,C", CASES)
def test_ties_round_to_even_and_cancellation(fxhost, K, C):
    # 1 + 2^-53 is a tie between 1 and 1 + 2^-52: nearest-even gives 1;
    # 1 + 2^-52 + 2^-53 ties to 1 + 2^-51
    rows = []
    z = [0.0] * (K + 1)
    r = list(z); r[0], r[1] = 1.0, 2.0 ** -53; rows.append(r)
    r = list(z); r[0], r[1], r[2] = 1.0, 2.0 ** -52, 2.0 ** -53; rows.append(r)
    r = list(z); r[0], r[1], r[2] = -1.0, -(2.0 ** -52), -(2.0 ** -53); rows.append(r)
    r = list(z); r[0], r[1] = 1.5, -1.5; rows.append(r)                     # exact zero
    r = list(z); r[0], r[1], r[2] = 1.0, -1.0 + 2.0 ** -52, 2.0 ** -55; rows.append(r)  # deep cancellation
    x = np.array(rows)
    if K < 3:   # rows 1, 2 and 4 need three terms
        x = x[[0, 3]]
        s, ok = fxhost(x, K, C)
        assert ok.all() and s[0] == 1.0 and s[1] == 0.0
        return
    s, ok = fxhost(x, K, C)
    assert ok.all()
    assert s[0] == 1.0
    assert s[1] == 1.0 + 2.0 ** -51
    assert s[2] == -(1.0 + 2.0 ** -51)
    assert s[3] == 0.0
    assert s[4] == float(exact(x[4], K, C))


@pytest.mark.parametrize("K,C", CASES)
def test_zero_and_subnormal_terms(fxhost, K, C):
    rng = np.random.default_rng(31 + K)
    n = 500
    x = rng.normal(size=(n, K + 1))                     # x[:, 0] stays a normal term
    for k in range(1, K):                               # zeros, negative zeros and subnormals
        x[k % 3::3, k] = 0.0
        x[(k + 1) % 3::3, k] = -0.0
        x[(k + 2) % 3::3, k] = 5e-324 * rng.integers(1, 1000, size=len(x[(k + 2) % 3::3]))
    s, ok = fxhost(x, K, C)
    assert ok.all()
    for i in range(n):
        ex = exact(x[i], K, C)
        assert abs(Fraction(float(s[i])) - ex) <= Fraction(ulp(float(ex))) / 2 + trunc_bound(x[i], K, C)


@pytest.mark.parametrize("K,C", CASES)
def test_unhandled_range_is_reported(fxhost, K, C):
    z = [0.0] * (K + 1)
    rows = [list(z)]                                   # all zero: caller adds in FP64
    r = list(z); r[0] = 1e-300; rows.append(r)         # largest term below 2^-959
    r = list(z); r[0] = 1e308; rows.append(r)          # near overflow
    r = list(z); r[0] = math.inf; rows.append(r)
    r = list(z); r[0] = math.nan; rows.append(r)
    r = list(z); r[0] = 1.0; r[1] = math.inf; rows.append(r)
    s, ok = fxhost(np.array(rows), K, C)
    assert not ok.any()
    # the edges of the handled range: 2^-959 (biased exponent 64) and 2^1017 (2040)
    r1 = list(z); r1[0] = 2.0 ** -959; r1[1] = 2.0 ** -960
    r2 = list(z); r2[0] = 2.0 ** 1017; r2[1] = -(2.0 ** 1016)
    s, ok = fxhost(np.array([r1, r2]), K, C)
    assert ok.all()
    assert s[0] == 1.5 * 2.0 ** -959 and s[1] == 2.0 ** 1016
