"""The FP64 stencil neighbour sum in 64-bit fixed point (csrc/fxsum.h),
compiled for the host with g++ and checked against exact rational sums
(no GPU): the error stays within K units of 2^(emax - 1081) plus half an ulp
of the result on random, widely spread, cancelling, subnormal-carrying and
signed operands; operands of one binade (nothing dropped) give the correctly
rounded sum; out-of-range operands (zeros only, tiny, huge, Inf, NaN) give
the plain FP64 additions bit for bit."""
import math
import os
import shutil
import struct
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fx(tmp_path_factory):
    if not shutil.which("g++"):
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("fx")
    src = d / "fx.cpp"
    src.write_text(r'''
#include <cstdio>
#include <cstdint>
#include <cstring>
#include "fxsum.h"
using namespace plcg;
static double rd(FILE *f) { unsigned long long u; if (fscanf(f, "%llx", &u) != 1) return 0; double x; memcpy(&x, &u, 8); return x; }
static void wr(double x) { unsigned long long u; memcpy(&u, &x, 8); printf("%016llx\n", u); }
int main() {
    int k;
    while (scanf("%d", &k) == 1) {
        double v[8];
        for (int i = 0; i < k; ++i) v[i] = rd(stdin);
        if (k == 4) { double x[4]; memcpy(x, v, sizeof x); wr(fx_sum<4>(x)); }
        else if (k == 6) { double x[6]; memcpy(x, v, sizeof x); wr(fx_sum<6>(x)); }
        else { double x[8]; memcpy(x, v, sizeof x); wr(fx_sum<8>(x)); }
    }
    return 0;
}
''')
    exe = d / "fx"
    subprocess.run(["g++", "-std=c++17", "-O2", "-I", os.path.join(ROOT, "paper_1905_06850_gb300", "csrc"),
                    str(src), "-o", str(exe)], check=True)

    def run(cases):
        inp = "".join(f"{len(c)} " + " ".join(struct.pack(">d", float(v)).hex() for v in c) + "\n"
                      for c in cases)
        out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, check=True).stdout
        return [struct.unpack(">d", bytes.fromhex(h))[0] for h in out.split()]
    return run


def emax_of(c):
    return max((struct.unpack(">Q", struct.pack(">d", float(v)))[0] >> 52) & 0x7ff for v in c)


def check_bound(c, got):
    exact = sum(Fraction(float(v)) for v in c)
    e = emax_of(c)
    ulp = math.ulp(got) if got != 0 else 0.0
    bound = Fraction(len(c)) * Fraction(2) ** (e - 1081) + Fraction(ulp) / 2
    err = abs(Fraction(got) - exact)
    assert err <= bound, (c, got, float(err), float(bound))
    return err


def seq(c):
    s = float(c[0])
    for v in c[1:]:
        s += float(v)
    return s


def test_random_operands_within_the_bound(fx):
    rng = np.random.default_rng(1)
    cases = []
    for k in (4, 6, 8):
        cases += [list(rng.standard_normal(k)) for _ in range(3000)]                 # one scale
        cases += [list(rng.standard_normal(k) * 2.0 ** rng.integers(-60, 61, k))       # spread
                  for _ in range(3000)]
        cases += [list(rng.choice([-1, 1], k) * rng.uniform(1, 2, k) * 2.0 ** rng.integers(-900, 900))
                  for _ in range(1000)]                                                  # far binades
    got = fx(cases)
    worse = 0
    for c, g in zip(cases, got):
        err = check_bound(c, g)
        exact = sum(Fraction(float(v)) for v in c)
        worse += err > abs(Fraction(seq(c)) - exact)
    # more accurate than the sequential FP64 additions in most cases
    assert worse < 0.2 * len(cases), worse


def test_cancellation_and_signs(fx):
    rng = np.random.default_rng(2)
    cases = []
    for _ in range(3000):
        a = rng.standard_normal(3)
        eps = rng.standard_normal(3) * 2.0 ** rng.integers(-50, -10, 3)
        c = [a[0], -a[0] * (1 + eps[0]), a[1], -(a[1] + eps[1]), a[2], -a[2]]
        rng.shuffle(c)
        cases.append(c)
    cases.append([1.0, -1.0, 2.0, -2.0, 0.5, -0.5])          # exact zero
    cases.append([1.0, 2.0 ** -52, 2.0 ** -53, -1.0, 0.0, 0.0])
    got = fx(cases)
    for c, g in zip(cases, got):
        check_bound(c, g)
    assert got[-2] == 0.0 and got[-1] == 2.0 ** -52 + 2.0 ** -53


def test_one_binade_is_correctly_rounded(fx):
    rng = np.random.default_rng(3)
    cases = [list(rng.choice([-1, 1], 6) * rng.uniform(1, 2, 6) * 2.0 ** rng.integers(-100, 100))
             for _ in range(4000)]
    got = fx(cases)
    for c, g in zip(cases, got):
        exact = sum(Fraction(float(v)) for v in c)
        # round-to-nearest of the exact rational: the neighbours of g bracket it
        lo, hi = np.nextafter(g, -np.inf), np.nextafter(g, np.inf)
        assert abs(Fraction(g) - exact) <= abs(Fraction(float(lo)) - exact)
        assert abs(Fraction(g) - exact) <= abs(Fraction(float(hi)) - exact)


def test_ties_round_to_even(fx):
    u = 2.0 ** -52
    cases = [[1.0, u / 2, 0.0, 0.0, 0.0, 0.0],             # 1 + u/2: tie, even is 1
             [1.0 + u, u / 2, 0.0, 0.0, 0.0, 0.0],         # tie, even is 1 + 2u
             [1.0, u / 2, u / 4, 0.0, 0.0, 0.0],           # above the tie: up
             [-1.0, -u / 2, 0.0, 0.0, 0.0, 0.0],           # negative tie
             [2.0 - u, u / 2, 0.0, 0.0, 0.0, 0.0],         # carry into the next binade: 2
             [3.0, 4.0, -2.0, 0.25, 0.0, 0.0]]             # exact
    assert fx(cases) == [1.0, 1.0 + 2 * u, 1.0 + u, -1.0, 2.0, 5.25]


def test_subnormal_operands_within_the_bound(fx):
    tiny = 5e-324 * 3
    cases = [[2.0 ** -960, tiny, -tiny * 2, 2.0 ** -1000, 0.0, 0.0],
             [2.0 ** -964, 2.0 ** -1022 * 0.75, -2.0 ** -1050, 0.0, -0.0, 2.0 ** -1000]]
    for c, g in zip(cases, fx(cases)):
        check_bound(c, g)


def test_out_of_range_takes_plain_additions(fx):
    cases = [[0.0] * 6, [-0.0] * 6, [1e-300, 2e-300, 0.0, 0.0, 0.0, 0.0],
             [1e308, 1e308, -1e308, 0.0, 0.0, 0.0], [math.inf, 1.0, 0.0, 0.0, 0.0, 0.0],
             [math.nan, 1.0, 2.0, 3.0, 4.0, 5.0], [math.inf, -math.inf, 0.0, 0.0]]
    got = fx(cases)
    for c, g in zip(cases, got):
        s = seq(c)
        assert (math.isnan(s) and math.isnan(g)) or struct.pack(">d", s) == struct.pack(">d", g), (c, g, s)
