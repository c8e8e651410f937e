"""Double-float arithmetic of the FP64 form's quadrature and corners
(paper_1709_06924_gb300/csrc/df.cuh), compiled for the host with g++ and
checked against exact rational arithmetic: TwoSum, Fast2Sum and the FMA form
of TwoProduct must be error-free, and the double-float add, multiply and
divide must stay within their error bounds (2^-47 of the operands for the
sum, 2^-45 relative for the product and quotient).  No GPU needed."""
import os
import subprocess
from fractions import Fraction

import numpy as np
import pytest

from paper_1709_06924_gb300 import build as B

SRC = r'''
#include <stdio.h>
#include <stdlib.h>
#include "df.cuh"
using namespace scvt;
int main(int argc, char **argv) {
    FILE *f = fopen(argv[1], "r");
    float a, b, c, d;
    while (fscanf(f, "%a %a %a %a", &a, &b, &c, &d) == 4) {
        const df s = two_sum(a, b);
        const df p = two_prod(a, b);
        const df x{a, c}, y{b, d};
        const df ad = df_add(x, y), mu = df_mul(x, y), dv = df_div(x, y);
        printf("%a %a %a %a %a %a %a %a %a %a\n", s.hi, s.lo, p.hi, p.lo, ad.hi, ad.lo, mu.hi, mu.lo, dv.hi, dv.lo);
    }
    return 0;
}
'''


def F(x):
    return Fraction(float(x))


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    tmp = tmp_path_factory.mktemp("df")
    src = tmp / "df_test.cpp"
    src.write_text(SRC)
    exe = tmp / "df_test"
    subprocess.run(["g++", "-O2", "-ffp-contract=off", "-I", os.path.join(B.PKG, "csrc"), str(src), "-o", str(exe)],
                   check=True)
    rng = np.random.default_rng(7)
    rows = []
    for _ in range(4000):
        a = np.float32(rng.standard_normal() * 10.0 ** rng.integers(-6, 6))
        b = np.float32(rng.standard_normal() * 10.0 ** rng.integers(-6, 6))
        if rng.random() < 0.2:
            b = np.float32(-a * (1 + rng.standard_normal() * 1e-6))  # near cancellation
        # low parts: below half an ulp of the high parts
        c = np.float32(rng.uniform(-0.5, 0.5) * np.spacing(np.float32(abs(a))))
        d = np.float32(rng.uniform(-0.5, 0.5) * np.spacing(np.float32(abs(b))))
        rows.append((a, b, c, d))
    inp = tmp / "in.txt"
    inp.write_text("\n".join(" ".join(float(v).hex() for v in r) for r in rows))
    out = subprocess.run([str(exe), str(inp)], capture_output=True, text=True, check=True).stdout.split("\n")
    res = [[float.fromhex(t) for t in line.split()] for line in out if line.strip()]
    return rows, res


def test_error_free_transformations(results):
    rows, res = results
    for (a, b, c, d), r in zip(rows, res):
        assert F(r[0]) + F(r[1]) == F(a) + F(b)          # TwoSum
        if a != 0 and b != 0 and abs(float(a) * float(b)) > 1e-30:
            assert F(r[2]) + F(r[3]) == F(a) * F(b)      # TwoProduct by FMA


def test_double_float_operations_within_their_bounds(results):
    rows, res = results
    worst = [0.0, 0.0, 0.0]
    for (a, b, c, d), r in zip(rows, res):
        x, y = F(a) + F(c), F(b) + F(d)
        add = F(r[4]) + F(r[5])
        err_add = abs(add - (x + y)) / (abs(x) + abs(y))
        worst[0] = max(worst[0], float(err_add))
        if x != 0 and y != 0 and abs(float(a) * float(b)) > 1e-30:
            mul = F(r[6]) + F(r[7])
            worst[1] = max(worst[1], float(abs(mul - x * y) / abs(x * y)))
            dv = F(r[8]) + F(r[9])
            worst[2] = max(worst[2], float(abs(dv - x / y) / abs(x / y)))
    assert worst[0] <= 2.0 ** -47, worst
    assert worst[1] <= 2.0 ** -45, worst
    assert worst[2] <= 2.0 ** -44, worst


LAZY_SRC = r'''
#include <stdio.h>
#include "df.cuh"
using namespace scvt;
int main(int argc, char **argv) {
    FILE *f = fopen(argv[1], "r");
    float a, b, c, d;
    while (fscanf(f, "%a %a %a %a", &a, &b, &c, &d) == 4) {
        const df x{a, c}, y{b, d};
        const df ad = dfl_add(x, y), mu = dfl_mul(x, y);
        // a chain: ((x y + x) y + y) x, unnormalized, then normalized
        const df ch = df_norm(dfl_mul(dfl_add(dfl_mul(dfl_add(dfl_mul(x, y), x), y), y), x));
        const df n = df_norm(ad);
        printf("%a %a %a %a %a %a %a %a\n", ad.hi, ad.lo, mu.hi, mu.lo, ch.hi, ch.lo, n.hi, n.lo);
    }
    return 0;
}
'''


def test_unnormalized_operations_within_their_bounds(tmp_path):
    src = tmp_path / "lazy_test.cpp"
    src.write_text(LAZY_SRC)
    exe = tmp_path / "lazy_test"
    subprocess.run(["g++", "-O2", "-ffp-contract=off", "-I", os.path.join(B.PKG, "csrc"), str(src), "-o", str(exe)],
                   check=True)
    rng = np.random.default_rng(13)
    rows = []
    for _ in range(3000):
        a = np.float32(rng.uniform(0.5, 2.0) * 10.0 ** rng.integers(-3, 3))
        b = np.float32(rng.uniform(0.5, 2.0) * 10.0 ** rng.integers(-3, 3))
        c = np.float32(rng.uniform(-0.5, 0.5) * np.spacing(a))
        d = np.float32(rng.uniform(-0.5, 0.5) * np.spacing(b))
        rows.append((a, b, c, d))
    inp = tmp_path / "in.txt"
    inp.write_text("\n".join(" ".join(float(v).hex() for v in r) for r in rows))
    out = subprocess.run([str(exe), str(inp)], capture_output=True, text=True, check=True).stdout.split("\n")
    res = [[float.fromhex(t) for t in line.split()] for line in out if line.strip()]
    worst = [0.0, 0.0, 0.0]
    for (a, b, c, d), r in zip(rows, res):
        x, y = F(a) + F(c), F(b) + F(d)
        worst[0] = max(worst[0], float(abs(F(r[0]) + F(r[1]) - (x + y)) / (abs(x) + abs(y))))
        worst[1] = max(worst[1], float(abs(F(r[2]) + F(r[3]) - x * y) / abs(x * y)))
        exact = ((x * y + x) * y + y) * x
        worst[2] = max(worst[2], float(abs(F(r[4]) + F(r[5]) - exact) / abs(exact)))
        assert F(r[6]) + F(r[7]) == F(r[0]) + F(r[1])   # normalizing keeps the value
        assert abs(r[7]) <= 0.5 * float(np.spacing(np.float32(abs(r[6]))))
    # positive operands: no cancellation, so the chain keeps double-float accuracy
    assert worst[0] <= 2.0 ** -47, worst
    assert worst[1] <= 2.0 ** -45, worst
    assert worst[2] <= 2.0 ** -42, worst
