"""The double-double oracle's exp (used by the point source's wavelet and Gaussian in the
long-run reference build) against mpmath at 40 digits: the reference of source runs is
double-double accurate in its source term, not only binary64 accurate."""
from __future__ import annotations

import os
import subprocess

import pytest

ORACLE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")

SRC = r'''
#include "dd.hpp"
#include <cstdio>
int main() {
    double x;
    while (std::scanf("%lf", &x) == 1) {
        orc_dd e = orc_dd_exp(orc_dd(x));
        std::printf("%.17g %.17g\n", e.hi, e.lo);
    }
}
'''


def test_dd_exp_is_double_double_accurate(tmp_path):
    mpmath = pytest.importorskip("mpmath")
    src = tmp_path / "ddexp.cpp"
    src.write_text(SRC)
    exe = tmp_path / "ddexp"
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I" + ORACLE, str(src), "-o", str(exe)],
                   check=True)
    xs = [-600.0, -71.3, -50.0, -12.25, -3.3, -0.7, -1e-9, 0.0, 0.1234, 1.0, 5.5, 40.0]
    out = subprocess.run([str(exe)], input="\n".join(repr(x) for x in xs), capture_output=True, text=True,
                         check=True).stdout.split("\n")
    mpmath.mp.dps = 40
    for x, line in zip(xs, out):
        hi, lo = (float(v) for v in line.split())
        got = mpmath.mpf(hi) + mpmath.mpf(lo)
        ref = mpmath.exp(mpmath.mpf(x))
        assert abs(got - ref) <= mpmath.mpf(2) ** -98 * ref, (x, float((got - ref) / ref))
