"""The FP32 form's error function (stage.cuh erf_ex: Abramowitz & Stegun
7.1.26 re-expanded about t = 1, from an exponential the edge solution has
formed already) against the library erf on the host: within the published
bound of 1.5e-7 plus FP32 rounding of its few operations over the arguments
the half-space moments meet (sqrt(lam) U up to several units, both signs),
odd and exact at zero, and proportional to x for tiny arguments (a state
near rest has tiny velocities, whose erf terms enter the deviation h-bar -
h_b directly: an error of the size of FP32 rounding of 1 there would swamp
them): relative error 1e-5 (the approximation's own slope at zero is 6e-6
off) plus 4e-8 absolute from rounding 1 - e^{-x^2}."""
import math
import os
import subprocess

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2306_04467_gb300", "csrc")

PROG = r'''
#include <cstdio>
#include <cmath>
#include "stage.cuh"
int main() {
  for (int i = -4000; i <= 4000; i++) {
    float x = i * 0.002f;
    float ex = std::exp(-x * x);
    printf("%.9g %.9g\n", (double)x, (double)gks2l::erf_ex<float>(x, ex));
  }
  for (int k = -30; k <= -2; k++) {
    float x = std::ldexp(1.3f, k);
    printf("%.9g %.9g\n", (double)x, (double)gks2l::erf_ex<float>(x, std::exp(-x * x)));
  }
  return 0;
}
'''


def test_erf_from_exponential_within_its_bound(tmp_path):
    src, exe = tmp_path / "e.cpp", tmp_path / "e"
    src.write_text(PROG)
    subprocess.check_call(["g++", "-std=c++17", "-O2", "-I", CSRC, str(src), "-o", str(exe)])
    xs, ys = np.loadtxt(subprocess.check_output([str(exe)], text=True).splitlines()).T
    ref = np.array([math.erf(x) for x in xs])
    assert np.abs(ys - ref).max() <= 1.5e-7 + 4 * 2.0 ** -24
    grid, tiny = slice(0, 8001), slice(8001, None)
    assert ys[4000] == 0.0 and np.array_equal(ys[grid], -ys[grid][::-1])
    assert np.all(np.abs(ys[tiny] - ref[tiny]) <= 1e-5 * ref[tiny] + 4e-8)
    assert (np.abs(ys[tiny][:12] - ref[tiny][:12]) / ref[tiny][:12]).max() <= 1e-5   # |x| < 2^-18
