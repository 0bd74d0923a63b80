"""nsn_f32_to_f64_exact (csrc/nsn_bits.h): the integer-pipe binary32 ->
binary64 re-encoding the kernels use before their FP64 accumulations, checked
on the host against the C conversion for every one of the 2^32 bit patterns
(NaNs: both NaN).  The device build compiles the same code with the CUDA
bit-cast and count-leading-zeros intrinsics in place of memcpy and
__builtin_clz."""
import os
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
HDR = os.path.join(HERE, "..", "paper_1907_04587_gb300", "csrc")

SRC = r'''
#include <math.h>
#include <stdio.h>
#include "nsn_bits.h"
int main(void) {
  unsigned long long bad = 0, nan = 0;
  uint32_t u = 0;
  do {
    float x; memcpy(&x, &u, 4);
    const double a = nsn_f32_to_f64_exact(x), b = (double)x;
    if (isnan(b)) { nan++; if (!isnan(a)) bad++; }
    else if (memcmp(&a, &b, 8) != 0) { if (bad < 5) printf("mismatch %08x\n", u); bad++; }
    u++;
  } while (u != 0);
  printf("%llu %llu\n", bad, nan);
  return bad != 0;
}
'''


def test_exhaustive_against_c_conversion(tmp_path):
    gcc = "gcc"
    c = tmp_path / "bits.c"
    c.write_text(SRC)
    exe = tmp_path / "bits"
    r = subprocess.run([gcc, "-O2", "-std=c99", "-I", HDR, str(c), "-o", str(exe), "-lm"], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail(r.stderr)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    print(r.stdout)
    bad, nan = (int(v) for v in r.stdout.split()[-2:])
    assert r.returncode == 0 and bad == 0
    assert nan == 2 * (2 ** 23 - 1)      # every NaN pattern was seen


APAP_SRC = r'''
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include "nsn_bits.h"
static unsigned long long s = 0x9E3779B97F4A7C15ull;
static double rnd(void) {   /* xorshift64*, uniform in [0, 1) */
  s ^= s >> 12; s ^= s << 25; s ^= s >> 27;
  return (double)((s * 2685821657736338717ull) >> 11) * (1.0 / 9007199254740992.0);
}
int main(int argc, char **argv) {
  const int n = atoi(argv[1]);
  for (int i = 0; i < n; i++) {
    const float beta = (float)(0.05 + 2.0 * rnd());
    const float d3 = (float)((rnd() - 0.5) * 8.0);
    const float d5 = (float)(0.1 + 4.0 * rnd());
    /* d2 cancels the other two terms to a relative 10^-k, k in 0 .. 7 */
    const double rest = 2.0 * beta * (double)d3 + (double)beta * beta * d5;
    const double rel = pow(10.0, -7.0 * rnd()) * (rnd() < 0.5 ? -1.0 : 1.0);
    const float d2 = (float)(-rest * (1.0 + rel));
    const float naive = d2 + 2.0f * beta * d3 + beta * beta * d5;
    printf("%a %a %a %a %a %a\n", d2, d3, d5, beta, nsn_apap_f32(d2, d3, d5, beta), naive);
  }
  return 0;
}
'''


def test_double_word_aptpap_against_exact_rationals(tmp_path):
    """nsn_apap_f32 (the FP32 build's ApTPAp = d2 + 2 beta d3 + beta^2 d5 in
    two binary32 words) against the exact rational value, on inputs whose
    terms cancel to a relative 1e-7 .. 1: within half an FP32 ulp of the exact
    value plus 2^-45 of the sum of the terms' magnitudes (the double-word
    error bound, with margin).  The plain FP32 evaluation misses that bound on
    most of the cancelling inputs, so a lost error term would be seen."""
    from fractions import Fraction
    import numpy as np
    c = tmp_path / "apap.c"
    c.write_text(APAP_SRC)
    exe = tmp_path / "apap"
    r = subprocess.run(["gcc", "-O2", "-std=c99", "-I", HDR, str(c), "-o", str(exe), "-lm"], capture_output=True,
                       text=True)
    if r.returncode != 0:
        pytest.fail(r.stderr)
    out = subprocess.run([str(exe), "20000"], capture_output=True, text=True, timeout=120).stdout.split("\n")
    fails = naive_fails = 0
    for line in out:
        if not line:
            continue
        d2, d3, d5, beta, got, naive = (float.fromhex(v) for v in line.split())
        F = Fraction
        terms = [F(d2), 2 * F(beta) * F(d3), F(beta) * F(beta) * F(d5)]
        exact = sum(terms)
        mag = sum(abs(t) for t in terms)
        ulp = np.spacing(np.float32(abs(float(exact)))) if exact != 0 else np.float32(0)
        bound = F(float(ulp)) / 2 + mag / 2 ** 45
        fails += abs(F(got) - exact) > bound
        naive_fails += abs(F(naive) - exact) > bound
    assert fails == 0
    assert naive_fails > 5000
