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
