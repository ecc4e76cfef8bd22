"""The emulated-FP64 product's slicing arithmetic, compiled for the host (no GPU).

paper_2310_14087_gb300/csrc/oz_slicing.cuh holds the integer code the CUDA kernels use to cut
operand values into fixed-point BF16 slices and to close exact accumulation groups.  A small C++
harness compiled with the host compiler checks, over many random values and every slice count:
  * each digit is at most 128 in magnitude (so slice products are at most 2^14);
  * the digits reconstruct |v| 2^(7 + 8(s-1) - e_r) rounded to an integer (error <= 1/2), with
    the sign of v, including subnormals, zeros and the row maximum itself;
  * every slice value d_i 2^(-8 i) is exact in BF16 (at most 8 significant bits);
  * over every (slice pair, k tile) sequence a split can see, no group of a level below the exact
    limit mixes levels or holds more than 512 products per output element (so its FP32 sum of
    integers below 2^14 in magnitude stays below 2^23, i.e. exact).
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2310_14087_gb300", "csrc")

HARNESS = r'''
#include "oz_slicing.cuh"
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
using namespace kot::oz;

static int fail(const char* what, double v, int s) {
  std::printf("FAIL %s v=%.17g s=%d\n", what, v, s);
  return 1;
}

int main() {
  std::mt19937_64 rng(12345);
  std::uniform_real_distribution<double> uni(-1.0, 1.0);
  std::uniform_int_distribution<int> expo(-60, 60), spread(0, 70);
  long long checked = 0;
  for (int s = 3; s <= kMaxSlices; ++s) {
    for (int row = 0; row < 4000; ++row) {
      // a row of values spanning up to 70 binades below its maximum, plus special values
      double vals[12];
      const int e0 = expo(rng);
      for (int k = 0; k < 8; ++k) vals[k] = std::ldexp(uni(rng), e0 - spread(rng));
      vals[8] = 0.0;
      vals[9] = -0.0;
      vals[10] = 4.9406564584124654e-324 * (row % 7);   // subnormals (and 0)
      vals[11] = std::ldexp(1.0, e0) * (1.0 - std::ldexp(1.0, -53));   // just below 2^e0
      int Emax = 0;
      for (double v : vals) Emax = Emax > biased_exp(v) ? Emax : biased_exp(v);
      const int er = Emax - 1022;
      for (double v : vals) {
        int d[kMaxSlices];
        digits(v, er, s, d);
        __int128 R = 0;
        for (int i = 0; i < s; ++i) {
          if (d[i] > 128 || d[i] < -128) return fail("digit bound", v, s);
          R = R * 256 + d[i];
          // slice value d_i 2^(-8 i) in BF16: the float's low 16 bits are zero
          const float f = std::ldexp((float)d[i], -8 * i);
          unsigned u;
          std::memcpy(&u, &f, 4);
          if (u & 0xFFFFu) return fail("bf16 exactness", v, s);
        }
        for (int i = s; i < kMaxSlices; ++i)
          if (d[i] != 0) return fail("unused digit", v, s);
        const long double x = std::ldexp((long double)std::fabs(v), 7 + 8 * (s - 1) - er);
        const long double r = (long double)(R < 0 ? -R : R);
        if (std::fabs(r - x) > 0.5L) return fail("reconstruction", v, s);
        if (v < 0 && R > 0) return fail("sign", v, s);
        if (v > 0 && R < 0) return fail("sign", v, s);
        ++checked;
      }
    }
    // group rule over every split range of every pair sequence
    int pa[64], pb[64], lv[64], np = 0;
    for (int t = 0; t < s; ++t)
      for (int i = 0; i <= t; ++i) {
        pa[np] = i;
        pb[np] = t - i;
        lv[np] = t;
        ++np;
      }
    for (int nk = 1; nk <= 33; ++nk) {
      const int T = np * nk;
      for (int splits = 1; splits <= 16; ++splits) {
        for (int z = 0; z < splits; ++z) {
          const int s0 = (int)((long long)z * T / splits), s1 = (int)((long long)(z + 1) * T / splits);
          int gt = 0, prev = -1, glevel = -1, gmixed = 0;
          for (int n = s0; n < s1; ++n) {
            const int l = lv[n / nk];
            if (new_group(prev, l, gt)) {
              gt = 0;
              glevel = l;
              gmixed = 0;
            }
            if (l != glevel) gmixed = 1;
            ++gt;
            prev = l;
            if (glevel < kExactLevels && (gmixed || gt * 64 > 512)) return fail("group rule", nk, s);
          }
        }
      }
    }
  }
  std::printf("ok %lld\n", checked);
  return 0;
}
'''


def test_slicing_arithmetic_on_the_host(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "harness.cpp"
    src.write_text(HARNESS)
    exe = tmp_path / "harness"
    r = subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.startswith("ok"), out.stdout + out.stderr
