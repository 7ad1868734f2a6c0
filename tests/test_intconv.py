"""Host checks of the integer FP64 -> FP32 / FP16 conversion helpers
(csrc/intconv.cuh) that the GPU kernels use in place of FP64 instructions:
compiled for the host with g++ and compared bit for bit with the C casts."""
import os
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_2605_24840_gb300", "csrc", "intconv.cuh")

PROG = r'''
#include "intconv.cuh"
#include <cstdio>
#include <cmath>
#include <random>
#include <cstring>
using namespace rsign;
static double f16v(uint16_t v) {
  int e = (v >> 10) & 0x1F; double m = v & 0x3FF;
  double x = e == 0 ? std::ldexp(m, -24) : std::ldexp(m + 1024, e - 25);
  return (v & 0x8000) ? -x : x;
}
int main() {
  std::mt19937_64 g(7);
  long bad = 0, n = 0;
  for (int it = 0; it < 2000000; ++it) {
    uint64_t b = g();
    int ex = 1023 + (int)(g() % 320) - 160;
    b = (b & 0x800FFFFFFFFFFFFFull) | ((uint64_t)ex << 52);
    if (it % 97 == 0) b &= 0x8000000000000000ull;          // zeros
    if (it % 89 == 0) b = (b & 0xFFF0000000000000ull);      // exact powers of two
    if (it % 83 == 0) b |= 0x0000000010000000ull;           // ties at the 24-bit cut
    const double x = ic_double(b);
    const int k = (int)(g() % 61) - 30;
    float hi, lo;
    ic_split_f32(x, k, &hi, &lo);
    const double xs = std::ldexp(x, k);
    ++n;
    if (std::fabs(xs) < std::ldexp(1.0, -126)) { bad += (hi != 0.0f || lo != 0.0f); continue; }
    if (std::fabs(xs) >= std::ldexp(1.0, 128) || std::isinf((float)xs)) { bad += !std::isinf(hi); continue; }
    const float rh = (float)xs;
    if (ic_fbits(hi) != ic_fbits(rh)) { ++bad; continue; }
    const double rem = xs - (double)hi;
    if (std::fabs(rem) < std::ldexp(1.0, -126)) { bad += std::fabs((double)lo - rem) > std::ldexp(1.0, -126); continue; }
    bad += ic_fbits(lo) != ic_fbits((float)rem);
  }
  long bad16 = 0;
  for (uint32_t h = 0; h < 65536; h += 3) {
    if (((h >> 10) & 0x1F) == 31) continue;
    for (int t = 0; t < 8; ++t) {
      const uint16_t l = (uint16_t)(g() & 0xFFFF);
      if (((l >> 10) & 0x1F) == 31) continue;
      const double ref = f16v((uint16_t)h) + f16v(l);
      const double got = ic_i64_scaled(ic_f16_units((uint16_t)h) + ic_f16_units(l), -24);
      bad16 += !(got == ref);
    }
  }
  long badf = 0;
  for (int it = 0; it < 2000000; ++it) {
    const uint32_t fb = (uint32_t)g();
    if (((fb >> 23) & 0xFF) == 255) continue;
    float f;
    std::memcpy(&f, &fb, 4);
    badf += ic_bits(ic_f2d(f)) != ic_bits((double)f);
  }
  std::printf("%ld %ld %ld %ld\n", n, bad, bad16, badf);
  return 0;
}
'''


def test_integer_conversions_match_the_c_casts(tmp_path):
    src = tmp_path / "t.cpp"
    src.write_text(PROG)
    exe = tmp_path / "t"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-I", os.path.dirname(HDR), str(src), "-o", str(exe)])
    n, bad, bad16, badf = map(int, subprocess.check_output([str(exe)]).split())
    assert n == 2000000 and bad == 0 and bad16 == 0 and badf == 0
