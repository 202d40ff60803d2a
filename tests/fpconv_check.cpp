// Host check of the integer-only FP32 <-> FP64 conversions the kernels use (md_fpconv.cuh):
// narrow_f64 against the host's own double -> float conversion (round to nearest, ties to even)
// and widen_f32 against float -> double, bit for bit, over random bit patterns of every class,
// exact ties at half a unit of the last place, and values around every FP32 binade edge. Prints
// "ok <cases>" or the first mismatch and exits 1.
#include <cfloat>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>

#include "md_fpconv.cuh"

static uint64_t bits_d(double d) { uint64_t b; std::memcpy(&b, &d, 8); return b; }
static uint32_t bits_f(float f) { uint32_t b; std::memcpy(&b, &f, 4); return b; }
static double from_bits_d(uint64_t b) { double d; std::memcpy(&d, &b, 8); return d; }
static float from_bits_f(uint32_t b) { float f; std::memcpy(&f, &b, 4); return f; }

static long cases = 0;

static bool check_narrow(double d) {
  ++cases;
  const float got = mdk::narrow_f64(d), want = (float)d;
  if (std::isnan(want) ? std::isnan(got) : bits_f(got) == bits_f(want)) return true;
  std::printf("narrow_f64 mismatch: d=%a got=%a want=%a\n", d, (double)got, (double)want);
  return false;
}

static bool check_widen(float f) {
  ++cases;
  const double got = mdk::widen_f32(f), want = (double)f;
  if (std::isnan(want) ? std::isnan(got) : bits_d(got) == bits_d(want)) return true;
  std::printf("widen_f32 mismatch: f=%a got=%a want=%a\n", (double)f, got, want);
  return false;
}

int main() {
  std::mt19937_64 rng(20181219);
  // random bit patterns: every exponent, sign and mantissa
  for (int k = 0; k < 2000000; ++k) {
    if (!check_narrow(from_bits_d(rng()))) return 1;
    if (!check_widen(from_bits_f((uint32_t)rng()))) return 1;
  }
  // doubles in the range of cell-local offsets and displacements
  std::uniform_real_distribution<double> u(-8.0, 8.0);
  for (int k = 0; k < 2000000; ++k)
    if (!check_narrow(u(rng)) || !check_narrow(u(rng) * 1e-6)) return 1;
  // exact ties and their neighbours: an FP32 value plus half its last-place unit (and one double
  // ulp either side), for odd and even kept mantissas
  for (int k = 0; k < 1000000; ++k) {
    const uint32_t fb = ((uint32_t)rng() & 0x807fffffu) | ((uint32_t)(1 + rng() % 253) << 23);
    const double f = (double)from_bits_f(fb);
    const double ulp = std::ldexp(1.0, (int)((fb >> 23) & 0xff) - 127 - 23);
    const double tie = f + std::copysign(0.5 * ulp, f);
    if (!check_narrow(tie) || !check_narrow(std::nextafter(tie, 0.0)) ||
        !check_narrow(std::nextafter(tie, 2.0 * tie)))
      return 1;
  }
  // binade edges (a mantissa carry into the exponent), FP32 limits, zeros, subnormals, infinities
  for (int e = -160; e <= 130; ++e) {
    const double p = std::ldexp(1.0, e);
    const double ds[] = {p, std::nextafter(p, 0.0), std::nextafter(p, 4.0 * p), -p,
                         p * (2.0 - std::ldexp(1.0, -24)), p * (2.0 - std::ldexp(1.0, -25))};
    for (double d : ds)
      if (!check_narrow(d)) return 1;
  }
  const double dspecial[] = {0.0, -0.0, INFINITY, -INFINITY, (double)FLT_MAX, (double)FLT_MIN,
                             3.4028235677973366e38, 1e-40, -1e-45, 5e-324};
  for (double d : dspecial)
    if (!check_narrow(d)) return 1;
  const float fspecial[] = {0.0f, -0.0f, INFINITY, -INFINITY, FLT_MAX, FLT_MIN, 1e-40f, -1e-45f,
                            1.0f};
  for (float f : fspecial)
    if (!check_widen(f)) return 1;
  std::printf("ok %ld\n", cases);
  return 0;
}
