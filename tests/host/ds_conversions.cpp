// Host check of the integer FP64 <-> FP32 conversions and the FP32-pair split of csrc/ds.cuh against the C++
// conversions: f2d is exact, d2f_rn equals the round-to-nearest conversion wherever |v| is at least FLT_MIN (a
// zero of v's sign below), d2ds leaves |v - (h + l)| <= 2^-48 |v| with h the rounded value.  Prints "ok" or the
// first failures.
#include <cfenv>
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <random>

#include "ds.cuh"

using namespace fetirp;

static int fails = 0;
static void fail(const char* what, double v, double got, double want) {
  if (++fails <= 10) std::printf("FAIL %s v=%.17g got=%.17g want=%.17g\n", what, v, got, want);
}

static float rn_ref(double v) {
  volatile double x = v;
  volatile float f = (float)x;
  return f;
}

int main() {
  std::mt19937_64 rng(12345);
  // f2d: every class of FP32 value, exact
  for (int i = 0; i < 2000000; ++i) {
    const uint32_t b = (uint32_t)rng();
    const float f = from_bits32(b);
    const double d = f2d(f);
    if (std::isnan(f)) {
      if (!std::isnan(d)) fail("f2d nan", f, d, f);
    } else if (bits64(d) != bits64((double)f)) {
      fail("f2d", f, d, (double)f);
    }
  }
  // d2f_rn: random bit patterns, random magnitudes around the FP32 range limits, and ties
  for (int i = 0; i < 4000000; ++i) {
    double v;
    if (i & 1) {
      v = from_bits64(rng());
    } else {
      const int e = (int)(rng() % 300) - 150;
      v = std::ldexp(1.0 + (double)(rng() >> 12) / 4503599627370496.0, e) * ((rng() & 1) ? -1.0 : 1.0);
    }
    if (i % 7 == 0) v = from_bits64((bits64(v) & ~0x1fffffffull) | 0x10000000ull);   // an exact tie
    const float got = d2f_rn(v);
    if (std::isnan(v)) {
      if (!std::isnan(got)) fail("d2f_rn nan", v, got, v);
      continue;
    }
    float want = rn_ref(v);
    if (std::fabs(v) < FLT_MIN) want = std::copysign(0.0f, v);
    if (bits32(got) != bits32(want)) fail("d2f_rn", v, got, want);
  }
  // d2ds: the pair's error bound on the range where l stays normal
  for (int i = 0; i < 4000000; ++i) {
    const int e = (int)(rng() % 187) - 60;   // 2^-60 .. 2^126
    const double v = std::ldexp(1.0 + (double)(rng() >> 12) / 4503599627370496.0, e) * ((rng() & 1) ? -1.0 : 1.0);
    float h, l;
    d2ds(v, h, l);
    const long double err = std::fabs((long double)v - ((long double)h + (long double)l));
    if (err > std::ldexp((long double)std::fabs(v), -48)) fail("d2ds", v, (double)err, std::ldexp(std::fabs(v), -48));
    if (bits32(h) != bits32(rn_ref(v))) fail("d2ds h", v, h, rn_ref(v));
    if (bits32(l) != bits32(rn_ref(v - (double)h))) fail("d2ds l", v, l, rn_ref(v - (double)h));
    const double back = ds2d(h, l);
    if (std::fabs(back - v) > std::ldexp(std::fabs(v), -48)) fail("ds2d", v, back, v);
  }
  // zeros keep their sign
  if (bits32(d2f_rn(-0.0)) != 0x80000000u || bits64(f2d(-0.0f)) != 0x8000000000000000ull) fail("signed zero", 0, 0, 0);
  if (fails == 0) std::printf("ok\n");
  return fails == 0 ? 0 : 1;
}
