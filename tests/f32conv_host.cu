// Host check of the bit-level conversions of csrc/f32conv.cuh.  Against the C library's
// IEEE conversions: f32_of must truncate toward zero (round to nearest, then one step
// toward zero where that rounded away), give a signed zero below 2^-126 and infinity from
// 2^128 on; f64_of must be exact on normal floats and give a signed zero for FP32
// subnormals.  Against the FP64 slicing loop of the FP64-accurate GEMM: fixed54's 6-bit
// groups must be its digits.  Random magnitudes plus edge values; prints the number of
// mismatches and exits non-zero on any.
#include <cfloat>
#include <cmath>
#include <cstdio>

#include "f32conv.cuh"

static uint64_t rng_state = 0x9e3779b97f4a7c15ull;
static uint64_t next_u64() {  // splitmix64
  uint64_t z = (rng_state += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

static float ref_f32(double x) {
  const double ax = std::fabs(x);
  if (ax < (double)FLT_MIN) return std::signbit(x) ? -0.0f : 0.0f;
  if (ax >= std::ldexp(1.0, 128)) return std::signbit(x) ? -INFINITY : INFINITY;
  float r = (float)x;
  if (std::fabs((double)r) > ax) r = std::nextafterf(r, 0.0f);
  return r;
}

static int check_f32(double x) {
  const float got = tnt::f32_of(x), want = ref_f32(x);
  if (tnt::bits_of(got) != tnt::bits_of(want)) {
    std::printf("f32_of(%.17g) = %.9g, expected %.9g\n", x, (double)got, (double)want);
    return 1;
  }
  return 0;
}

static int check_f64(float f) {
  const double got = tnt::f64_of(f);
  double want;
  if (std::isnan(f)) return std::isnan(got) ? 0 : 1;
  if (f != 0.0f && std::fabs(f) < FLT_MIN) want = std::signbit(f) ? -0.0 : 0.0;
  else want = (double)f;
  if (tnt::bits_of(got) != tnt::bits_of(want)) {
    std::printf("f64_of(%.9g) = %.17g, expected %.17g\n", (double)f, got, want);
    return 1;
  }
  return 0;
}

// fixed54's 6-bit groups against the FP64 loop the slicing of the FP64-accurate GEMM
// defines: t = |v| / 2^esc, then nine times t *= 64, digit = trunc(t), t -= digit (each
// step exact)
static int check_fixed54(double v, int esc) {
  double t = std::fabs(v) * std::ldexp(1.0, -esc);
  const uint64_t F = tnt::fixed54(v, esc);
  for (int p = 0; p < 9; ++p) {
    t *= 64.0;
    const double d = std::trunc(t);
    t -= d;
    const uint64_t got = (F >> (48 - 6 * p)) & 63u;
    if ((double)got != d) {
      std::printf("fixed54(%.17g, %d): digit %d = %llu, expected %.0f\n", v, esc, p + 1,
                  (unsigned long long)got, d);
      return 1;
    }
  }
  return 0;
}

int main() {
  int bad = 0;
  for (int i = 0; i < 400000; ++i) {  // |v| < 2^esc, esc one to four above v's exponent
    const uint64_t r = next_u64();
    const double mant = 1.0 + (double)(r >> 12) * std::ldexp(1.0, -52);
    const int ex = (int)(next_u64() % 600) - 300;
    const double v = std::ldexp((r & 1) ? -mant : mant, ex);
    bad += check_fixed54(v, ex + 1 + (int)(next_u64() % 4));
  }
  bad += check_fixed54(0.0, 0) + check_fixed54(-0.0, 5) + check_fixed54(4.9e-324, -1020) +
         check_fixed54(std::nextafter(1.0, 0.0), 0) + check_fixed54(-0.75, 0);
  const double edges[] = {0.0, -0.0, 1.0, -1.0, 0.5, 3.0, (double)FLT_MIN, -(double)FLT_MIN,
                          std::ldexp(1.0, -127), std::ldexp(1.0, -149), (double)FLT_MAX,
                          std::nextafter((double)FLT_MAX, INFINITY), std::ldexp(1.0, 128),
                          -std::ldexp(1.0, 128), 1e300, -1e-300, 4.9e-324, INFINITY, -INFINITY,
                          1.0 + std::ldexp(1.0, -23), 1.0 + std::ldexp(1.0, -24),
                          1.0 - std::ldexp(1.0, -54), 0.1, -0.3333333333333333};
  for (double x : edges) bad += check_f32(x);
  for (int i = 0; i < 2000000; ++i) {
    const uint64_t r = next_u64();
    // mantissa from the random bits, exponent spread over [-140, 140), both signs
    const double mant = 1.0 + (double)(r >> 12) * std::ldexp(1.0, -52);
    const int ex = (int)(next_u64() % 280) - 140;
    const double x = std::ldexp((r & 1) ? -mant : mant, ex);
    bad += check_f32(x);
    bad += check_f64(tnt::float_of_bits((unsigned)(next_u64() >> 32)));
  }
  const float fedges[] = {0.0f, -0.0f, 1.0f, FLT_MIN, FLT_MAX, -FLT_MAX, 1e-40f, -1e-45f,
                          INFINITY, -INFINITY, NAN};
  for (float f : fedges) bad += check_f64(f);
  std::printf("mismatches %d\n", bad);
  return bad ? 1 : 0;
}
