// Host check of the integer binary32 <-> binary64 conversions of the FP64
// M-step tail against the C casts (IEEE 754 conversions, round to nearest
// even under the default rounding mode):
//  * widen_bits on every binary32 encoding (subnormals must be declined);
//  * narrow_bits on doubles at and around every rounding boundary class:
//    exact binary32 values, midpoints between neighbours (ties to even),
//    one binary64 ulp either side of the midpoints, the overflow threshold,
//    the normal/subnormal threshold, zeros, infinities and NaNs, plus random
//    encodings over all exponents.  Where narrow_bits accepts an input its
//    bits must equal the cast's; it may decline only NaNs, infinities and
//    magnitudes outside [2^-126, 2^128) other than zero.
// Prints "ok <counts>" and exits 0, or prints the first mismatch and exits 1.
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "gmmsp_fpconv.cuh"

static uint32_t f2u(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }
static float u2f(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }
static uint64_t d2u(double d) { uint64_t u; memcpy(&u, &d, 8); return u; }
static double u2d(uint64_t u) { double d; memcpy(&d, &u, 8); return d; }

static uint64_t state = 0x9e3779b97f4a7c15ull;
static uint64_t next_u64() {  // splitmix64
  uint64_t z = (state += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

static long long accepted = 0, declined = 0;

static bool check_narrow(double d) {
  const uint64_t u = d2u(d);
  uint32_t out = 0;
  const bool ok = gmmsp::narrow_bits(uint32_t(u >> 32), uint32_t(u), out);
  const float ref = (float)d;
  if (ok) {
    ++accepted;
    if (out != f2u(ref)) {
      printf("narrow mismatch: %a -> %08x, cast %08x\n", d, out, f2u(ref));
      return false;
    }
  } else {
    ++declined;
    // only NaNs, infinities, nonzero magnitudes below the smallest normal
    // binary32 number and magnitudes of 2^128 and above may be declined
    const double m = fabs(d);
    if (!(isnan(d) || isinf(d) || (m != 0.0 && m < (double)FLT_MIN) || m >= ldexp(1.0, 128))) {
      printf("narrow declined %a (cast %a)\n", d, (double)ref);
      return false;
    }
  }
  return true;
}

int main() {
  // widen: every binary32 encoding
  long long wide = 0;
  for (uint64_t b = 0; b <= 0xffffffffull; ++b) {
    uint32_t hi = 0, lo = 0;
    const float f = u2f(uint32_t(b));
    const bool ok = gmmsp::widen_bits(uint32_t(b), hi, lo);
    const bool sub = fpclassify(f) == FP_SUBNORMAL;
    if (ok == sub) {
      printf("widen accept/decline wrong at %08llx\n", (unsigned long long)b);
      return 1;
    }
    if (!ok) continue;
    const double got = u2d((uint64_t(hi) << 32) | lo), ref = (double)f;
    if (isnan(ref) ? !isnan(got) : d2u(got) != d2u(ref)) {
      printf("widen mismatch at %08llx\n", (unsigned long long)b);
      return 1;
    }
    ++wide;
  }
  // narrow: boundary classes around binary32 values of every exponent
  for (int i = 0; i < 4000000; ++i) {
    const uint32_t fb = uint32_t(next_u64());
    const float f = u2f(fb);
    if (isnan(f) || isinf(f)) continue;
    const double a = (double)f;
    const float g = nextafterf(f, f2u(f) & 0x80000000u ? -INFINITY : INFINITY);
    const double mid = isinf(g) ? a + (a - (double)nextafterf(f, 0.0f)) / 2 : (a + (double)g) / 2;
    const double cases[6] = {a, mid, nextafter(mid, 0.0), nextafter(mid, INFINITY), nextafter(mid, -INFINITY),
                             nextafter(a, INFINITY)};
    for (double d : cases)
      if (!check_narrow(d)) return 1;
  }
  // random binary64 encodings (all exponents, the float range is a small part)
  for (int i = 0; i < 4000000; ++i) {
    if (!check_narrow(u2d(next_u64()))) return 1;
    // and encodings with the exponent in or near the binary32 range
    const uint64_t r = next_u64();
    const uint64_t e = 860 + (r >> 53) % 330;  // 860..1189
    if (!check_narrow(u2d((r & 0x800fffffffffffffull) | (e << 52)))) return 1;
  }
  const double fixed[] = {0.0, -0.0, INFINITY, -INFINITY, NAN, (double)FLT_MAX,
                          nextafter((double)FLT_MAX, INFINITY), (double)FLT_MAX + ldexp(1.0, 103),
                          nextafter((double)FLT_MAX + ldexp(1.0, 103), 0.0), (double)FLT_MIN,
                          nextafter((double)FLT_MIN, 0.0), (double)FLT_MIN / 2, ldexp(1.0, -149), 1.0, -1.0,
                          1.0 + ldexp(1.0, -24), 1.0 + 3 * ldexp(1.0, -24), 1e-300, 1e300};
  for (double d : fixed)
    if (!check_narrow(d)) return 1;
  printf("ok widen %lld narrow accepted %lld declined %lld\n", wide, accepted, declined);
  return 0;
}
