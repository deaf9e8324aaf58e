/*
 * fp8_oracle.c -- FP8 E4M3 storage with one FP32 scale per 64 consecutive
 * elements, written from the format's definition.  TEST INFRASTRUCTURE ONLY
 * (tests/, __graft_entry__.smoke() and bench.py's CPU legs); shares nothing
 * with the CUDA path.
 *
 * E4M3 (the "fn" variant: no infinities, one NaN pattern per sign): 1 sign
 * bit, 4 exponent bits with bias 7, 3 mantissa bits.  Exponent field 0 holds
 * the subnormals m/8 * 2^-6; exponent field e > 0 holds (1 + m/8) * 2^(e-7);
 * e = 15 with m = 7 is NaN, so the largest finite magnitude is 1.75 * 2^8 =
 * 448.
 *
 * Quantisation of a slab x[0..63] (the last slab may be shorter), the reading
 * of "per-64-slab scales" used here: amax = max |x_i| (FP32), s = amax / 448
 * in FP32 (s = 1 when amax = 0), q_i = E4M3 of the FP32 quotient x_i / s,
 * rounded to nearest with ties to the even code and saturated to +-448.  The
 * stored value is s * decode(q_i).
 */
#include <math.h>
#include <stdint.h>

/* Value of an E4M3 code (NaN for the two NaN codes). */
double orc_e4m3_decode(int code) {
  const int sign = (code >> 7) & 1, e = (code >> 3) & 15, m = code & 7;
  if (e == 15 && m == 7) return NAN;
  const double mag = (e == 0) ? ldexp((double)m / 8.0, -6) : ldexp(1.0 + (double)m / 8.0, e - 7);
  return sign ? -mag : mag;
}

/* E4M3 code of v: nearest representable value, ties to the even code,
 * magnitudes beyond 448 saturate to 448, NaN gives 0x7F. */
int orc_e4m3_encode(float v) {
  if (v != v) return 0x7F;
  const int sign = signbit(v) ? 0x80 : 0;
  const double a = fabs((double)v);
  if (a >= 448.0) return sign | 0x7E;
  /* positive codes 0x00 .. 0x7E increase with their value: find the last code
   * whose value is <= a, then compare with the next one */
  int lo = 0, hi = 0x7E;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (orc_e4m3_decode(mid) <= a) lo = mid;
    else hi = mid - 1;
  }
  int code = lo;
  if (lo < 0x7E) {
    const double dl = a - orc_e4m3_decode(lo), dh = orc_e4m3_decode(lo + 1) - a;
    if (dh < dl || (dh == dl && (lo & 1))) code = lo + 1;
  }
  return sign | code;
}

/* Quantise n floats: q[n] codes, s[ceil(n / 64)] scales. */
void orc_fp8_quantize(int64_t n, const float* x, unsigned char* q, float* s) {
  for (int64_t j0 = 0; j0 < n; j0 += 64) {
    const int64_t j1 = (j0 + 64 < n) ? j0 + 64 : n;
    float amax = 0.0f;
    for (int64_t i = j0; i < j1; ++i) {
      const float a = fabsf(x[i]);
      if (a > amax) amax = a;
    }
    const float sc = (amax > 0.0f) ? amax / 448.0f : 1.0f;
    s[j0 / 64] = sc;
    for (int64_t i = j0; i < j1; ++i) {
      const float t = x[i] / sc;
      q[i] = (unsigned char)orc_e4m3_encode(t);
    }
  }
}

/* out[i] = s[i / 64] * decode(q[i]) in double (exact). */
void orc_fp8_dequantize(int64_t n, const unsigned char* q, const float* s, double* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = (double)s[i / 64] * orc_e4m3_decode(q[i]);
}
