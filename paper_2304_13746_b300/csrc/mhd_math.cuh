// mhd_math.cuh -- per-face and per-edge arithmetic of the ideal-MHD stage (device code).
//
// Written for the FP64 pipe of sm_103a (and its FP32 pipe in the FP32-bulk variant):
// reciprocals are formed once and reused, only the upwind side's physical flux and
// star state are built, and the E^c edge formula uses the cancelled form (the cell
// sizes drop out).  The scalar type T is double (FP64 path) or float (FP32 bulk).
#pragma once
#include <cuda_runtime.h>

namespace idx {

template <typename T> struct Eps;
template <> struct Eps<double> {
  // HLLD degeneracy thresholds (relative): D_alpha ~ 0 and Bx^2 ~ 0 (HLLC limit)
  static constexpr double degen = 1e-12;
  static constexpr double hllc = 1e-12;
};
template <> struct Eps<float> {
  // FP32 keeps ~7 digits: the same tests with a threshold above its rounding level
  static constexpr float degen = 2e-6f;
  static constexpr float hllc = 2e-6f;
};

template <typename T> __device__ __forceinline__ T tmax(T a, T b) { return a < b ? b : a; }
template <typename T> __device__ __forceinline__ T tmin(T a, T b) { return b < a ? b : a; }

// Sign and order tests.  On this part an FP64 compare or min/max takes an FP64-pipe slot,
// like an FMA, and the FP64 stage is bound by that pipe, so for doubles the tests run on
// the bit pattern in the integer pipe.  FP32 compares are cheap and stay native.  For
// non-NaN arguments each equals the IEEE comparison in its name, signed zeros included.
__device__ __forceinline__ long long ibits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ bool gt0(double x) { return ibits(x) > 0; }  // x > 0
__device__ __forceinline__ bool gt0(float x) { return x > 0.f; }
__device__ __forceinline__ bool lt0(double x) {                         // x < 0
  const long long b = ibits(x);
  return b < 0 && (b << 1) != 0;  // -0 is not < 0
}
__device__ __forceinline__ bool lt0(float x) { return x < 0.f; }
template <typename T> __device__ __forceinline__ bool ge0(T x) { return !lt0(x); }  // x >= 0
// Larger of two values that are >= 0 (non-negative doubles order like their bit
// patterns); a <= b and a < b for two such values.
__device__ __forceinline__ double max_nn(double a, double b) { return ibits(a) < ibits(b) ? b : a; }
__device__ __forceinline__ float max_nn(float a, float b) { return a < b ? b : a; }
__device__ __forceinline__ bool le_nn(double a, double b) {
  return ibits(a) <= ibits(b) || (ibits(a) << 1) == 0;  // +0 <= -0 too
}
__device__ __forceinline__ bool le_nn(float a, float b) { return a <= b; }
__device__ __forceinline__ bool lt_nn(double a, double b) {
  return ibits(a) < ibits(b) && (ibits(b) << 1) != 0;
}
__device__ __forceinline__ bool lt_nn(float a, float b) { return a < b; }
// max(x, 0) for any x (a negative value or -0 gives +0)
__device__ __forceinline__ double pos_part(double x) { return ibits(x) > 0 ? x : 0.0; }
__device__ __forceinline__ float pos_part(float x) { return x > 0.f ? x : 0.f; }
// min / max of two doubles of any sign through integer keys that order like the values
__device__ __forceinline__ long long okey(double x) {
  const long long b = ibits(x);
  return b < 0 ? (b ^ 0x7fffffffffffffffll) : b;  // negative values: reverse the magnitude order
}
__device__ __forceinline__ double imin(double a, double b) { return okey(b) < okey(a) ? b : a; }
__device__ __forceinline__ double imax(double a, double b) { return okey(a) < okey(b) ? b : a; }
__device__ __forceinline__ float imin(float a, float b) { return b < a ? b : a; }
__device__ __forceinline__ float imax(float a, float b) { return a < b ? b : a; }
// 0 < x < infinity, and x finite, for doubles on the bit patterns
__device__ __forceinline__ bool pos_finite(double x) {
  return (unsigned long long)ibits(x) - 1ull < 0x7fefffffffffffffull;
}
__device__ __forceinline__ bool finite_bits(double x) {
  return ((unsigned long long)ibits(x) & 0x7ff0000000000000ull) != 0x7ff0000000000000ull;
}
// dl * dr > 0: same sign and both non-zero
__device__ __forceinline__ bool same_sign_nz(double dl, double dr, double) {
  const long long a = ibits(dl), b = ibits(dr);
  return (a ^ b) >= 0 && (a << 1) != 0 && (b << 1) != 0;
}
__device__ __forceinline__ bool same_sign_nz(float, float, float prod) { return prod > 0.f; }
__device__ __forceinline__ double tsqrt(double a);   // below the conversion helpers
// FP32 bulk: the hardware's approximate square root (one instruction, relative error near
// 2^-23) in place of the correctly rounded FP32 root, a sequence of about 11 FMA-pipe slots;
// FP32 rounding already bounds the bulk arithmetic.
__device__ __forceinline__ float tsqrt(float a) {
  float r;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
}
__device__ __forceinline__ double tabs(double a) { return fabs(a); }
__device__ __forceinline__ float tabs(float a) { return fabsf(a); }
__device__ __forceinline__ double trsqrt(double a);
__device__ __forceinline__ float trsqrt(float a) { return rsqrtf(a); }
// 1/a: the correctly rounded reciprocal in FP64; in the FP32 bulk the fast one (within 2 ulp
// of 1/a for |a| < 2^126), far below the variant's own FP32 rounding budget, where the
// correctly rounded FP32 division takes about 11 FMA slots.
__device__ __forceinline__ double trcp(double a) { return 1.0 / a; }
__device__ __forceinline__ float trcp(float a) { return __fdividef(1.0f, a); }

// float <-> double conversions rebuilt from the IEEE-754 bit layouts in the integer pipe.
// On this part the converters run on the FP64 pipe at its rate, which the FP32-bulk
// kernels otherwise spend on format changes.  Results equal the round-to-nearest-even
// conversions; inputs outside the fast ranges (subnormals, infinities, NaNs, doubles
// outside the normal float range) go to the converter.
//
// binary32 -> binary64 is exact: same sign, exponent rebiased by 1023 - 127 = 896,
// mantissa shifted left by 29.
__host__ __device__ __forceinline__ unsigned long long f2d_bits(unsigned u, bool* slow) {
  const unsigned a = u & 0x7fffffffu;
  *slow = (a - 1u) < 0x007fffffu || a >= 0x7f800000u;  // subnormal, infinity, NaN
  const unsigned hi = (u & 0x80000000u) | (a == 0u ? 0u : (a >> 3) + 0x38000000u);
  return ((unsigned long long)hi << 32) | (unsigned long long)(u << 29);
}
// binary64 -> binary32 for |x| in [2^-126, 2^128) (and zeros), on the two 32-bit words:
// the float's exponent and mantissa are the rebiased high word shifted left by 3 with
// the top 3 bits of the low word; the low word's other 29 bits round it to nearest, ties
// to even.  A carry out of the mantissa steps the exponent (up to infinity, as overflow
// under rounding to nearest).
__host__ __device__ __forceinline__ unsigned d2f_bits(unsigned hi, unsigned lo, bool* slow) {
  const unsigned ahi = hi & 0x7fffffffu;
  const bool zero = (ahi | lo) == 0u;
  *slow = !zero && (ahi - 0x38100000u) >= 0x0fe00000u;
  const unsigned q = ((ahi - 0x38000000u) << 3) | (lo >> 29);
  const unsigned up = ((lo & 0x1fffffffu) + (q & 1u)) > 0x10000000u ? 1u : 0u;
  return (hi & 0x80000000u) | (zero ? 0u : q + up);
}
// Where the fallback converter runs decides the cost, and the compiler may execute a
// guarded conversion on every lane and select afterwards.  Three forms, each used where
// it measured fastest: f2d selects (its guard compiles to a branch), d2f calls an
// out-of-line converter (a real branch; for kernels with registers to spare), d2f_warp
// runs the converter only in warps with a lane outside the fast range (no call, so no
// spills in the register-heavy sweeps).
__device__ __noinline__ float d2f_slow(double x) { return (float)x; }
__device__ __forceinline__ double f2d(float x) {
  bool slow;
  const unsigned long long b = f2d_bits(__float_as_uint(x), &slow);
  return slow ? (double)x : __longlong_as_double((long long)b);
}
__device__ __forceinline__ float d2f(double x) {
  bool slow;
  const unsigned u = d2f_bits((unsigned)__double2hiint(x), (unsigned)__double2loint(x), &slow);
  float r = __uint_as_float(u);
  if (__builtin_expect(slow, 0)) r = d2f_slow(x);
  return r;
}
// float -> double with the converter only in warps that hold a subnormal, infinite or NaN
// value (no select that would run it on every lane).
__device__ __forceinline__ double f2d_warp(float x) {
  bool slow;
  const unsigned long long b = f2d_bits(__float_as_uint(x), &slow);
  double r = __longlong_as_double((long long)b);
  if (__any_sync(__activemask(), slow)) r = slow ? (double)x : r;
  return r;
}
// N values float -> double with one vote: the converter runs only in warps where some
// lane holds a subnormal, infinite or NaN value among them (a select per value would run
// it on every lane, at the FP64 pipe's rate).
template <int N>
__device__ __forceinline__ void f2d_many(const float (&x)[N], double (&y)[N]) {
  bool slow = false;
#pragma unroll
  for (int q = 0; q < N; ++q) {
    bool s;
    y[q] = __longlong_as_double((long long)f2d_bits(__float_as_uint(x[q]), &s));
    slow |= s;
  }
  if (__any_sync(__activemask(), slow)) {
#pragma unroll
    for (int q = 0; q < N; ++q) y[q] = (double)x[q];
  }
}
// x / 2 for x the FP64 image of a float (so x is 0, infinite, NaN or has an exponent far
// above the subnormal range): the exponent field less one, in the integer pipe; exact.
__device__ __forceinline__ double half_of_f32_image(double x) {
  const unsigned hi = (unsigned)__double2hiint(x);
  const unsigned e = (hi >> 20) & 0x7ffu;
  const unsigned h = (e - 1u) < 0x7feu ? hi - 0x00100000u : hi;  // 0, inf, NaN unchanged
  return __hiloint2double((int)h, __double2loint(x));
}
// The vote names only the lanes executing it (__activemask): callers may sit behind an
// early return or a bounds test, where the rest of the warp never gets here.
__device__ __forceinline__ float d2f_warp(double x) {
  bool slow;
  const unsigned u = d2f_bits((unsigned)__double2hiint(x), (unsigned)__double2loint(x), &slow);
  float r = __uint_as_float(u);
  if (__any_sync(__activemask(), slow)) r = slow ? (float)x : r;
  return r;
}

// FP64 square root and reciprocal square root of the production kernels.  On this part
// the library's correctly rounded FP64 square root costs about 7.6 FMA slots of the FP64
// pipe, which bounds the FP64 sweeps.  Here: the FP32 hardware estimate y ~ 1/sqrt(x)
// (from x's float image, truncated; ~2^-21 relative), then two Newton-Raphson steps in
// FP64 in residual form (Markstein 1990: s <- s + (x - s^2) y/2 for the root,
// y <- y + y (1 - x y^2)/2 for its reciprocal; each residual formed by an FMA).  The
// error falls to ~1.5 e^2 after one step and ~e^3 after the second, ~2^-62 before the
// final rounding: faithful (within 1 ulp of the exact value), nearly always correctly
// rounded, and 5 (root) or 6 (reciprocal root) FP64 operations.  A warp with an argument
// outside (2^-120, 2^121), or zero, negative, infinite or NaN, takes the library function.
__device__ __forceinline__ bool nr_root_ok(double x) {
  // positive with biased exponent in [1023 - 120, 1023 + 120]; a set sign bit fails
  return ((unsigned)__double2hiint(x) >> 20) - (1023u - 120u) <= 240u;
}
__device__ __forceinline__ float nr_root_seed(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  return rsqrtf(__uint_as_float(((hi - 0x38000000u) << 3) | (lo >> 29)));
}
__device__ __forceinline__ double f2d_normal(float x) {  // x a normal float: exact
  bool slow;
  return __longlong_as_double((long long)f2d_bits(__float_as_uint(x), &slow));
}
__device__ __forceinline__ double sqrt_nr(double x) {
  if (!__all_sync(__activemask(), nr_root_ok(x))) return sqrt(x);
  const float y = nr_root_seed(x);
  const double h = f2d_normal(0.5f * y);  // y / 2, exact
  double s = x * f2d_normal(y);
  s = fma(fma(-s, s, x), h, s);
  return fma(fma(-s, s, x), h, s);
}
__device__ __forceinline__ double rsqrt_nr(double x) {
  if (!__all_sync(__activemask(), nr_root_ok(x))) return rsqrt(x);
  const float y0 = nr_root_seed(x);
  const double h = f2d_normal(0.5f * y0);
  double y = f2d_normal(y0);
  y = fma(fma(-(x * y), y, 1.0), h, y);
  return fma(fma(-(x * y), y, 1.0), h, y);
}
#ifdef IDX_STRICT_ROUNDING
__device__ __forceinline__ double tsqrt(double a) { return sqrt(a); }
__device__ __forceinline__ double trsqrt(double a) { return rsqrt(a); }
#else
__device__ __forceinline__ double tsqrt(double a) { return sqrt_nr(a); }
__device__ __forceinline__ double trsqrt(double a) { return rsqrt_nr(a); }
#endif

// Double-float values (an unevaluated sum h + l of two binary32 numbers, Dekker 1971) for
// the FP32-bulk energy-to-pressure recovery: the kinetic and magnetic energies formed on
// the FP32 pipe to ~2^-46 relative, so that only the cancellation E - K - M needs FP64.
struct DF {
  float h, l;
};
// |x| in [2^-32, 2^32), or x = 0: the range where df_split is exact to 2^-46
__device__ __forceinline__ bool df_in_range(double x) {
  const unsigned hw = (unsigned)__double2hiint(x), lw = (unsigned)__double2loint(x);
  const unsigned ahw = hw & 0x7fffffffu;
  return (ahw | lw) == 0u || ((ahw >> 20) - 991u) < 64u;  // biased exponent 1023 -/+ 32
}
// x = h + l with h the first 24 significant bits of x (truncated) and l the next 23, from
// the bit layout alone (integer pipe and one FP32 multiply), for x in df_in_range.
__device__ __forceinline__ DF df_split(double x) {
  DF r;
  const unsigned hw = (unsigned)__double2hiint(x), lw = (unsigned)__double2loint(x);
  const unsigned ahw = hw & 0x7fffffffu, sgn = hw & 0x80000000u;
  const unsigned e = ahw >> 20;  // biased exponent
  const bool zero = (ahw | lw) == 0u;
  // high part: exponent rebiased by 1023 - 127, top 23 bits of the 52-bit mantissa
  const unsigned hb = sgn | (((ahw - 0x38000000u) << 3) | (lw >> 29));
  // low part: the remaining 29 mantissa bits less their last 6, i.e. an integer below
  // 2^23 (exact through the 2^23 magic constant) in units of 2^(e - 1075 + 6)
  const float m = __fsub_rn(__uint_as_float(0x4b000000u | ((lw & 0x1fffffffu) >> 6)), 8388608.0f);
  const float sc = __uint_as_float((e - 942u) << 23);  // 2^(e - 1069)
  r.h = zero ? 0.f : __uint_as_float(hb);
  r.l = zero ? 0.f : __uint_as_float(__float_as_uint(__fmul_rn(m, sc)) | sgn);
  return r;
}
// s + t = a + b exactly (Knuth's two-sum)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& t) {
  s = __fadd_rn(a, b);
  const float v = __fsub_rn(s, a);
  t = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
  DF r;
  float t;
  two_sum(a.h, b.h, r.h, t);
  r.l = __fadd_rn(t, __fadd_rn(a.l, b.l));
  return r;
}
// a^2, dropping l^2 (2^-46 relative)
__device__ __forceinline__ DF df_sqr(DF a) {
  DF r;
  r.h = __fmul_rn(a.h, a.h);
  r.l = __fmaf_rn(a.h + a.h, a.l, __fmaf_rn(a.h, a.h, -r.h));
  return r;
}
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  DF r;
  r.h = __fmul_rn(a.h, b.h);
  r.l = __fmaf_rn(a.l, b.h, __fmaf_rn(a.h, b.l, __fmaf_rn(a.h, b.h, -r.h)));
  return r;
}
__device__ __forceinline__ DF df_sum3(DF a, DF b, DF c) { return df_add(df_add(a, b), c); }

// van Leer (harmonic) limited slope from the two one-sided differences (Sec. 2.3).
// The kernels use half the slope, dl dr / (dl + dr) (the slope is 2 dl dr / (dl + dr)): the
// face states take w -/+ slope / 2, and forming the half directly gives the same bits (the
// factors 2 and 1/2 are exact) with two multiplies fewer per variable and face.
template <typename T> __device__ __forceinline__ T vanleer_half(T dl, T dr) {
  const T prod = dl * dr;
  return same_sign_nz(dl, dr, prod) ? __fdividef(prod, dl + dr) : T(0);
}
// In FP64 the quotient is a product with the reciprocal: a reciprocal costs fewer FP64-pipe
// slots than a general division, for one more rounding (within an ulp of the quotient).  The
// test is on the rounded product itself: where dl * dr underflows to 0 (both differences
// near the subnormal range, as ahead of a blast into gas at rest) 1/(dl + dr) could overflow
// and 0 * inf give NaN; a positive product bounds |dl + dr| >= 2 sqrt(dl dr) > 4e-162.
template <> __device__ __forceinline__ double vanleer_half<double>(double dl, double dr) {
  const double prod = dl * dr;
#ifdef IDX_STRICT_ROUNDING
  return gt0(prod) ? prod / (dl + dr) : 0.0;  // one correctly rounded quotient
#else
  return gt0(prod) ? prod * (1.0 / (dl + dr)) : 0.0;
#endif
}

// The half slopes of the 7 reconstructed variables of one cell, from their one-sided
// differences.  In FP64 the 7 quotients share one reciprocal (Montgomery's trick: prefix
// products of the denominators, one reciprocal of the last, then each reciprocal by one
// product walking back), 18 products and one reciprocal in place of 7 reciprocals, on the
// FP64 pipe that bounds the sweeps.  Each reciprocal is then within a few ulps of 1/x.
// The trick runs when every denominator's exponent lies within 2^+-130, so that no prefix
// product can leave the double range; otherwise (steep fronts into near-vacuum, with
// differences near the subnormal range) each slope takes its own reciprocal.  The FP32 bulk
// and the strict-rounding build form each slope by itself.
template <int N, typename T> struct VanLeerN {
  static __device__ __forceinline__ void run(const T dl[N], const T dr[N], T out[N]) {
#pragma unroll
    for (int q = 0; q < N; ++q) out[q] = vanleer_half(dl[q], dr[q]);
  }
};
#ifndef IDX_STRICT_ROUNDING
template <int N> struct VanLeerN<N, double> {
  static __device__ __forceinline__ void run(const double dl[N], const double dr[N],
                                             double out[N]) {
    double prod[N], den[N];
    bool pos[N];
    unsigned long long bad = 0;
#pragma unroll
    for (int q = 0; q < N; ++q) {
      prod[q] = dl[q] * dr[q];
      pos[q] = gt0(prod[q]);
      den[q] = pos[q] ? dl[q] + dr[q] : 1.0;
      // biased exponent outside [1023 - 130, 1023 + 130]
      const unsigned e = (unsigned)((unsigned long long)ibits(den[q]) >> 52) & 0x7ffu;
      bad |= (unsigned long long)((e - 893u) > 260u);
    }
    if (bad) {
#pragma unroll
      for (int q = 0; q < N; ++q) out[q] = pos[q] ? prod[q] * (1.0 / den[q]) : 0.0;
      return;
    }
    double pre[N];
    pre[0] = den[0];
#pragma unroll
    for (int q = 1; q < N; ++q) pre[q] = pre[q - 1] * den[q];
    double inv = 1.0 / pre[N - 1];  // 1 / (den[0] ... den[N-1])
#pragma unroll
    for (int q = N - 1; q >= 1; --q) {
      const double r = inv * pre[q - 1];  // 1 / den[q]
      inv = inv * den[q];                 // 1 / (den[0] ... den[q-1])
      out[q] = pos[q] ? prod[q] * r : 0.0;
    }
    out[0] = pos[0] ? prod[0] * inv : 0.0;
  }
};
#endif
// the half slopes of N variables of one cell (N = 7 for the flux sweeps, 5 for the
// speed-only pass); FP64 forms them with one reciprocal as above
template <int N, typename T>
__device__ __forceinline__ void vanleer_half_n(const T dl[N], const T dr[N], T out[N]) {
  VanLeerN<N, T>::run(dl, dr, out);
}
template <typename T>
__device__ __forceinline__ void vanleer_half7(const T dl[7], const T dr[7], T out[7]) {
  VanLeerN<7, T>::run(dl, dr, out);
}

// x with its sign flipped where y is negative (x * sign(y), signed zeros included), on the
// bit patterns.
__device__ __forceinline__ double xsign(double x, double y) {
  return __longlong_as_double(ibits(x) ^ (ibits(y) & (long long)0x8000000000000000ull));
}
__device__ __forceinline__ float xsign(float x, float y) {
  return __int_as_float(__float_as_int(x) ^ (__float_as_int(y) & (int)0x80000000u));
}

// LimO3, the compact third-order reconstruction of Sec. 2.3 (Cada & Torrilhon 2009), as the
// change of a cell's value at one face: with dt the difference toward that face's
// neighbour and db the difference from the neighbour behind, the face value is
// w + phi(db / dt) dt / 2 with
//   phi(t) = max(0, min(P3, max(-t/2, min(2t, P3, 3/2)))),   P3 = (2 + t) / 3
// (P3 alone: the unlimited third-order value).  Every piece of phi is linear in t, so
// phi(db/dt) dt / 2 is the same chain in a = sign(dt) db / 2 and b = |dt| / 2 (b >= 0 keeps
// each min and max in place), formed without a division; dt = 0 gives 0, the limit.
template <typename T> __device__ __forceinline__ T limo3_half(T db, T dt) {
  const T b = T(0.5) * tabs(dt);
  const T a = T(0.5) * xsign(db, dt);
  const T p3 = (T(2) * b + a) * T(1.0 / 3.0);
  const T chain = imin(imin(T(2) * a, p3), T(1.5) * b);
  return xsign(pos_part(imin(p3, imax(T(-0.5) * a, chain))), dt);
}

// Primitive state on one side of a face, rotated so that "u" is the normal velocity.
template <typename T> struct Side {
  T r, u, v, w, p, b1, b2;  // rho, v_n, v_t1, v_t2, P, B_t1, B_t2
};

// HLLD flux (Miyoshi & Kusano 2005) at a face with normal field bx.  Output order:
// rho, m_n, m_t1, m_t2, E, B_t1, B_t2; c = max(|S_L|, |S_R|) for the CFL condition.
template <typename T>
__device__ __forceinline__ void hlld(const Side<T>& L, const Side<T>& R, T bx, T gamma,
                                     T gm1inv, T F[7], T& c) {
  const T bx2 = bx * bx;
  const T b2L = bx2 + L.b1 * L.b1 + L.b2 * L.b2, b2R = bx2 + R.b1 * R.b1 + R.b2 * R.b2;
  const T magL = T(0.5) * b2L, magR = T(0.5) * b2R;
  const T pTL = L.p + magL, pTR = R.p + magR;

  // outer speeds from the fast magnetosonic speeds (MK05 eq. 67)
  const T gpL = gamma * L.p, gpR = gamma * R.p;
  const T aL = gpL + b2L, aR = gpR + b2R;  // 2 magL is b2L exactly
  const T bx2x4 = T(4) * bx2;               // exact scaling, shared by both sides
  const T dL = pos_part(aL * aL - gpL * bx2x4);
  const T dR = pos_part(aR * aR - gpR * bx2x4);
  // 0.5/rho_L and 0.5/rho_R from one reciprocal (cheaper than a division; the factor 1/2
  // is exact)
  const T hLR = T(0.5) * trcp(L.r * R.r);
  // only the larger fast speed enters, the root of the larger square: one square root fewer
  // (with a correctly rounded root this equals the larger root bit for bit; with the
  // faithful FP64 root of the production build, within its ulp)
  const T cf2L = (aL + tsqrt(dL)) * (R.r * hLR);
  const T cf2R = (aR + tsqrt(dR)) * (L.r * hLR);
  const T cfm = tsqrt(max_nn(cf2L, cf2R));
  const T SL = imin(L.u, R.u) - cfm;
  const T SR = imax(L.u, R.u) + cfm;
  c = max_nn(tabs(SL), tabs(SR));

  const bool sup_l = gt0(SL);
  if (sup_l || lt0(SR)) {  // supersonic: upwind physical flux
    const Side<T>& s = sup_l ? L : R;
    const T pT = sup_l ? pTL : pTR;
    const T E = s.p * gm1inv + T(0.5) * s.r * (s.u * s.u + s.v * s.v + s.w * s.w) +
                (sup_l ? magL : magR);
    const T vb = s.u * bx + s.v * s.b1 + s.w * s.b2;
    const T ru = s.r * s.u;
    F[0] = ru;
    F[1] = ru * s.u + pT - bx2;
    F[2] = ru * s.v - bx * s.b1;
    F[3] = ru * s.w - bx * s.b2;
    F[4] = (E + pT) * s.u - bx * vb;
    F[5] = s.b1 * s.u - bx * s.v;
    F[6] = s.b2 * s.u - bx * s.w;
    return;
  }

  // contact speed and star total pressure
  const T sLu = SL - L.u, sRu = SR - R.u;
  const T qL = sLu * L.r, qR = sRu * R.r;
  const T SM = (qR * R.u - qL * L.u - pTR + pTL) * trcp(qR - qL);
  const T pTs = pTL + qL * (SM - L.u);

  // single-star transverse states, both sides (needed by the double-star average), with
  // D = rho (S - u)(S - S_M) - Bx^2 per side (MK05 eqs. 44-47); a side where D vanishes
  // against its terms keeps its transverse state (the HLLC limit)
  const T eL = SL - SM, eR = SR - SM;
  const T qeL = qL * eL, qeR = qR * eR;
  const T DL = qeL - bx2, DR = qeR - bx2;
  const bool degL = le_nn(tabs(DL), Eps<T>::degen * (tabs(qeL) + bx2));
  const bool degR = le_nn(tabs(DR), Eps<T>::degen * (tabs(qeR) + bx2));
  // 1/(S_L - S_M), 1/(S_R - S_M), 1/D_L and 1/D_R from one division of their product
  // (S_L < S_M < S_R: the e's are O(c_f); a degenerate side's D stays out of it)
  const T kL = degL ? T(1) : DL, kR = degR ? T(1) : DR;
  const T eLR = eL * eR, kLR = kL * kR;
  const T inv = trcp(eLR * kLR);
  const T iLR = kLR * inv, eLRinv = eLR * inv;
  const T iL = eR * iLR, iR = eL * iLR;
  const T iDL = kR * eLRinv, iDR = kL * eLRinv;
  const T rsL = qL * iL, rsR = qR * iR;  // rho*
  T vsL, wsL, b1sL, b2sL, vsR, wsR, b1sR, b2sR;
  {
    if (degL) {
      vsL = L.v; wsL = L.w; b1sL = L.b1; b2sL = L.b2;
    } else {
      const T iD = iDL;
      const T t = bx * (SM - L.u) * iD;
      vsL = L.v - L.b1 * t;
      wsL = L.w - L.b2 * t;
      const T g = (qL * sLu - bx2) * iD;
      b1sL = L.b1 * g;
      b2sL = L.b2 * g;
    }
  }
  {
    if (degR) {
      vsR = R.v; wsR = R.w; b1sR = R.b1; b2sR = R.b2;
    } else {
      const T iD = iDR;
      const T t = bx * (SM - R.u) * iD;
      vsR = R.v - R.b1 * t;
      wsR = R.w - R.b2 * t;
      const T g = (qR * sRu - bx2) * iD;
      b1sR = R.b1 * g;
      b2sR = R.b2 * g;
    }
  }

  // Alfven fan speeds
  // sqrt(rho*) and |Bx|/sqrt(rho*) from one reciprocal square root per side
  const T rqL = trsqrt(rsL), rqR = trsqrt(rsR);
  const T sqL = rsL * rqL, sqR = rsR * rqR;
  const T abx = tabs(bx);
  const T SsL = SM - abx * rqL;
  const T SsR = SM + abx * rqR;

  // the side that contains x/t = 0
  const bool left = ge0(SM);
  const Side<T>& s = left ? L : R;
  const T S = left ? SL : SR;
  const T su = left ? sLu : sRu;
  const T is = left ? iL : iR;
  const T rs = left ? rsL : rsR;
  const T pT = left ? pTL : pTR;
  const T vs = left ? vsL : vsR, ws = left ? wsL : wsR;
  const T b1s = left ? b1sL : b1sR, b2s = left ? b2sL : b2sR;

  const T E = s.p * gm1inv + T(0.5) * s.r * (s.u * s.u + s.v * s.v + s.w * s.w) +
              (left ? magL : magR);
  const T vb = s.u * bx + s.v * s.b1 + s.w * s.b2;
  const T vbs = SM * bx + vs * b1s + ws * b2s;
  const T Es = (su * E - pT * s.u + pTs * SM + bx * (vb - vbs)) * is;

  // physical flux and conserved vector of the side
  const T ru = s.r * s.u;
  T Fs[7], Us[7], Ustar[7];
  Fs[0] = ru;
  Fs[1] = ru * s.u + pT - bx2;
  Fs[2] = ru * s.v - bx * s.b1;
  Fs[3] = ru * s.w - bx * s.b2;
  Fs[4] = (E + pT) * s.u - bx * vb;
  Fs[5] = s.b1 * s.u - bx * s.v;
  Fs[6] = s.b2 * s.u - bx * s.w;
  Us[0] = s.r; Us[1] = ru; Us[2] = s.r * s.v; Us[3] = s.r * s.w; Us[4] = E;
  Us[5] = s.b1; Us[6] = s.b2;
  Ustar[0] = rs; Ustar[1] = rs * SM; Ustar[2] = rs * vs; Ustar[3] = rs * ws; Ustar[4] = Es;
  Ustar[5] = b1s; Ustar[6] = b2s;
#pragma unroll
  for (int q = 0; q < 7; ++q) F[q] = Fs[q] + S * (Ustar[q] - Us[q]);

  const bool dbl = left ? lt0(SsL) : ge0(SsR);
  if (dbl && !lt_nn(T(0.5) * bx2, Eps<T>::hllc * pTs)) {
    const T sgn = lt0(bx) ? T(-1) : T(1);
    const T isum = trcp(sqL + sqR);
    const T v2 = (sqL * vsL + sqR * vsR + (b1sR - b1sL) * sgn) * isum;
    const T w2 = (sqL * wsL + sqR * wsR + (b2sR - b2sL) * sgn) * isum;
    const T sLR = sqL * sqR;
    const T b12 = (sqL * b1sR + sqR * b1sL + sLR * (vsR - vsL) * sgn) * isum;
    const T b22 = (sqL * b2sR + sqR * b2sL + sLR * (wsR - wsL) * sgn) * isum;
    const T vb2 = SM * bx + v2 * b12 + w2 * b22;
    const T sq = left ? sqL : sqR;
    const T E2 = left ? Es - sq * (vbs - vb2) * sgn : Es + sq * (vbs - vb2) * sgn;
    const T Ss = left ? SsL : SsR;
    F[2] += Ss * (rs * v2 - Ustar[2]);
    F[3] += Ss * (rs * w2 - Ustar[3]);
    F[4] += Ss * (E2 - Es);
    F[5] += Ss * (b12 - b1s);
    F[6] += Ss * (b22 - b2s);
    // rho and m_n are continuous across the rotational waves: no change in F[0], F[1]
  }
}

// x * 2^K (K = -2, -1 or 2) by the exponent field in the integer pipe, for the FP64
// kernels that the FP64 pipe bounds: exact, the same bits as the product, where x and the
// result are normal (zeros unchanged); a warp with any other value multiplies.
template <int K>
__device__ __forceinline__ double pow2_fp64(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned e = (hi >> 20) & 0x7ffu;
  constexpr unsigned kLo = K < 0 ? (unsigned)(1 - K) : 1u;   // smallest exponent field kept normal
  constexpr unsigned kHi = K > 0 ? (unsigned)(0x7fe - K) : 0x7feu;  // largest
  const bool fast = (e - kLo) <= (kHi - kLo);
  const bool zero = ((hi & 0x7fffffffu) | lo) == 0u;
  double r = __hiloint2double((int)(fast ? hi + (unsigned)(K * (1 << 20)) : hi), (int)lo);
  if (!__all_sync(__activemask(), fast || zero)) r = x * (K == 2 ? 4.0 : (K == -1 ? 0.5 : 0.25));
  return r;
}
template <int K, typename T>
__device__ __forceinline__ T pow2_scale(T x) {
  if constexpr (sizeof(T) == 8) return pow2_fp64<K>(x);
  else return x * T(K == 2 ? 4.0 : (K == -1 ? 0.5 : 0.25));
}

// The two HLLD threshold tests in FP64 (the degeneracy |D| <= 1e-12 (|q e| + Bx^2) of a
// side, and the HLLC limit Bx^2 / 2 < 1e-12 p_T*), decided from the binary exponents in the
// integer pipe wherever those settle them, and by the FP64 comparison otherwise, in the
// warps that hold such a lane: the same decisions as the comparisons alone.  With e_x the
// biased exponent (|x| in [2^(e_x - 1023), 2^(e_x - 1022))) and 1e-12 < 2^-39.8:
//   degeneracy: 1e-12 (|q e| + Bx^2) < 2^-39.8 * 2^(e_m - 1021) with e_m the larger exponent
//     of the two terms, so e_D >= e_m - 37 gives |D| >= 2^(e_m - 1060) above it: not degenerate;
//   HLLC limit (p_T* positive and normal): e_b >= e_p - 37 with Bx^2 normal gives Bx^2/2 >=
//     2^(e_b - 1024) above 1e-12 p_T* (not the limit); e_b < e_p - 41 gives Bx^2/2 <
//     2^(e_p - 1064) below it (the limit).  Zero and subnormal values go to the comparison.
__device__ __forceinline__ int bexp(double x) {
  return (int)(((unsigned)__double2hiint(x) >> 20) & 0x7ffu);
}
__device__ __forceinline__ bool degenerate_fp64(double D, double qe, double bx2) {
  const int eq = bexp(qe), eb = bexp(bx2), eD = bexp(D);
  const bool undecided = eD == 0 || eD < (eq > eb ? eq : eb) - 37;  // D = 0 or subnormal too
  bool deg = false;
  if (__any_sync(__activemask(), undecided)) {
    const bool exact = le_nn(tabs(D), Eps<double>::degen * (tabs(qe) + bx2));
    deg = undecided && exact;
  }
  return deg;
}
__device__ __forceinline__ bool hllc_limit_fp64(double bx2, double pTs) {
  const int eb = bexp(bx2), ep = bexp(pTs);
  const bool quick = ep > 0 && !(__double2hiint(pTs) < 0);  // p_T* positive and normal
  bool lim = quick && eb < ep - 41;
  const bool undecided = !quick || (!lim && (eb == 0 || eb < ep - 37));
  if (__any_sync(__activemask(), undecided)) {
    const bool exact = lt_nn(0.5 * bx2, Eps<double>::hllc * pTs);
    lim = undecided ? exact : lim;
  }
  return lim;
}

// HLLD as above, for the FP64 sweeps, which the FP64 pipe bounds: the single-star state and
// sqrt(rho*) of the side that contains x/t = 0 are formed first, the other side's only on
// faces inside the Alfven fan, where the double-star average needs them (an Alfven root
// and about 10 operations fewer elsewhere; the same values).  The FP32 sweeps, bound by
// instruction issue, measured faster with both sides formed at once (hlld).
template <typename T>
__device__ __forceinline__ void hlld_lazy(const Side<T>& L, const Side<T>& R, T bx, T gamma,
                                     T gm1inv, T F[7], T& c) {
  const T bx2 = bx * bx;
  const T b2L = bx2 + L.b1 * L.b1 + L.b2 * L.b2, b2R = bx2 + R.b1 * R.b1 + R.b2 * R.b2;
  // p_T = p + |B|^2 / 2 with the exact halving inside the FMA (the same bits as the sum)
  const T pTL = fma(T(0.5), b2L, L.p), pTR = fma(T(0.5), b2R, R.p);

  // outer speeds from the fast magnetosonic speeds (MK05 eq. 67)
  const T gpL = gamma * L.p, gpR = gamma * R.p;
  const T aL = gpL + b2L, aR = gpR + b2R;
  const T bx2x4 = pow2_scale<2>(bx2);       // exact scaling, shared by both sides
  const T dL = pos_part(aL * aL - gpL * bx2x4);
  const T dR = pos_part(aR * aR - gpR * bx2x4);
  // 0.5/rho_L and 0.5/rho_R from one reciprocal (cheaper than a division; the factor 1/2
  // is exact)
  const T hLR = pow2_scale<-1>(trcp(L.r * R.r));
  // only the larger fast speed enters, the root of the larger square: one square root fewer
  // (with a correctly rounded root this equals the larger root bit for bit; with the
  // faithful FP64 root of the production build, within its ulp)
  const T cf2L = (aL + tsqrt(dL)) * (R.r * hLR);
  const T cf2R = (aR + tsqrt(dR)) * (L.r * hLR);
  const T cfm = tsqrt(max_nn(cf2L, cf2R));
  const T SL = imin(L.u, R.u) - cfm;
  const T SR = imax(L.u, R.u) + cfm;
  c = max_nn(tabs(SL), tabs(SR));

  const bool sup_l = gt0(SL);
  if (sup_l || lt0(SR)) {  // supersonic: upwind physical flux
    const Side<T>& s = sup_l ? L : R;
    const T pT = sup_l ? pTL : pTR;
    const T E = fma(T(0.5), sup_l ? b2L : b2R,
                    s.p * gm1inv + pow2_scale<-1>(s.r) * (s.u * s.u + s.v * s.v + s.w * s.w));
    const T vb = s.u * bx + s.v * s.b1 + s.w * s.b2;
    const T ru = s.r * s.u;
    F[0] = ru;
    F[1] = ru * s.u + pT - bx2;
    F[2] = ru * s.v - bx * s.b1;
    F[3] = ru * s.w - bx * s.b2;
    F[4] = (E + pT) * s.u - bx * vb;
    F[5] = s.b1 * s.u - bx * s.v;
    F[6] = s.b2 * s.u - bx * s.w;
    return;
  }

  // contact speed and star total pressure
  const T sLu = SL - L.u, sRu = SR - R.u;
  const T qL = sLu * L.r, qR = sRu * R.r;
  const T SM = (qR * R.u - qL * L.u - pTR + pTL) * trcp(qR - qL);
  const T pTs = pTL + qL * (SM - L.u);

  // single-star transverse states, both sides (needed by the double-star average), with
  // D = rho (S - u)(S - S_M) - Bx^2 per side (MK05 eqs. 44-47); a side where D vanishes
  // against its terms keeps its transverse state (the HLLC limit)
  const T eL = SL - SM, eR = SR - SM;
  const T qeL = qL * eL, qeR = qR * eR;
  const T DL = qeL - bx2, DR = qeR - bx2;
  const bool degL = degenerate_fp64(DL, qeL, bx2);
  const bool degR = degenerate_fp64(DR, qeR, bx2);
  // 1/(S_L - S_M), 1/(S_R - S_M), 1/D_L and 1/D_R from one division of their product
  // (S_L < S_M < S_R: the e's are O(c_f); a degenerate side's D stays out of it)
  const T kL = degL ? T(1) : DL, kR = degR ? T(1) : DR;
  const T eLR = eL * eR, kLR = kL * kR;
  const T inv = trcp(eLR * kLR);
  const T iLR = kLR * inv, eLRinv = eLR * inv;
  const T iL = eR * iLR, iR = eL * iLR;
  const T iDL = kR * eLRinv, iDR = kL * eLRinv;
  const T rsL = qL * iL, rsR = qR * iR;  // rho*
  // single-star transverse state of one side (MK05 eqs. 44-47)
  auto star_t = [&](const Side<T>& w, T q, T su, T iD, bool deg, T& vs, T& ws, T& b1s, T& b2s) {
    if (deg) {
      vs = w.v; ws = w.w; b1s = w.b1; b2s = w.b2;
    } else {
      const T t = bx * (SM - w.u) * iD;
      vs = w.v - w.b1 * t;
      ws = w.w - w.b2 * t;
      const T g = (q * su - bx2) * iD;
      b1s = w.b1 * g;
      b2s = w.b2 * g;
    }
  };

  // the side that contains x/t = 0: its single-star state and Alfven speed now; the other
  // side's only where the double-star states need them
  const bool left = ge0(SM);
  const Side<T>& s = left ? L : R;
  const T S = left ? SL : SR;
  const T su = left ? sLu : sRu;
  const T is = left ? iL : iR;
  const T rs = left ? rsL : rsR;
  const T pT = left ? pTL : pTR;
  T vs, ws, b1s, b2s;
  star_t(s, left ? qL : qR, su, left ? iDL : iDR, left ? degL : degR, vs, ws, b1s, b2s);
  // sqrt(rho*) and |Bx|/sqrt(rho*) from one reciprocal square root
  const T rq = trsqrt(rs);
  const T abx = tabs(bx);
  const T Ss = left ? SM - abx * rq : SM + abx * rq;  // the Alfven speed on that side

  const T E = fma(T(0.5), left ? b2L : b2R,
                  s.p * gm1inv + pow2_scale<-1>(s.r) * (s.u * s.u + s.v * s.v + s.w * s.w));
  const T vb = s.u * bx + s.v * s.b1 + s.w * s.b2;
  const T vbs = SM * bx + vs * b1s + ws * b2s;
  const T Es = (su * E - pT * s.u + pTs * SM + bx * (vb - vbs)) * is;

  // physical flux and conserved vector of the side
  const T ru = s.r * s.u;
  T Fs[7], Us[7], Ustar[7];
  Fs[0] = ru;
  Fs[1] = ru * s.u + pT - bx2;
  Fs[2] = ru * s.v - bx * s.b1;
  Fs[3] = ru * s.w - bx * s.b2;
  Fs[4] = (E + pT) * s.u - bx * vb;
  Fs[5] = s.b1 * s.u - bx * s.v;
  Fs[6] = s.b2 * s.u - bx * s.w;
  Us[0] = s.r; Us[1] = ru; Us[2] = s.r * s.v; Us[3] = s.r * s.w; Us[4] = E;
  Us[5] = s.b1; Us[6] = s.b2;
  Ustar[0] = rs; Ustar[1] = rs * SM; Ustar[2] = rs * vs; Ustar[3] = rs * ws; Ustar[4] = Es;
  Ustar[5] = b1s; Ustar[6] = b2s;
#pragma unroll
  for (int q = 0; q < 7; ++q) F[q] = Fs[q] + S * (Ustar[q] - Us[q]);

  const bool dbl = left ? lt0(Ss) : ge0(Ss);
  if (dbl && !hllc_limit_fp64(bx2, pTs)) {
    // the other side's single-star state and sqrt(rho*)
    T vso, wso, b1so, b2so;
    star_t(left ? R : L, left ? qR : qL, left ? sRu : sLu, left ? iDR : iDL,
           left ? degR : degL, vso, wso, b1so, b2so);
    const T rso = left ? rsR : rsL;
    const T sq = rs * rq, sqo = rso * trsqrt(rso);
    const T sqL = left ? sq : sqo, sqR = left ? sqo : sq;
    const T vsL = left ? vs : vso, vsR = left ? vso : vs;
    const T wsL = left ? ws : wso, wsR = left ? wso : ws;
    const T b1sL = left ? b1s : b1so, b1sR = left ? b1so : b1s;
    const T b2sL = left ? b2s : b2so, b2sR = left ? b2so : b2s;
    const T sgn = lt0(bx) ? T(-1) : T(1);
    const T isum = trcp(sqL + sqR);
    const T v2 = (sqL * vsL + sqR * vsR + (b1sR - b1sL) * sgn) * isum;
    const T w2 = (sqL * wsL + sqR * wsR + (b2sR - b2sL) * sgn) * isum;
    const T sLR = sqL * sqR;
    const T b12 = (sqL * b1sR + sqR * b1sL + sLR * (vsR - vsL) * sgn) * isum;
    const T b22 = (sqL * b2sR + sqR * b2sL + sLR * (wsR - wsL) * sgn) * isum;
    const T vb2 = SM * bx + v2 * b12 + w2 * b22;
    const T E2 = left ? Es - sq * (vbs - vb2) * sgn : Es + sq * (vbs - vb2) * sgn;
    F[2] += Ss * (rs * v2 - Ustar[2]);
    F[3] += Ss * (rs * w2 - Ustar[3]);
    F[4] += Ss * (E2 - Es);
    F[5] += Ss * (b12 - b1s);
    F[6] += Ss * (b22 - b2s);
    // rho and m_n are continuous across the rotational waves: no change in F[0], F[1]
  }
}

#ifdef IDX_STRICT_ROUNDING
// ---------------------------------------------------------------------------
// Strict-rounding build (a test build, compiled with -fmad=false): the FP64 HLLD with
// every formula of Miyoshi & Kusano (2005) evaluated in its plain written order -- each
// quotient a correctly rounded division, both fast speeds with their own square roots,
// both sides' star states in full, sums left to right -- so that this build rounds the
// way a plain reading of the method does.  It exists to show, on the GPU, that what
// separates the production kernels from such a reading is rounding order only: near the
// single-star degeneracy (D -> 0) any reordering is amplified by ~1/|D|.
// ---------------------------------------------------------------------------
struct StarPlain {
  double rho, v, w, by, bz, E;
};

__device__ __forceinline__ double energy_plain(const Side<double>& s, double bx, double gm1) {
  return s.p / gm1 + 0.5 * s.r * (s.u * s.u + s.v * s.v + s.w * s.w) +
         0.5 * (bx * bx + s.b1 * s.b1 + s.b2 * s.b2);
}

__device__ __forceinline__ double fast_plain(const Side<double>& s, double bx, double gamma) {
  const double gp = gamma * s.p;
  const double b2 = bx * bx + s.b1 * s.b1 + s.b2 * s.b2;
  const double a = gp + b2;
  const double disc = a * a - 4.0 * gp * bx * bx;
  return sqrt((a + sqrt(disc > 0.0 ? disc : 0.0)) / (2.0 * s.r));
}

__device__ __forceinline__ void flux_plain(const Side<double>& s, double bx, double E,
                                           double F[7]) {
  const double pT = s.p + 0.5 * (bx * bx + s.b1 * s.b1 + s.b2 * s.b2);
  const double vb = s.u * bx + s.v * s.b1 + s.w * s.b2;
  F[0] = s.r * s.u;
  F[1] = s.r * s.u * s.u + pT - bx * bx;
  F[2] = s.r * s.u * s.v - bx * s.b1;
  F[3] = s.r * s.u * s.w - bx * s.b2;
  F[4] = (E + pT) * s.u - bx * vb;
  F[5] = s.b1 * s.u - bx * s.v;
  F[6] = s.b2 * s.u - bx * s.w;
}

// max(|S_L|, |S_R|) of the outer speeds (MK05 eq. 67), plain form; also returns S_L, S_R
__device__ __forceinline__ double outer_plain(const Side<double>& L, const Side<double>& R,
                                              double bx, double gamma, double& SL, double& SR) {
  const double cfL = fast_plain(L, bx, gamma), cfR = fast_plain(R, bx, gamma);
  const double cfm = cfL < cfR ? cfR : cfL;
  SL = (R.u < L.u ? R.u : L.u) - cfm;
  SR = (L.u < R.u ? R.u : L.u) + cfm;
  const double aL = fabs(SL), aR = fabs(SR);
  return aL < aR ? aR : aL;
}

__device__ __forceinline__ void hlld_plain(const Side<double>& L, const Side<double>& R,
                                           double bx, double gamma, double F[7], double& c) {
  const double gm1 = gamma - 1.0;
  const double EL = energy_plain(L, bx, gm1), ER = energy_plain(R, bx, gm1);
  const double bx2 = bx * bx;
  const double pTL = L.p + 0.5 * (bx2 + L.b1 * L.b1 + L.b2 * L.b2);
  const double pTR = R.p + 0.5 * (bx2 + R.b1 * R.b1 + R.b2 * R.b2);
  double SL, SR;
  c = outer_plain(L, R, bx, gamma, SL, SR);
  double FL[7], FR[7];
  flux_plain(L, bx, EL, FL);
  flux_plain(R, bx, ER, FR);
  if (SL > 0.0) {
    for (int q = 0; q < 7; ++q) F[q] = FL[q];
    return;
  }
  if (SR < 0.0) {
    for (int q = 0; q < 7; ++q) F[q] = FR[q];
    return;
  }
  const double UL[7] = {L.r, L.r * L.u, L.r * L.v, L.r * L.w, EL, L.b1, L.b2};
  const double UR[7] = {R.r, R.r * R.u, R.r * R.v, R.r * R.w, ER, R.b1, R.b2};
  // contact speed and star total pressure (MK05 eqs. 38, 41)
  const double aL = (SL - L.u) * L.r, aR = (SR - R.u) * R.r;
  const double SM = (aR * R.u - aL * L.u - pTR + pTL) / (aR - aL);
  const double pTs = pTL + L.r * (SL - L.u) * (SM - L.u);
  // single-star states (MK05 eqs. 43-48)
  auto star = [&](const Side<double>& s, double S, double E, double pT) {
    StarPlain o;
    const double su = S - s.u, ssm = S - SM;
    o.rho = s.r * su / ssm;
    const double D = s.r * su * ssm - bx2;
    const double scale = fabs(s.r * su * ssm) + bx2;
    if (fabs(D) <= Eps<double>::degen * scale) {
      o.v = s.v; o.w = s.w; o.by = s.b1; o.bz = s.b2;
    } else {
      o.v = s.v - bx * s.b1 * (SM - s.u) / D;
      o.w = s.w - bx * s.b2 * (SM - s.u) / D;
      const double num = s.r * su * su - bx2;
      o.by = s.b1 * num / D;
      o.bz = s.b2 * num / D;
    }
    const double vb = s.u * bx + s.v * s.b1 + s.w * s.b2;
    const double vbs = SM * bx + o.v * o.by + o.w * o.bz;
    o.E = (su * E - pT * s.u + pTs * SM + bx * (vb - vbs)) / ssm;
    return o;
  };
  const StarPlain sl = star(L, SL, EL, pTL), sr = star(R, SR, ER, pTR);
  const double UsL[7] = {sl.rho, sl.rho * SM, sl.rho * sl.v, sl.rho * sl.w, sl.E, sl.by, sl.bz};
  const double UsR[7] = {sr.rho, sr.rho * SM, sr.rho * sr.v, sr.rho * sr.w, sr.E, sr.by, sr.bz};
  // double-star states (MK05 eqs. 51, 59-63), skipped in the HLLC limit
  const double sqL = sqrt(sl.rho), sqR = sqrt(sr.rho);
  const double SsL = SM - fabs(bx) / sqL, SsR = SM + fabs(bx) / sqR;
  double UssL[7], UssR[7];
  if (0.5 * bx2 < Eps<double>::hllc * pTs) {
    for (int q = 0; q < 7; ++q) { UssL[q] = UsL[q]; UssR[q] = UsR[q]; }
  } else {
    const double sgn = bx < 0.0 ? -1.0 : 1.0;
    const double isum = 1.0 / (sqL + sqR);
    const double v2 = (sqL * sl.v + sqR * sr.v + (sr.by - sl.by) * sgn) * isum;
    const double w2 = (sqL * sl.w + sqR * sr.w + (sr.bz - sl.bz) * sgn) * isum;
    const double by2 = (sqL * sr.by + sqR * sl.by + sqL * sqR * (sr.v - sl.v) * sgn) * isum;
    const double bz2 = (sqL * sr.bz + sqR * sl.bz + sqL * sqR * (sr.w - sl.w) * sgn) * isum;
    const double vb2 = SM * bx + v2 * by2 + w2 * bz2;
    const double vbL = SM * bx + sl.v * sl.by + sl.w * sl.bz;
    const double vbR = SM * bx + sr.v * sr.by + sr.w * sr.bz;
    const double E2L = sl.E - sqL * (vbL - vb2) * sgn;
    const double E2R = sr.E + sqR * (vbR - vb2) * sgn;
    UssL[0] = sl.rho; UssL[1] = sl.rho * SM; UssL[2] = sl.rho * v2; UssL[3] = sl.rho * w2;
    UssL[4] = E2L; UssL[5] = by2; UssL[6] = bz2;
    UssR[0] = sr.rho; UssR[1] = sr.rho * SM; UssR[2] = sr.rho * v2; UssR[3] = sr.rho * w2;
    UssR[4] = E2R; UssR[5] = by2; UssR[6] = bz2;
  }
  // flux of the region that holds x/t = 0 (MK05 eq. 66)
  if (SsL >= 0.0) {
    for (int q = 0; q < 7; ++q) F[q] = FL[q] + SL * (UsL[q] - UL[q]);
  } else if (SM >= 0.0) {
    for (int q = 0; q < 7; ++q) F[q] = FL[q] + SL * (UsL[q] - UL[q]) + SsL * (UssL[q] - UsL[q]);
  } else if (SsR >= 0.0) {
    for (int q = 0; q < 7; ++q) F[q] = FR[q] + SR * (UsR[q] - UR[q]) + SsR * (UssR[q] - UsR[q]);
  } else {
    for (int q = 0; q < 7; ++q) F[q] = FR[q] + SR * (UsR[q] - UR[q]);
  }
}

// E^c edge EMF (Gardiner & Stone 2005) in its written form, with the one-sided
// derivatives 2 (a - b) / d and the corrections (d / 8)(q3 - q1); arguments as emf_ec,
// da and db the cell sizes along a and b.
__device__ __forceinline__ double emf_ec_plain(double X0, double X1, double Y0, double Y1,
                                               double C00, double C01, double C10, double C11,
                                               double Fa0, double Fa1, double Fb0, double Fb1,
                                               double da, double db) {
  auto pick = [](double f, double up, double dn) {
    return f > 0.0 ? up : (f < 0.0 ? dn : 0.5 * (up + dn));
  };
  const double dB1 = pick(Fa0, 2.0 * (C10 - Y1) / db, 2.0 * (C00 - Y0) / db);
  const double dB3 = pick(Fa1, 2.0 * (Y1 - C11) / db, 2.0 * (Y0 - C01) / db);
  const double dA1 = pick(Fb0, 2.0 * (C01 - X1) / da, 2.0 * (C00 - X0) / da);
  const double dA3 = pick(Fb1, 2.0 * (X1 - C11) / da, 2.0 * (X0 - C10) / da);
  return 0.25 * (X0 + X1 + Y0 + Y1) + (db / 8.0) * (dB3 - dB1) + (da / 8.0) * (dA3 - dA1);
}
#endif  // IDX_STRICT_ROUNDING

// The two more diffusive solvers of the paper's list (Sec. 2.3), same interface as hlld
// and the same outer speed estimates (so the CFL speed c does not depend on the solver):
//   Rusanov:  F = (F_L + F_R)/2 - (S_max/2)(U_R - U_L), S_max = max(|u_L|+c_fL, |u_R|+c_fR)
//   HLL:      F_L if S_L > 0, F_R if S_R < 0, else
//             (S_R F_L - S_L F_R + S_L S_R (U_R - U_L)) / (S_R - S_L)
template <typename T>
__device__ __forceinline__ void side_flux(const Side<T>& s, T bx, T gm1inv, T F[7], T U[7]) {
  const T mag = T(0.5) * (bx * bx + s.b1 * s.b1 + s.b2 * s.b2);
  const T pT = s.p + mag;
  const T E = s.p * gm1inv + T(0.5) * s.r * (s.u * s.u + s.v * s.v + s.w * s.w) + mag;
  const T vb = s.u * bx + s.v * s.b1 + s.w * s.b2;
  const T ru = s.r * s.u;
  F[0] = ru;
  F[1] = ru * s.u + pT - bx * bx;
  F[2] = ru * s.v - bx * s.b1;
  F[3] = ru * s.w - bx * s.b2;
  F[4] = (E + pT) * s.u - bx * vb;
  F[5] = s.b1 * s.u - bx * s.v;
  F[6] = s.b2 * s.u - bx * s.w;
  U[0] = s.r; U[1] = ru; U[2] = s.r * s.v; U[3] = s.r * s.w; U[4] = E; U[5] = s.b1; U[6] = s.b2;
}

template <typename T>
__device__ __forceinline__ void fast_speeds(const Side<T>& L, const Side<T>& R, T bx, T gamma,
                                            T& cfL, T& cfR) {
  const T bx2 = bx * bx;
  const T gpL = gamma * L.p, gpR = gamma * R.p;
  const T aL = gpL + bx2 + L.b1 * L.b1 + L.b2 * L.b2;
  const T aR = gpR + bx2 + R.b1 * R.b1 + R.b2 * R.b2;
  const T dL = pos_part(aL * aL - T(4) * gpL * bx2);
  const T dR = pos_part(aR * aR - T(4) * gpR * bx2);
  const T hLR = T(0.5) * trcp(L.r * R.r);  // 0.5/rho_L, 0.5/rho_R from one reciprocal
  cfL = tsqrt((aL + tsqrt(dL)) * (R.r * hLR));
  cfR = tsqrt((aR + tsqrt(dR)) * (L.r * hLR));
}

// The larger of the two fast speeds, from one outer square root (see hlld).
template <typename T>
__device__ __forceinline__ T fast_speed_max(const Side<T>& L, const Side<T>& R, T bx, T gamma) {
  const T bx2 = bx * bx;
  const T gpL = gamma * L.p, gpR = gamma * R.p;
  const T aL = gpL + bx2 + L.b1 * L.b1 + L.b2 * L.b2;
  const T aR = gpR + bx2 + R.b1 * R.b1 + R.b2 * R.b2;
  const T dL = pos_part(aL * aL - T(4) * gpL * bx2);
  const T dR = pos_part(aR * aR - T(4) * gpR * bx2);
  const T hLR = T(0.5) * trcp(L.r * R.r);
  return tsqrt(max_nn((aL + tsqrt(dL)) * (R.r * hLR), (aR + tsqrt(dR)) * (L.r * hLR)));
}

template <typename T>
__device__ __forceinline__ void rusanov(const Side<T>& L, const Side<T>& R, T bx, T gamma,
                                        T gm1inv, T F[7], T& c) {
  T cfL, cfR;
  fast_speeds(L, R, bx, gamma, cfL, cfR);
  const T cfm = max_nn(cfL, cfR);
  c = max_nn(tabs(imin(L.u, R.u) - cfm), tabs(imax(L.u, R.u) + cfm));
  const T smax = max_nn(tabs(L.u) + cfL, tabs(R.u) + cfR);
  T FL[7], UL[7], FR[7], UR[7];
  side_flux(L, bx, gm1inv, FL, UL);
  side_flux(R, bx, gm1inv, FR, UR);
#pragma unroll
  for (int q = 0; q < 7; ++q) F[q] = T(0.5) * (FL[q] + FR[q]) - T(0.5) * smax * (UR[q] - UL[q]);
}

template <typename T>
__device__ __forceinline__ void hll(const Side<T>& L, const Side<T>& R, T bx, T gamma, T gm1inv,
                                    T F[7], T& c) {
  const T cfm = fast_speed_max(L, R, bx, gamma);
  const T SL = imin(L.u, R.u) - cfm;
  const T SR = imax(L.u, R.u) + cfm;
  c = max_nn(tabs(SL), tabs(SR));
  T FL[7], UL[7], FR[7], UR[7];
  side_flux(L, bx, gm1inv, FL, UL);
  side_flux(R, bx, gm1inv, FR, UR);
  if (gt0(SL)) {
#pragma unroll
    for (int q = 0; q < 7; ++q) F[q] = FL[q];
  } else if (lt0(SR)) {
#pragma unroll
    for (int q = 0; q < 7; ++q) F[q] = FR[q];
  } else {
    const T inv = trcp(SR - SL);
    const T sLR = SL * SR;
#pragma unroll
    for (int q = 0; q < 7; ++q) F[q] = (SR * FL[q] - SL * FR[q] + sLR * (UR[q] - UL[q])) * inv;
  }
}

// The CFL signal speed c = max(|S_L|, |S_R|) of a face alone, as each solver forms it (the
// same outer speed estimates and operations), for the signal-speed pass that fixes the
// first dt of a new state: no star states, no fluxes.
template <typename T>
__device__ __forceinline__ T outer_speed(int solver, const Side<T>& L, const Side<T>& R, T bx,
                                         T gamma) {
#ifdef IDX_STRICT_ROUNDING
  if constexpr (sizeof(T) == 8) {
    if (solver == 4) {
      double SL, SR;
      return outer_plain(L, R, bx, gamma, SL, SR);
    }
  }
#endif
  T cfm;
  if (solver == 4) {
    const T bx2 = bx * bx;
    const T b2L = bx2 + L.b1 * L.b1 + L.b2 * L.b2, b2R = bx2 + R.b1 * R.b1 + R.b2 * R.b2;
    const T gpL = gamma * L.p, gpR = gamma * R.p;
    const T aL = gpL + b2L, aR = gpR + b2R;
    const T bx2x4 = pow2_scale<2>(bx2);  // exact scalings, as in hlld_lazy
    const T dL = pos_part(aL * aL - gpL * bx2x4);
    const T dR = pos_part(aR * aR - gpR * bx2x4);
    const T hLR = pow2_scale<-1>(trcp(L.r * R.r));
    cfm = tsqrt(max_nn((aL + tsqrt(dL)) * (R.r * hLR), (aR + tsqrt(dR)) * (L.r * hLR)));
  } else if (solver == 2) {
    cfm = fast_speed_max(L, R, bx, gamma);
  } else {
    T cfL, cfR;
    fast_speeds(L, R, bx, gamma, cfL, cfR);
    cfm = max_nn(cfL, cfR);
  }
  return max_nn(tabs(imin(L.u, R.u) - cfm), tabs(imax(L.u, R.u) + cfm));
}

// Riemann solver by code: 1 Rusanov, 2 HLL, 4 HLLD (uniform over a sim, so warp-uniform).
template <typename T>
__device__ __forceinline__ void riemann_flux(int solver, const Side<T>& L, const Side<T>& R, T bx,
                                             T gamma, T gm1inv, T F[7], T& c) {
#ifdef IDX_STRICT_ROUNDING
  if constexpr (sizeof(T) == 8) {
    if (solver == 4) {
      hlld_plain(L, R, bx, gamma, F, c);
      return;
    }
  }
#endif
  if (solver == 4) {
    if constexpr (sizeof(T) == 8) hlld_lazy(L, R, bx, gamma, gm1inv, F, c);
    else hlld(L, R, bx, gamma, gm1inv, F, c);
  } else if (solver == 2) hll(L, R, bx, gamma, gm1inv, F, c);
  else rusanov(L, R, bx, gamma, gm1inv, F, c);
}

// E^c EMF at one edge (Gardiner & Stone 2005), cancelled form: with X, Y the a- and
// b-face EMFs, C the cell-centre EMFs and the upwind choice of each one-sided
// derivative taken from the sign of the matching face mass flux (mean at zero),
//   E = 1/4 [X0 + X1 + Y0 + Y1 + (dB3 - dB1) + (dA3 - dA1)]
// where dB1 = C(c,J) - Y(c), dB3 = Y(c) - C(c,J-1), dA1 = C(I,r) - X(r),
// dA3 = X(r) - C(I-1,r).  Index 0 = J or I, index 1 = J-1 or I-1; C[c][r].
template <typename T>
__device__ __forceinline__ T emf_ec(T X0, T X1, T Y0, T Y1, T C00, T C01, T C10, T C11, T Fa0,
                                    T Fa1, T Fb0, T Fb1) {
  // FP64 (bound by the FP64 pipe): each one-sided difference p - q is formed once, from
  // operands chosen by the flux sign (selects in the integer pipe, not arithmetic); where a
  // flux is exactly 0 the mean of both differences is formed instead, in the rare warps
  // that hold such a lane.  Same values as forming both differences and choosing between
  // them.  FP32 (bound by load latency, where the extra vote cost more than the two
  // subtractions) forms both differences and chooses.
  auto pick = [](T f, T p_up, T q_up, T p_dn, T q_dn) {
    if constexpr (sizeof(T) == 8) {
      const bool up = gt0(f);
      T r = (up ? p_up : p_dn) - (up ? q_up : q_dn);
      const bool zero = !up && !lt0(f);
      if (__any_sync(__activemask(), zero)) {
        const T m = T(0.5) * ((p_up - q_up) + (p_dn - q_dn));
        r = zero ? m : r;
      }
      return r;
    } else {
      const T up = p_up - q_up, dn = p_dn - q_dn;
      return gt0(f) ? up : (lt0(f) ? dn : T(0.5) * (up + dn));
    }
  };
  const T dB1 = pick(Fa0, C10, Y1, C00, Y0);
  const T dB3 = pick(Fa1, Y1, C11, Y0, C01);
  const T dA1 = pick(Fb0, C01, X1, C00, X0);
  const T dA3 = pick(Fb1, X1, C11, X0, C10);
  return pow2_scale<-2>((X0 + X1) + (Y0 + Y1) + (dB3 - dB1) + (dA3 - dA1));
}

}  // namespace idx
