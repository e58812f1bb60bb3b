// Arithmetic types of the operator kernels.
//
// R = double : native FP64 (2 DFMA per clock per SM on GB300).
// R = dd     : "double-float", an unevaluated sum hi + lo of two FP32 numbers
//              (|lo| <= ulp(hi)/2), about 48 significant bits, evaluated on
//              the FP32 pipes (128 lanes per clock per SM).  Built from the
//              classical error-free transformations: Knuth's TwoSum, Dekker's
//              FastTwoSum, and the FMA form of TwoProd (Dekker 1971; Knuth,
//              TAOCP vol. 2, 4.2.2).  Division and square root take one
//              Newton/Karp correction on top of the FP32 result.
// R = tf     : a first-order forward-mode (tangent) pair of FP32 numbers:
//              v, the value at the linearisation point, and t, the
//              directional derivative along a correction.  Every operation
//              applies the chain rule, so an operator evaluated on tf
//              returns J(Q) dQ, its Jacobian applied to a correction, with a
//              rounding error proportional to |dQ| (the mixed-precision
//              cycle's correction solves use it).
// Every kernel loads and stores FP64 in memory; the state update of the
// smoother stays in FP64.
#pragma once

#include <cuda_runtime.h>

#include <cmath>

namespace dg {

#define DGR __device__ __forceinline__

struct dd {
  float hi, lo;
  dd() = default;
  DGR constexpr dd(float h, float l) : hi(h), lo(l) {}
  // exact split of a double into a (rounded-to-48-bit) pair
  DGR explicit dd(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
};

DGR dd fast_two_sum(float a, float b) {  // requires |a| >= |b|
  float s = a + b;
  return dd(s, b - (s - a));
}
DGR dd two_sum(float a, float b) {
  float s = a + b;
  float bb = s - a;
  return dd(s, (a - (s - bb)) + (b - bb));
}
DGR dd operator+(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  float e = s.lo + (a.lo + b.lo);
  return fast_two_sum(s.hi, e);
}
DGR dd operator-(dd a) { return dd(-a.hi, -a.lo); }
DGR dd operator-(dd a, dd b) { return a + (-b); }
DGR dd operator*(dd a, dd b) {
  float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}
DGR dd operator/(dd a, dd b) {
  float q1 = a.hi / b.hi;
  // remainder a - q1 * b, exactly enough for the correction
  float p = q1 * b.hi;
  float pe = fmaf(q1, b.hi, -p);
  dd r = a - dd(p, pe) - dd(q1 * b.lo, 0.0f);
  float q2 = r.hi / b.hi;
  return fast_two_sum(q1, q2);
}
// acc + a * b.  For dd the product's error terms are added into the sum
// without renormalising the product first (15 FP32 operations instead of
// 18); the result keeps the ~48-bit accuracy of the pair arithmetic.
DGR dd madd(dd acc, dd a, dd b) {
  float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  dd s = two_sum(acc.hi, p);
  float t = s.lo + (acc.lo + e);
  return fast_two_sum(s.hi, t);
}
DGR dd& operator+=(dd& a, dd b) { return a = a + b; }
DGR dd& operator-=(dd& a, dd b) { return a = a - b; }
DGR dd& operator*=(dd& a, dd b) { return a = a * b; }
DGR bool operator<(dd a, dd b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
DGR bool operator>(dd a, dd b) { return b < a; }
DGR dd sqrt(dd a) {
  if (a.hi <= 0.0f) return dd(0.0f, 0.0f);
  float y = sqrtf(a.hi);
  // Karp: sqrt(a) ~ y + (a - y^2) / (2 y)
  float p = y * y;
  float pe = fmaf(y, y, -p);
  dd r = a - dd(p, pe);
  return fast_two_sum(y, r.hi / (2.0f * y));
}
DGR dd fabs(dd a) { return (a.hi < 0.0f) ? -a : a; }
DGR dd fmax(dd a, dd b) { return (a < b) ? b : a; }
// ---- tangent pairs ----
struct tf {
  float v, t;
  tf() = default;
  DGR constexpr tf(float a, float b) : v(a), t(b) {}
};
DGR tf operator+(tf a, tf b) { return tf(a.v + b.v, a.t + b.t); }
DGR tf operator-(tf a) { return tf(-a.v, -a.t); }
DGR tf operator-(tf a, tf b) { return tf(a.v - b.v, a.t - b.t); }
DGR tf operator*(tf a, tf b) { return tf(a.v * b.v, fmaf(a.v, b.t, a.t * b.v)); }
DGR tf operator/(tf a, tf b) {
  const float q = a.v / b.v;
  return tf(q, (a.t - q * b.t) / b.v);  // (a/b)' = (a' - (a/b) b') / b
}
DGR tf madd(tf acc, tf a, tf b) { return tf(fmaf(a.v, b.v, acc.v), fmaf(a.v, b.t, fmaf(a.t, b.v, acc.t))); }
DGR tf& operator+=(tf& a, tf b) { return a = a + b; }
DGR tf& operator-=(tf& a, tf b) { return a = a - b; }
DGR tf& operator*=(tf& a, tf b) { return a = a * b; }
DGR bool operator<(tf a, tf b) { return a.v < b.v; }
DGR bool operator>(tf a, tf b) { return a.v > b.v; }
DGR tf sqrt(tf a) {
  if (a.v <= 0.0f) return tf(0.0f, 0.0f);
  const float r = sqrtf(a.v);
  return tf(r, 0.5f * a.t / r);  // (sqrt a)' = a' / (2 sqrt a)
}
DGR tf fabs(tf a) { return (a.v < 0.0f) ? -a : a; }  // |a|' = sign(a) a'
DGR tf fmax(tf a, tf b) { return (a.v < b.v) ? b : a; }
// the operator's output in tangent arithmetic is its derivative J(Q) dQ
DGR double to_double(tf a) { return (double)a.t; }

// the double versions live in the same namespace, so that the dd overloads
// above do not hide them
__host__ __device__ __forceinline__ double sqrt(double x) { return ::sqrt(x); }
__host__ __device__ __forceinline__ double fabs(double x) { return ::fabs(x); }
__host__ __device__ __forceinline__ double fmax(double a, double b) { return ::fmax(a, b); }
__host__ __device__ __forceinline__ double fmin(double a, double b) { return ::fmin(a, b); }

__host__ __device__ __forceinline__ double madd(double acc, double a, double b) { return ::fma(a, b, acc); }

DGR double to_double(dd a) { return (double)a.hi + (double)a.lo; }
DGR double to_double(double a) { return a; }
DGR bool is_nan(dd a) { return a.hi != a.hi; }

// ---- uniform helpers for generic kernel code ----
template <typename R>
DGR R from_double(double x);
template <>
DGR double from_double<double>(double x) {
  return x;
}
template <>
DGR dd from_double<dd>(double x) {
  return dd(x);
}
// A state value for the operator kernels: q[i] in FP64 or double-float; in
// tangent arithmetic the pair (base[i], q[i]) -- the linearisation point and
// the correction the Jacobian is applied to.
template <typename R>
DGR R state_value(const double* q, const double* base, size_t i) {
  return from_double<R>(q[i]);
}
template <>
DGR tf state_value<tf>(const double* q, const double* base, size_t i) {
  return tf((float)base[i], (float)q[i]);
}
// the same for a state value already in a register (the smoother's update)
template <typename R>
DGR R state_of(double qi, const double* base, size_t i) {
  return from_double<R>(qi);
}
template <>
DGR tf state_of<tf>(double qi, const double* base, size_t i) {
  return tf((float)base[i], (float)qi);
}

// storage type of tables for R (double for R = double, float2 for R = dd)
template <typename R>
struct Store;
template <>
struct Store<double> {
  using T = double;
  static DGR double get(const double* p, size_t i) { return p[i]; }
  static DGR void put(double* p, size_t i, double v) { p[i] = v; }
};
template <>
struct Store<dd> {
  using T = float2;
  static DGR dd get(const float2* p, size_t i) {
    float2 v = p[i];
    return dd(v.x, v.y);
  }
  static DGR void put(float2* p, size_t i, dd v) { p[i] = make_float2(v.hi, v.lo); }
};
// tangent pairs: (value, derivative); tables and geometry are stored with a
// zero derivative
template <>
struct Store<tf> {
  using T = float2;
  static DGR tf get(const float2* p, size_t i) {
    float2 v = p[i];
    return tf(v.x, v.y);
  }
  static DGR void put(float2* p, size_t i, tf v) { p[i] = make_float2(v.v, v.t); }
};

}  // namespace dg
