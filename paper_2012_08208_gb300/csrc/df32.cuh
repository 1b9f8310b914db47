// Double-word FP32 arithmetic ("double-float": a value is hi + lo with
// |lo| <= ulp(hi) / 2, about 48 significant bits) for kernels whose FP64
// arithmetic would run on GB300's FP64 pipe, 1/64 of the FP32 rate.  The
// algorithms are the classical error-free transformations (Knuth's TwoSum,
// Dekker's Fast2Sum, the FMA form of TwoProd) combined as in Joldes, Muller
// and Popescu, "Tight and rigorous error bounds for basic building blocks of
// double-word arithmetic" (ACM TOMS 44, 2017):
//   addition        AccurateDWPlusDW, relative error <= 3 u^2 (u = 2^-24), or
//                   the sloppy sum (its error bounded by the operands);
//   multiplication  DWTimesDW with the lo x lo term, relative error <= 5 u^2.
// Every FP32 operation is an explicit round-to-nearest intrinsic, so the
// compiler neither contracts nor reassociates them.
//
// The type plugs into the templated element operators (strain.cuh,
// tileop.cuh): arithmetic operators, fma, a comparison, warp shuffles and the
// read-only load are overloaded for it.
#pragma once
#include <cuda_runtime.h>

namespace tp {

// The global overloads stay visible beside the ones below (a declaration in
// tp would otherwise hide them for float and double arguments).
using ::fma;
using ::__ldg;
using ::__shfl_up_sync;
using ::__shfl_down_sync;

// A value is hi + lo.  ACC selects the addition: the accurate double-word sum
// (relative error <= 3 u^2 of the result, about 20 FP32 operations) or the
// "sloppy" one (one TwoSum and a renormalisation, 11 operations; its error is
// bounded by u^2 (|x| + |y|), the operands rather than the result, so it can
// lose relative accuracy where x + y cancels).
template <bool ACC>
struct dword {
  float hi, lo;
  __host__ __device__ constexpr dword() : hi(0.f), lo(0.f) {}
  // explicit: no float or double silently becomes a double-word (so fma on
  // doubles keeps resolving to the FP64 function)
  __host__ __device__ constexpr explicit dword(float h, float l = 0.f) : hi(h), lo(l) {}
  __host__ __device__ constexpr explicit dword(int v) : hi((float)v), lo(0.f) {}
  // nearest double-word of an FP64 value (exact for values with <= 48 significant bits)
  __host__ __device__ static dword of(double x) {
    const float h = (float)x;
    return dword(h, (float)(x - (double)h));
  }
  __host__ __device__ double to_double() const { return (double)hi + (double)lo; }
};
using df32 = dword<true>;    // accurate addition
using df32f = dword<false>;  // sloppy addition

namespace dw {
// s + e = a + b exactly (Knuth)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// s + e = a + b exactly when |a| >= |b| or a = 0 (Dekker)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
}  // namespace dw

template <bool A>
__device__ __forceinline__ dword<A> operator+(dword<A> x, dword<A> y) {
  float sh, sl, zh, zl;
  dw::two_sum(x.hi, y.hi, sh, sl);
  if constexpr (A) {
    float th, tl, vh, vl;
    dw::two_sum(x.lo, y.lo, th, tl);
    dw::fast_two_sum(sh, __fadd_rn(sl, th), vh, vl);
    dw::fast_two_sum(vh, __fadd_rn(tl, vl), zh, zl);
  } else {
    dw::fast_two_sum(sh, __fadd_rn(sl, __fadd_rn(x.lo, y.lo)), zh, zl);
  }
  return dword<A>(zh, zl);
}
template <bool A>
__device__ __forceinline__ dword<A> operator-(dword<A> x) { return dword<A>(-x.hi, -x.lo); }
template <bool A>
__device__ __forceinline__ dword<A> operator-(dword<A> x, dword<A> y) { return x + (-y); }
template <bool A>
__device__ __forceinline__ dword<A> operator*(dword<A> x, dword<A> y) {
  const float ch = __fmul_rn(x.hi, y.hi);
  const float cl1 = __fmaf_rn(x.hi, y.hi, -ch);  // exact low part of hi x hi
  const float tl1 = __fmaf_rn(x.hi, y.lo, __fmul_rn(x.lo, y.lo));
  const float cl2 = __fmaf_rn(x.lo, y.hi, tl1);
  float zh, zl;
  dw::fast_two_sum(ch, __fadd_rn(cl1, cl2), zh, zl);
  return dword<A>(zh, zl);
}
template <bool A>
__device__ __forceinline__ dword<A>& operator+=(dword<A>& x, dword<A> y) { return x = x + y; }
template <bool A>
__device__ __forceinline__ dword<A>& operator-=(dword<A>& x, dword<A> y) { return x = x - y; }
template <bool A>
__device__ __forceinline__ dword<A>& operator*=(dword<A>& x, dword<A> y) { return x = x * y; }
template <bool A>
__device__ __forceinline__ dword<A> fma(dword<A> a, dword<A> b, dword<A> c) { return a * b + c; }
template <bool A>
__device__ __forceinline__ bool operator>=(dword<A> x, dword<A> y) {
  return x.hi > y.hi || (x.hi == y.hi && x.lo >= y.lo);
}

template <bool A>
__device__ __forceinline__ dword<A> __shfl_up_sync(unsigned mask, dword<A> v, unsigned delta) {
  return dword<A>(::__shfl_up_sync(mask, v.hi, delta), ::__shfl_up_sync(mask, v.lo, delta));
}
template <bool A>
__device__ __forceinline__ dword<A> __shfl_down_sync(unsigned mask, dword<A> v, unsigned delta) {
  return dword<A>(::__shfl_down_sync(mask, v.hi, delta), ::__shfl_down_sync(mask, v.lo, delta));
}
template <bool A>
__device__ __forceinline__ dword<A> __ldg(const dword<A>* p) {
  const float2 v = ::__ldg(reinterpret_cast<const float2*>(p));
  return dword<A>(v.x, v.y);
}

}  // namespace tp
