// Helpers shared by the operator, CG and sensitivity translation units.
#pragma once
#include <type_traits>

#include "host.h"
#include "tileop.cuh"

namespace tp {

// Constant-index access to small per-case register arrays (a runtime index
// into a register array would force it into local memory).
template <typename T, int N>
__device__ __forceinline__ T pick(const T (&a)[N], int i) {
  T v = a[0];
#pragma unroll
  for (int c = 1; c < N; c++)
    if (i == c) v = a[c];
  return v;
}
template <int N>
__device__ __forceinline__ void addto(double (&acc)[N], int i, double x) {
#pragma unroll
  for (int c = 0; c < N; c++)
    if (i == c) acc[c] += x;
}

template <int DIM, typename T>
inline void fill_c(CMat<DIM, T>& m, const double* C) {
  constexpr int n = DIM == 2 ? 25 : 324;
  for (int i = 0; i < n; i++) m.k[i] = (T)C[i];
}

}  // namespace tp
