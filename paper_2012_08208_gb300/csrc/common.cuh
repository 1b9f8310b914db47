// Shared device helpers of the GB300 SIMP library: bounded grid barrier,
// deterministic block / grid reductions, structured-grid geometry.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace tp {

constexpr int kThreads = 256;           // threads per CTA for every persistent kernel
constexpr long long kSpinCycles = 2000000000LL;  // ~1 s at 2 GHz: bound on any device wait

// Error bits written by kernels into a device status word.
enum : int { ERR_TIMEOUT = 1, ERR_BREAKDOWN = 2, ERR_NAN = 4, ERR_BOUNDS = 8 };

struct GridBar {
  unsigned int count;
  unsigned int gen;
  int err;
  unsigned int budget;  // wait limit of grid_sync in clock cycles; 0 = kSpinCycles
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_volatile_i32(const int* p) { return *(volatile const int*)p; }
// Stop flag of a graph-captured solver segment: a kernel whose flag is set
// returns at once (the flag changes only between kernels of the stream).
__device__ __forceinline__ bool halted(const int* stop) { return stop != nullptr && *stop != 0; }
// Hint: bring the line holding p into L2 (no register result).
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Grid-wide barrier for a cooperative launch (all CTAs co-resident).  The
// barrier word must be zeroed before the launch; `gen` is the CTA-local count
// of barriers passed, starting at 0.  Each CTA adds 1 to a monotone arrival
// counter with release semantics and waits (acquire) until the counter reaches
// gridDim.x * (gen + 1).  The wait is bounded: on expiry the CTA records
// ERR_TIMEOUT and returns false, and every CTA returns false once the error word
// is set, so no CTA can wait forever.  The limit is kSpinCycles unless the
// barrier word's `budget` holds a smaller nonzero cycle count (a test aid).
// The returned flag is decided by thread 0 and shared through shared memory, so
// it is uniform across the CTA (all threads take the same branch afterwards).
__device__ __forceinline__ bool grid_sync(GridBar* b, unsigned& gen) {
  __shared__ int s_ok;
  __syncthreads();
  gen++;
  if (threadIdx.x == 0) {
    const unsigned target = gen * gridDim.x;
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(&b->count), "r"(1u) : "memory");
    const unsigned bud = *(volatile const unsigned*)&b->budget;
    const long long limit = bud ? (long long)bud : kSpinCycles;
    const long long t0 = clock64();
    while (ld_acquire_u32(&b->count) < target) {
      if (clock64() - t0 > limit) {
        atomicOr(&b->err, ERR_TIMEOUT);
        break;
      }
      if (ld_volatile_i32(&b->err) & ERR_TIMEOUT) break;
    }
    s_ok = (ld_volatile_i32(&b->err) & ERR_TIMEOUT) == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

// Double-float accumulator (hi + lo, ~48-bit mantissa) built from FP32
// operations only: on GB300 an FP64 add costs 64 FP32 issue slots, so
// reductions of FP32 data accumulate in pairs of floats (TwoSum, Knuth).
struct dfl {
  float hi, lo;
};
__device__ __forceinline__ dfl dfl_add(dfl a, dfl b) {
  const float s = a.hi + b.hi;
  const float v = s - a.hi;
  float e = (a.hi - (s - v)) + (b.hi - v);
  e += a.lo + b.lo;
  const float hi = s + e;
  return dfl{hi, e - (hi - s)};
}

// CTA partial of NV per-thread FP32 values: FP32 warp trees, then one thread
// per value combines the per-warp sums in double-float and stores the pair in
// slot[i * gridDim.x + blockIdx.x].  `sm` holds 32 * NV floats.
template <int NV>
__device__ __forceinline__ void block_partial_f(float (&v)[NV], float2* slot, unsigned char* sm) {
  float* sw = reinterpret_cast<float*>(sm);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; i++) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
  }
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < NV; i++) sw[warp * NV + i] = v[i];
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    dfl s{0.f, 0.f};
    for (int w = 0; w < nw; w++) s = dfl_add(s, dfl{sw[w * NV + threadIdx.x], 0.f});
    slot[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = make_float2(s.hi, s.lo);
  }
}

// Grid total of NV per-CTA double-float partials part[i * gridDim.x + cta]
// (stored as float2): warp w sums values w, w + nw, ... over all CTAs in
// double-float, in a fixed order, so every CTA obtains the identical total.
template <int NV>
__device__ __forceinline__ void grid_total_f(const float2* part, double (&out)[NV], unsigned char* sm) {
  double* sd = reinterpret_cast<double*>(sm);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nb = gridDim.x;
  for (int i = warp; i < NV; i += nw) {
    dfl s{0.f, 0.f};
    for (int b = lane; b < nb; b += 32) {
      const float2 p = __ldcg(part + (size_t)i * nb + b);
      s = dfl_add(s, dfl{p.x, p.y});
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const dfl t{__shfl_xor_sync(0xffffffffu, s.hi, o), __shfl_xor_sync(0xffffffffu, s.lo, o)};
      s = dfl_add(s, t);
    }
    if (lane == 0) sd[i] = (double)s.hi + (double)s.lo;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; i++) out[i] = sd[i];
  __syncthreads();
}

// FP64 counterparts (the plain FP64 solver): FP64 warp trees; the per-warp and
// per-CTA sums are combined by one warp lane-parallel instead of by every thread.
template <int NV>
__device__ __forceinline__ void block_partial_d(double (&v)[NV], double* slot, unsigned char* sm) {
  double* sw = reinterpret_cast<double*>(sm);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; i++) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
  }
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < NV; i++) sw[warp * NV + i] = v[i];
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double s = 0.0;
    for (int w = 0; w < nw; w++) s += sw[w * NV + threadIdx.x];
    slot[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = s;
  }
}

template <int NV>
__device__ __forceinline__ void grid_total_d(const double* part, double (&out)[NV], unsigned char* sm) {
  double* sd = reinterpret_cast<double*>(sm);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nb = gridDim.x;
  for (int i = warp; i < NV; i += nw) {
    double s = 0.0;
    for (int b = lane; b < nb; b += 32) s += __ldcg(part + (size_t)i * nb + b);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) sd[i] = s;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; i++) out[i] = sd[i];
  __syncthreads();
}

// Deterministic reduction of NV doubles over the CTA; result valid in all
// threads.  FP64 warp trees; the per-warp sums are combined by NV threads and
// broadcast.  `sm` must hold 32 * NV doubles.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; i++) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
  }
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < NV; i++) sm[warp * NV + i] = v[i];
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double s = 0.0;
    for (int w = 0; w < nw; w++) s += sm[w * NV + threadIdx.x];
    sm[threadIdx.x] = s;  // only this thread reads warp 0's slot threadIdx.x
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; i++) v[i] = sm[i];
  __syncthreads();
}

// Sum, over all CTAs, NV per-CTA partials stored as part[i * gridDim.x + cta].
// Every CTA computes the identical total in the same fixed order.
template <int NV>
__device__ __forceinline__ void grid_total(const double* part, double (&out)[NV], double* sm) {
  const int nb = gridDim.x;
#pragma unroll
  for (int i = 0; i < NV; i++) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += __ldcg(part + (size_t)i * nb + b);
    out[i] = s;
  }
  block_sum<NV>(out, sm);
}

__device__ __forceinline__ double block_max(double v, double* sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) sm[warp] = v;
  __syncthreads();
  double m = sm[0];
  for (int w = 1; w < nw; w++) m = fmax(m, sm[w]);
  __syncthreads();
  return m;
}

// Structured-grid geometry passed by value to kernels.
struct Grid {
  int dim;
  int ex, ey, ez;   // elements per axis (ez = 1 in 2D)
  int nx, ny, nz;   // nodes per axis (nz = 1 in 2D)
  long long nn;     // nodes
  long long ne;     // elements
};

}  // namespace tp
