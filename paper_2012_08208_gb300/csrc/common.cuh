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
  int pad;
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_volatile_i32(const int* p) { return *(volatile const int*)p; }

// Grid-wide barrier for a cooperative launch (all CTAs co-resident).  The
// barrier word must be zeroed before the launch; `gen` is the CTA-local
// generation counter starting at 0.  The wait is bounded: on expiry the CTA
// records ERR_TIMEOUT and returns false, and every CTA returns false once the
// error word is set, so no CTA can wait forever.
__device__ __forceinline__ bool grid_sync(GridBar* b, unsigned& gen) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned nb = gridDim.x;
    __threadfence();
    const unsigned arrived = atomicAdd(&b->count, 1u);
    if (arrived == nb - 1) {
      atomicExch(&b->count, 0u);
      __threadfence();
      atomicAdd(&b->gen, 1u);
    } else {
      const long long t0 = clock64();
      while (ld_acquire_u32(&b->gen) == gen) {
        if (clock64() - t0 > kSpinCycles) {
          atomicOr(&b->err, ERR_TIMEOUT);
          break;
        }
        if (ld_volatile_i32(&b->err) & ERR_TIMEOUT) break;
      }
    }
    __threadfence();
  }
  __syncthreads();
  gen++;
  return (ld_volatile_i32(&b->err) & ERR_TIMEOUT) == 0;
}

// Deterministic reduction of NV doubles over the CTA; result valid in all threads.
// `sm` must hold 32 * NV doubles.
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
#pragma unroll
  for (int i = 0; i < NV; i++) {
    double s = 0.0;
    for (int w = 0; w < nw; w++) s += sm[w * NV + i];
    v[i] = s;
  }
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
