// The learned warm start: a small 3D convolutional U-Net on the element grid,
// with hand-written forward / backward / Adam kernels.  Weights and stored
// activations are bfloat16; every product is accumulated in FP32; gradients are
// FP32; Adam keeps FP32 master weights.  (The paper has no network: this is the
// learned PCG warm start that sits beside the solver.)
//
// Layout: activations [n][C][D][H][W] (D = z, H = y, W = x); 3 x 3 x 3 weights
// [C_out][C_in][27], tap t = (dz+1)*9 + (dy+1)*3 + (dx+1), zero padding 1.
// Topology (the same as the oracle's network):
//   enc0 conv(in,c0) conv(c0,c0)=s0 pool | enc1 conv(c0,c1) conv(c1,c1)=s1 pool |
//   enc2 conv(c1,c2) conv(c2,c2)=s2 pool | mid conv(c2,c3) up +s2 |
//   dec2 conv(c3,c1) up +s1 | dec1 conv(c1,c0) up +s0 | dec0 conv(c0,c0) | head conv(c0,out)
// ReLU after every convolution except the head.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "../../include/topo_nn.h"
#include "common.cuh"

namespace tpn {

constexpr int TXV = 8, TYV = 8, TZV = 4;  // voxel tile of the convolution kernels (256 threads)
constexpr int HXV = TXV + 2, HYV = TYV + 2, HZV = TZV + 2;
constexpr int HALO = HXV * HYV * HZV;      // 600 values
constexpr int KC = 4;                      // input channels staged per pass

__device__ __forceinline__ float ld_as_float(const __nv_bfloat16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ float ld_as_float(const float* p) { return *p; }
__device__ __forceinline__ void st_from_float(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ void st_from_float(float* p, float v) { *p = v; }

// y[n][co][v] = bias[co] + sum_{ci,t} w[co][ci][t] x[n][ci][v + tap t]  (optional ReLU).
// One CTA computes all CO output channels of an 8 x 8 x 4 voxel tile; the input
// halo and the weights of KC input channels are staged in shared memory per pass.
template <int CO, typename TIN, typename TOUT>
__global__ void __launch_bounds__(256) conv_fwd_kernel(const TIN* __restrict__ x, const __nv_bfloat16* __restrict__ w,
                                                       const float* __restrict__ bias, TOUT* __restrict__ y, int ci_n,
                                                       int D, int H, int W, int relu, int tiles_x, int tiles_y) {
  __shared__ float s_in[KC * HALO];
  __shared__ __align__(16) float s_w[KC * 27 * CO];  // [k][t][co]
  const int n = blockIdx.y;
  const int t = blockIdx.x;
  const int x0 = (t % tiles_x) * TXV, y0 = ((t / tiles_x) % tiles_y) * TYV, z0 = (t / (tiles_x * tiles_y)) * TZV;
  const int tx = threadIdx.x % TXV, ty = (threadIdx.x / TXV) % TYV, tz = threadIdx.x / (TXV * TYV);
  const long long vol = (long long)D * H * W;
  float acc[CO];
#pragma unroll
  for (int c = 0; c < CO; c++) acc[c] = 0.f;
  for (int cb = 0; cb < ci_n; cb += KC) {
    const int kn = min(KC, ci_n - cb);
    for (int i = threadIdx.x; i < kn * HALO; i += blockDim.x) {
      const int k = i / HALO, h = i - k * HALO;
      const int hx = h % HXV, hy = (h / HXV) % HYV, hz = h / (HXV * HYV);
      const int gx = x0 - 1 + hx, gy = y0 - 1 + hy, gz = z0 - 1 + hz;
      float v = 0.f;
      if (gx >= 0 && gx < W && gy >= 0 && gy < H && gz >= 0 && gz < D)
        v = ld_as_float(x + ((long long)n * ci_n + cb + k) * vol + ((long long)gz * H + gy) * W + gx);
      s_in[i] = v;
    }
    for (int i = threadIdx.x; i < kn * 27 * CO; i += blockDim.x) {
      const int co = i % CO, r = i / CO, tap = r % 27, k = r / 27;
      s_w[i] = __bfloat162float(w[((long long)co * ci_n + cb + k) * 27 + tap]);
    }
    __syncthreads();
    for (int k = 0; k < kn; k++) {
      const float* si = s_in + k * HALO;
      const float* sw = s_w + k * 27 * CO;
#pragma unroll
      for (int tap = 0; tap < 27; tap++) {
        const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
        const float xv = si[((tz + 1 + dz) * HYV + (ty + 1 + dy)) * HXV + (tx + 1 + dx)];
#pragma unroll
        for (int c = 0; c < CO; c++) acc[c] = fmaf(sw[tap * CO + c], xv, acc[c]);
      }
    }
    __syncthreads();
  }
  const int gx = x0 + tx, gy = y0 + ty, gz = z0 + tz;
  if (gx < W && gy < H && gz < D) {
    const long long off = ((long long)gz * H + gy) * W + gx;
#pragma unroll
    for (int c = 0; c < CO; c++) {
      float v = acc[c] + (bias ? bias[c] : 0.f);
      if (relu) v = fmaxf(v, 0.f);
      st_from_float(y + ((long long)n * CO + c) * vol + off, v);
    }
  }
}

// Weight-gradient partials: part[chunk][co][ci][t] = sum over the chunk's voxels of
// g[n][co][v] x[n][ci][v + tap t].  Block (ci, chunk); a chunk is a fixed set of
// (sample, tile) pairs, so the later sum over chunks has a fixed order.
template <int CO>
__global__ void __launch_bounds__(256) conv_bwdw_kernel(const __nv_bfloat16* __restrict__ x, const float* __restrict__ g,
                                                        float* __restrict__ part, int ci_n, int n_samples, int D, int H,
                                                        int W, int tiles_x, int tiles_y, int ntiles, int nchunk) {
  constexpr int CG = CO < 16 ? CO : 16;  // output channels staged per pass
  constexpr int NV = TXV * TYV * TZV;
  __shared__ float s_in[HALO];
  __shared__ float s_g[CG * NV];
  const int ci = blockIdx.x;
  const int chunk = blockIdx.y;
  const long long vol = (long long)D * H * W;
  const int total = n_samples * ntiles;
  constexpr int NPAIR = (CG * 27 + 255) / 256;  // (co, tap) pairs per thread within a group
  float acc[(CO / CG) * NPAIR];
#pragma unroll
  for (int i = 0; i < (CO / CG) * NPAIR; i++) acc[i] = 0.f;
  for (int item = chunk; item < total; item += nchunk) {
    const int n = item / ntiles, t = item % ntiles;
    const int x0 = (t % tiles_x) * TXV, y0 = ((t / tiles_x) % tiles_y) * TYV, z0 = (t / (tiles_x * tiles_y)) * TZV;
    const __nv_bfloat16* xc = x + ((long long)n * ci_n + ci) * vol;
    __syncthreads();
    for (int i = threadIdx.x; i < HALO; i += blockDim.x) {
      const int hx = i % HXV, hy = (i / HXV) % HYV, hz = i / (HXV * HYV);
      const int gx = x0 - 1 + hx, gy = y0 - 1 + hy, gz = z0 - 1 + hz;
      float v = 0.f;
      if (gx >= 0 && gx < W && gy >= 0 && gy < H && gz >= 0 && gz < D) v = __bfloat162float(xc[((long long)gz * H + gy) * W + gx]);
      s_in[i] = v;
    }
#pragma unroll
    for (int grp = 0; grp < CO / CG; grp++) {
      __syncthreads();
      for (int i = threadIdx.x; i < CG * NV; i += blockDim.x) {
        const int c = i / NV, v = i % NV;
        const int vx = v % TXV, vy = (v / TXV) % TYV, vz = v / (TXV * TYV);
        const int gx = x0 + vx, gy = y0 + vy, gz = z0 + vz;
        float gv = 0.f;
        if (gx < W && gy < H && gz < D) gv = g[((long long)n * CO + grp * CG + c) * vol + ((long long)gz * H + gy) * W + gx];
        s_g[i] = gv;
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < NPAIR; k++) {
        const int pr = threadIdx.x + k * 256;
        if (pr < CG * 27) {
          const int c = pr / 27, tap = pr % 27;
          const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
          const float* sg = s_g + c * NV;
          const float* si = s_in + (1 + dz) * HYV * HXV + (1 + dy) * HXV + (1 + dx);
          float s = 0.f;
#pragma unroll 4
          for (int v = 0; v < NV; v++) {
            const int vx = v % TXV, vy = (v / TXV) % TYV, vz = v / (TXV * TYV);
            s = fmaf(sg[v], si[(vz * HYV + vy) * HXV + vx], s);
          }
          acc[grp * NPAIR + k] += s;
        }
      }
    }
  }
#pragma unroll
  for (int grp = 0; grp < CO / CG; grp++)
#pragma unroll
    for (int k = 0; k < NPAIR; k++) {
      const int pr = threadIdx.x + k * 256;
      if (pr < CG * 27) {
        const int co = grp * CG + pr / 27, tap = pr % 27;
        part[(((long long)chunk * CO + co) * ci_n + ci) * 27 + tap] = acc[grp * NPAIR + k];
      }
    }
}

// out[i] (+)= sum_c part[c][i] in chunk order
__global__ void sum_chunks_kernel(const float* __restrict__ part, float* out, long long m, int nchunk, int accumulate) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int c = 0; c < nchunk; c++) s += part[(long long)c * m + i];
    out[i] = accumulate ? out[i] + s : s;
  }
}

// Bias gradient: gb[co] += sum over samples and voxels of g[n][co][v]
__global__ void bias_grad_kernel(const float* __restrict__ g, float* gb, int co_n, int n_samples, long long vol) {
  __shared__ float sred[32];
  const int co = blockIdx.x;
  float s = 0.f;
  for (int n = 0; n < n_samples; n++)
    for (long long v = threadIdx.x; v < vol; v += blockDim.x) s += g[((long long)n * co_n + co) * vol + v];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) t += sred[i];
    gb[co] += t;
  }
}

// wT[ci][co][26 - t] = w[co][ci][t]: weights of the data-gradient convolution
// (the adjoint of a zero-padded convolution is the convolution with the
// flipped, transposed kernel).
__global__ void flip_transpose_kernel(const __nv_bfloat16* __restrict__ w, __nv_bfloat16* wt, int co_n, int ci_n) {
  const long long m = (long long)co_n * ci_n * 27;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(i % 27);
    const long long r = i / 27;
    const int ci = (int)(r % ci_n), co = (int)(r / ci_n);
    wt[((long long)ci * co_n + co) * 27 + (26 - t)] = w[i];
  }
}

// 2 x 2 x 2 average pooling (bf16 -> bf16) and its adjoint (f32, optionally +=)
__global__ void pool_fwd_kernel(const __nv_bfloat16* __restrict__ x, __nv_bfloat16* y, long long nc, int D, int H, int W) {
  const int d = D / 2, h = H / 2, w = W / 2;
  const long long m = nc * d * h * w;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
    const int ox = (int)(i % w), oy = (int)((i / w) % h), oz = (int)((i / ((long long)w * h)) % d);
    const long long c = i / ((long long)w * h * d);
    const __nv_bfloat16* xc = x + c * D * H * W;
    float s = 0.f;
    for (int k = 0; k < 8; k++)
      s += __bfloat162float(xc[((long long)(2 * oz + (k >> 2)) * H + 2 * oy + ((k >> 1) & 1)) * W + 2 * ox + (k & 1)]);
    y[i] = __float2bfloat16_rn(s * 0.125f);
  }
}
__global__ void pool_bwd_kernel(const float* __restrict__ gy, float* gx, long long nc, int D, int H, int W, int accumulate) {
  const long long m = nc * D * H * W;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
    const int xx = (int)(i % W), yy = (int)((i / W) % H), zz = (int)((i / ((long long)W * H)) % D);
    const long long c = i / ((long long)W * H * D);
    const float v = 0.125f * gy[((c * (D / 2) + zz / 2) * (H / 2) + yy / 2) * (W / 2) + xx / 2];
    gx[i] = accumulate ? gx[i] + v : v;
  }
}
// Nearest upsampling by 2 plus a skip tensor: y = up(x) + s (bf16).  Adjoint of
// the upsampling: gx = sum of the 8 children.
__global__ void up_add_kernel(const __nv_bfloat16* __restrict__ x, const __nv_bfloat16* __restrict__ s, __nv_bfloat16* y,
                              long long nc, int D, int H, int W) {
  const long long m = nc * D * H * W;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
    const int xx = (int)(i % W), yy = (int)((i / W) % H), zz = (int)((i / ((long long)W * H)) % D);
    const long long c = i / ((long long)W * H * D);
    const float v = __bfloat162float(x[((c * (D / 2) + zz / 2) * (H / 2) + yy / 2) * (W / 2) + xx / 2]) + __bfloat162float(s[i]);
    y[i] = __float2bfloat16_rn(v);
  }
}
__global__ void up_bwd_kernel(const float* __restrict__ gy, float* gx, long long nc, int d, int h, int w) {
  const long long m = nc * d * h * w;
  const int D = 2 * d, H = 2 * h, W = 2 * w;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
    const int ox = (int)(i % w), oy = (int)((i / w) % h), oz = (int)((i / ((long long)w * h)) % d);
    const long long c = i / ((long long)w * h * d);
    const float* gc = gy + c * D * H * W;
    float s = 0.f;
    for (int k = 0; k < 8; k++) s += gc[((long long)(2 * oz + (k >> 2)) * H + 2 * oy + ((k >> 1) & 1)) * W + 2 * ox + (k & 1)];
    gx[i] = s;
  }
}
// ReLU adjoint on the post-activation values: g *= (y > 0)
__global__ void relu_bwd_kernel(const __nv_bfloat16* __restrict__ y, float* g, long long m) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x)
    if (!(__bfloat162float(y[i]) > 0.f)) g[i] = 0.f;
}
__global__ void f32_to_bf16_kernel(const float* __restrict__ a, __nv_bfloat16* b, long long m) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x)
    b[i] = __float2bfloat16_rn(a[i]);
}
// Adam on the FP32 master parameters (bias-corrected moments); refreshes the
// bf16 copies of the weights.
__global__ void adam_kernel(float* p, const float* __restrict__ g, float* m1, float* m2, __nv_bfloat16* pb, long long n,
                            float lr, float b1, float b2, float eps, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    const float v = p[i] - lr * (a / c1) / (sqrtf(b / c2) + eps);
    p[i] = v;
    pb[i] = __float2bfloat16_rn(v);
  }
}
// Mean squared error against bf16 targets: gy = 2 (y - t) / m, per-block
// partial sums of (y - t)^2 in FP64.
__global__ void mse_kernel(const float* __restrict__ y, const __nv_bfloat16* __restrict__ t, float* gy, double* part,
                           long long m) {
  __shared__ double sred[32];
  double s = 0.0;
  const float inv = 2.f / (float)m;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
    const float d = y[i] - __bfloat162float(t[i]);
    gy[i] = inv * d;
    s += (double)d * d;
  }
  double a[1] = {s};
  tp::block_sum<1>(a, sred);
  if (threadIdx.x == 0) part[blockIdx.x] = a[0];
}

int nblk(long long m) { return (int)std::min<long long>(std::max<long long>((m + 255) / 256, 1), 152 * 16); }

}  // namespace tpn

using namespace tpn;

// ===========================================================================
// Host side: the network object.

struct tpnn {
  int cin = 0, cout = 0, c[4] = {};
  cudaStream_t s = nullptr;
  struct Layer {
    int ci, co;
    long long woff, boff;  // offsets into the packed parameter vector
  };
  std::vector<Layer> L;
  long long nparam = 0;
  float* p = nullptr;   // FP32 master parameters, per layer [w (co*ci*27) | b (co)]
  float* gp = nullptr;  // gradients (same packing)
  float* m1 = nullptr;  // Adam moments
  float* m2 = nullptr;
  __nv_bfloat16* pb = nullptr;  // bf16 copy of p (the weights the kernels read)
  __nv_bfloat16* wt = nullptr;  // flipped / transposed weights of one layer
  int adam_t = 0;
  // activations of the last forward (bf16) and the backward scratch (f32)
  int n = 0, D = 0, H = 0, Wd = 0;
  std::vector<__nv_bfloat16*> act;
  float* gbuf[2] = {nullptr, nullptr};
  float* skip[3] = {nullptr, nullptr, nullptr};
  float* part = nullptr;
  long long part_size = 0;
  double* lpart = nullptr;
  float* ybuf = nullptr;  // output of tpnn_train_step's forward
  float* gybuf = nullptr;
  std::string err;
  bool fwd_ok = false;
};

namespace {

tp_status nfail(tpnn* m, tp_status s, const std::string& e) {
  if (m) m->err = e;
  return s;
}

#define NCK(call, what)                                                           \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      cudaGetLastError();                                                         \
      return nfail(m, e_ == cudaErrorMemoryAllocation ? TP_ERR_OOM : TP_ERR_CUDA, \
                   std::string(what) + ": " + cudaGetErrorString(e_));            \
    }                                                                             \
  } while (0)

// activation slots of the forward pass
enum { A_X, A_A0, A_S0, A_P0, A_A1, A_S1, A_P1, A_A2, A_S2, A_P2, A_M, A_U2, A_D2, A_U1, A_D1, A_U0, A_D0, A_N };

template <typename TIN, typename TOUT>
cudaError_t conv(cudaStream_t s, int co, const TIN* x, const __nv_bfloat16* w, const float* b, TOUT* y, int n, int ci,
                 int D, int H, int W, int relu) {
  const int tx = (W + TXV - 1) / TXV, ty = (H + TYV - 1) / TYV, tz = (D + TZV - 1) / TZV;
  dim3 grid(tx * ty * tz, n);
#define CONV_CASE(C)                                                                           \
  case C:                                                                                      \
    conv_fwd_kernel<C, TIN, TOUT><<<grid, 256, 0, s>>>(x, w, b, y, ci, D, H, W, relu, tx, ty); \
    break;
  switch (co) {
    CONV_CASE(3)
    CONV_CASE(16)
    CONV_CASE(32)
    CONV_CASE(64)
    default:
      return cudaErrorInvalidValue;
  }
#undef CONV_CASE
  return cudaGetLastError();
}

cudaError_t conv_bwdw(tpnn* m, int co, const __nv_bfloat16* x, const float* g, float* gw, int n, int ci, int D, int H,
                      int W) {
  const int tx = (W + TXV - 1) / TXV, ty = (H + TYV - 1) / TYV, tz = (D + TZV - 1) / TZV;
  const int ntiles = tx * ty * tz;
  // enough CTAs to fill the GPU (ci * nchunk >= ~2 per SM), at least 2 items each
  const int want = std::max(1, (2 * 152 + ci - 1) / ci);
  const int nchunk = std::max(1, std::min(want, (n * ntiles + 1) / 2));
  const long long need = (long long)nchunk * co * ci * 27;
  if (need > m->part_size) {
    if (m->part) cudaFree(m->part);
    m->part = nullptr;
    m->part_size = 0;
    cudaError_t e = cudaMalloc(&m->part, need * sizeof(float));
    if (e != cudaSuccess) return e;
    m->part_size = need;
  }
  dim3 grid(ci, nchunk);
#define BW_CASE(C)                                                                                     \
  case C:                                                                                              \
    conv_bwdw_kernel<C><<<grid, 256, 0, m->s>>>(x, g, m->part, ci, n, D, H, W, tx, ty, ntiles, nchunk); \
    break;
  switch (co) {
    BW_CASE(3)
    BW_CASE(16)
    BW_CASE(32)
    BW_CASE(64)
    default:
      return cudaErrorInvalidValue;
  }
#undef BW_CASE
  const long long mm = (long long)co * ci * 27;
  sum_chunks_kernel<<<nblk(mm), 256, 0, m->s>>>(m->part, gw, mm, nchunk, 1);
  return cudaGetLastError();
}

void free_acts(tpnn* m) {
  for (size_t i = 1; i < m->act.size(); i++)  // slot 0 (the input) is borrowed
    if (m->act[i]) cudaFree(m->act[i]);
  m->act.clear();
  for (auto*& q : m->gbuf) {
    if (q) cudaFree(q);
    q = nullptr;
  }
  for (auto*& q : m->skip) {
    if (q) cudaFree(q);
    q = nullptr;
  }
  if (m->ybuf) cudaFree(m->ybuf);
  if (m->gybuf) cudaFree(m->gybuf);
  m->ybuf = m->gybuf = nullptr;
}

// (Re)allocate the activation and gradient buffers for an input of n x D x H x W.
tp_status ensure_acts(tpnn* m, int n, int D, int H, int W) {
  if (!m->act.empty() && n == m->n && D == m->D && H == m->H && W == m->Wd) return TP_OK;
  free_acts(m);
  m->fwd_ok = false;
  m->n = n;
  m->D = D;
  m->H = H;
  m->Wd = W;
  const int c0 = m->c[0], c1 = m->c[1], c2 = m->c[2], c3 = m->c[3];
  const long long v0 = (long long)D * H * W, v1 = v0 / 8, v2 = v0 / 64, v3 = v0 / 512;
  const long long N = n;
  const long long sz[A_N] = {N * m->cin * v0, N * c0 * v0, N * c0 * v0, N * c0 * v1, N * c1 * v1, N * c1 * v1,
                             N * c1 * v2,     N * c2 * v2, N * c2 * v2, N * c2 * v3, N * c3 * v3, N * c2 * v2,
                             N * c1 * v2,     N * c1 * v1, N * c0 * v1, N * c0 * v0, N * c0 * v0};
  m->act.assign(A_N, nullptr);
  for (int i = 1; i < A_N; i++) NCK(cudaMalloc((void**)&m->act[i], sz[i] * 2), "alloc activation");
  long long gmax = N * m->cout * v0;
  for (int i = 0; i < A_N; i++) gmax = std::max(gmax, sz[i]);
  for (auto*& q : m->gbuf) NCK(cudaMalloc((void**)&q, gmax * 4), "alloc gradient");
  const long long vs[3] = {N * c0 * v0, N * c1 * v1, N * c2 * v2};
  for (int i = 0; i < 3; i++) NCK(cudaMalloc((void**)&m->skip[i], vs[i] * 4), "alloc skip gradient");
  NCK(cudaMalloc((void**)&m->ybuf, N * m->cout * v0 * 4), "alloc output");
  NCK(cudaMalloc((void**)&m->gybuf, N * m->cout * v0 * 4), "alloc output gradient");
  return TP_OK;
}

}  // namespace

extern "C" {

tp_status tpnn_create(int c_in, int c_out, const int* widths, void* cuda_stream, tpnn** out) {
  if (!out || !widths || c_in < 1 || c_in > 64 || c_out != 3) return TP_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < 4; i++)
    if (widths[i] != 16 && widths[i] != 32 && widths[i] != 64) return TP_ERR_ARG;
  if (widths[3] != widths[2]) return TP_ERR_ARG;  // the mid-level skip adds c3 to c2 channels
  tpnn* m = new tpnn();
  m->cin = c_in;
  m->cout = c_out;
  for (int i = 0; i < 4; i++) m->c[i] = widths[i];
  m->s = (cudaStream_t)cuda_stream;
  const int c0 = widths[0], c1 = widths[1], c2 = widths[2], c3 = widths[3];
  const int shp[11][2] = {{c0, c_in}, {c0, c0}, {c1, c0}, {c1, c1}, {c2, c1}, {c2, c2},
                          {c3, c2},   {c1, c3}, {c0, c1}, {c0, c0}, {c_out, c0}};
  long long off = 0;
  for (auto& sh : shp) {
    tpnn::Layer l;
    l.co = sh[0];
    l.ci = sh[1];
    l.woff = off;
    off += (long long)l.co * l.ci * 27;
    l.boff = off;
    off += l.co;
    m->L.push_back(l);
  }
  m->nparam = off;
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t b) {
    if (e == cudaSuccess) e = cudaMalloc(p, b);
  };
  A((void**)&m->p, off * 4);
  A((void**)&m->gp, off * 4);
  A((void**)&m->m1, off * 4);
  A((void**)&m->m2, off * 4);
  A((void**)&m->pb, off * 2);
  long long maxw = 0;
  for (auto& l : m->L) maxw = std::max(maxw, (long long)l.co * l.ci * 27);
  A((void**)&m->wt, maxw * 2);
  A((void**)&m->lpart, 152 * 16 * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(m->p, 0, off * 4);
  if (e == cudaSuccess) e = cudaMemset(m->gp, 0, off * 4);
  if (e == cudaSuccess) e = cudaMemset(m->m1, 0, off * 4);
  if (e == cudaSuccess) e = cudaMemset(m->m2, 0, off * 4);
  if (e == cudaSuccess) e = cudaMemset(m->pb, 0, off * 2);
  if (e != cudaSuccess) {
    cudaGetLastError();
    tpnn_destroy(m);
    return e == cudaErrorMemoryAllocation ? TP_ERR_OOM : TP_ERR_CUDA;
  }
  *out = m;
  return TP_OK;
}

void tpnn_destroy(tpnn* m) {
  if (!m) return;
  cudaStreamSynchronize(m->s);
  void* ptrs[] = {m->p, m->gp, m->m1, m->m2, m->pb, m->wt, m->part, m->lpart};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  free_acts(m);
  delete m;
}

const char* tpnn_last_error(const tpnn* m) { return m ? m->err.c_str() : "null network"; }

long long tpnn_param_count(const tpnn* m) { return m ? m->nparam : 0; }

tp_status tpnn_info(const tpnn* m, int* c_in, int* c_out, int* widths) {
  if (!m) return TP_ERR_ARG;
  if (c_in) *c_in = m->cin;
  if (c_out) *c_out = m->cout;
  if (widths)
    for (int i = 0; i < 4; i++) widths[i] = m->c[i];
  return TP_OK;
}

tp_status tpnn_set_params(tpnn* m, const float* src) {
  if (!m || !src) return nfail(m, TP_ERR_ARG, "null argument");
  for (long long i = 0; i < m->nparam; i++)
    if (!std::isfinite(src[i])) return nfail(m, TP_ERR_ARG, "parameters contain NaN or Inf");
  NCK(cudaMemcpyAsync(m->p, src, m->nparam * 4, cudaMemcpyHostToDevice, m->s), "copy params");
  f32_to_bf16_kernel<<<nblk(m->nparam), 256, 0, m->s>>>(m->p, m->pb, m->nparam);
  NCK(cudaGetLastError(), "cast");
  NCK(cudaMemsetAsync(m->m1, 0, m->nparam * 4, m->s), "memset");
  NCK(cudaMemsetAsync(m->m2, 0, m->nparam * 4, m->s), "memset");
  m->adam_t = 0;
  NCK(cudaStreamSynchronize(m->s), "sync");
  return TP_OK;
}

tp_status tpnn_get_params(tpnn* m, float* dst) {
  if (!m || !dst) return nfail(m, TP_ERR_ARG, "null argument");
  NCK(cudaMemcpyAsync(dst, m->p, m->nparam * 4, cudaMemcpyDeviceToHost, m->s), "copy params");
  NCK(cudaStreamSynchronize(m->s), "sync");
  return TP_OK;
}

tp_status tpnn_get_grads(tpnn* m, float* dst) {
  if (!m || !dst) return nfail(m, TP_ERR_ARG, "null argument");
  NCK(cudaMemcpyAsync(dst, m->gp, m->nparam * 4, cudaMemcpyDeviceToHost, m->s), "copy grads");
  NCK(cudaStreamSynchronize(m->s), "sync");
  return TP_OK;
}

tp_status tpnn_forward(tpnn* m, const void* x_bf16, int n, int D, int H, int W, float* y) {
  if (!m || !x_bf16 || !y) return nfail(m, TP_ERR_ARG, "null argument");
  if (n < 1 || D < 8 || H < 8 || W < 8 || D % 8 || H % 8 || W % 8)
    return nfail(m, TP_ERR_ARG, "input must be [n][c_in][D][H][W] with D, H, W >= 8 and divisible by 8");
  tp_status st = ensure_acts(m, n, D, H, W);
  if (st != TP_OK) return st;
  auto& a = m->act;
  a[A_X] = (__nv_bfloat16*)x_bf16;  // borrowed until the next forward
  auto W_ = [&](int l) { return m->pb + m->L[l].woff; };
  auto B_ = [&](int l) { return m->p + m->L[l].boff; };
  cudaStream_t s = m->s;
  const int c0 = m->c[0], c1 = m->c[1], c2 = m->c[2], c3 = m->c[3];
  const int D1 = D / 2, H1 = H / 2, W1 = W / 2, D2 = D / 4, H2 = H / 4, W2 = W / 4, D3 = D / 8, H3 = H / 8, W3 = W / 8;
  const long long N = n, v0 = (long long)D * H * W, v1 = v0 / 8, v2 = v0 / 64;
  m->fwd_ok = false;
  NCK(conv(s, c0, a[A_X], W_(0), B_(0), a[A_A0], n, m->cin, D, H, W, 1), "conv0");
  NCK(conv(s, c0, a[A_A0], W_(1), B_(1), a[A_S0], n, c0, D, H, W, 1), "conv1");
  pool_fwd_kernel<<<nblk(N * c0 * v1), 256, 0, s>>>(a[A_S0], a[A_P0], N * c0, D, H, W);
  NCK(conv(s, c1, a[A_P0], W_(2), B_(2), a[A_A1], n, c0, D1, H1, W1, 1), "conv2");
  NCK(conv(s, c1, a[A_A1], W_(3), B_(3), a[A_S1], n, c1, D1, H1, W1, 1), "conv3");
  pool_fwd_kernel<<<nblk(N * c1 * v2), 256, 0, s>>>(a[A_S1], a[A_P1], N * c1, D1, H1, W1);
  NCK(conv(s, c2, a[A_P1], W_(4), B_(4), a[A_A2], n, c1, D2, H2, W2, 1), "conv4");
  NCK(conv(s, c2, a[A_A2], W_(5), B_(5), a[A_S2], n, c2, D2, H2, W2, 1), "conv5");
  pool_fwd_kernel<<<nblk(N * c2 * v2 / 8), 256, 0, s>>>(a[A_S2], a[A_P2], N * c2, D2, H2, W2);
  NCK(conv(s, c3, a[A_P2], W_(6), B_(6), a[A_M], n, c2, D3, H3, W3, 1), "conv6");
  up_add_kernel<<<nblk(N * c2 * v2), 256, 0, s>>>(a[A_M], a[A_S2], a[A_U2], N * c2, D2, H2, W2);
  NCK(conv(s, c1, a[A_U2], W_(7), B_(7), a[A_D2], n, c3, D2, H2, W2, 1), "conv7");
  up_add_kernel<<<nblk(N * c1 * v1), 256, 0, s>>>(a[A_D2], a[A_S1], a[A_U1], N * c1, D1, H1, W1);
  NCK(conv(s, c0, a[A_U1], W_(8), B_(8), a[A_D1], n, c1, D1, H1, W1, 1), "conv8");
  up_add_kernel<<<nblk(N * c0 * v0), 256, 0, s>>>(a[A_D1], a[A_S0], a[A_U0], N * c0, D, H, W);
  NCK(conv(s, c0, a[A_U0], W_(9), B_(9), a[A_D0], n, c0, D, H, W, 1), "conv9");
  NCK(conv(s, m->cout, a[A_D0], W_(10), B_(10), y, n, c0, D, H, W, 0), "conv10");
  m->fwd_ok = true;
  return TP_OK;
}

tp_status tpnn_backward(tpnn* m, const float* gy) {
  if (!m || !gy) return nfail(m, TP_ERR_ARG, "null argument");
  if (!m->fwd_ok) return nfail(m, TP_ERR_STATE, "tpnn_forward must precede tpnn_backward");
  cudaStream_t s = m->s;
  auto& a = m->act;
  const int n = m->n, D = m->D, H = m->H, W = m->Wd;
  const int c0 = m->c[0], c1 = m->c[1], c2 = m->c[2], c3 = m->c[3];
  const int D1 = D / 2, H1 = H / 2, W1 = W / 2, D2 = D / 4, H2 = H / 4, W2 = W / 4, D3 = D / 8, H3 = H / 8, W3 = W / 8;
  float* G0 = m->gbuf[0];
  float* G1 = m->gbuf[1];
  const long long N = n, V0 = (long long)D * H * W, V1 = V0 / 8, V2 = V0 / 64, V3 = V0 / 512;
  // Backward of one convolution: weight and bias gradients from (input
  // activation, output gradient); data gradient into gx when gx != nullptr.
  auto bconv = [&](int l, const __nv_bfloat16* xin, const float* g, float* gx, int ci, int co, int Dd, int Hh,
                   int Ww) -> cudaError_t {
    cudaError_t e = conv_bwdw(m, co, xin, g, m->gp + m->L[l].woff, n, ci, Dd, Hh, Ww);
    if (e != cudaSuccess) return e;
    bias_grad_kernel<<<co, 256, 0, s>>>(g, m->gp + m->L[l].boff, co, n, (long long)Dd * Hh * Ww);
    if (gx) {
      flip_transpose_kernel<<<nblk((long long)co * ci * 27), 256, 0, s>>>(m->pb + m->L[l].woff, m->wt, co, ci);
      e = conv<float, float>(s, ci, g, m->wt, nullptr, gx, n, co, Dd, Hh, Ww, 0);
      if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
  };
  auto relub = [&](const __nv_bfloat16* y, float* g, long long cnt) {
    relu_bwd_kernel<<<nblk(cnt), 256, 0, s>>>(y, g, cnt);
  };
  const cudaMemcpyKind dd = cudaMemcpyDeviceToDevice;
  // head (no ReLU): input d0
  NCK(bconv(10, a[A_D0], gy, G0, c0, m->cout, D, H, W), "backward conv10");
  relub(a[A_D0], G0, N * c0 * V0);
  NCK(bconv(9, a[A_U0], G0, G1, c0, c0, D, H, W), "backward conv9");  // G1 = grad u0
  NCK(cudaMemcpyAsync(m->skip[0], G1, N * c0 * V0 * 4, dd, s), "copy");
  up_bwd_kernel<<<nblk(N * c0 * V1), 256, 0, s>>>(G1, G0, N * c0, D1, H1, W1);  // grad d1
  relub(a[A_D1], G0, N * c0 * V1);
  NCK(bconv(8, a[A_U1], G0, G1, c1, c0, D1, H1, W1), "backward conv8");  // grad u1
  NCK(cudaMemcpyAsync(m->skip[1], G1, N * c1 * V1 * 4, dd, s), "copy");
  up_bwd_kernel<<<nblk(N * c1 * V2), 256, 0, s>>>(G1, G0, N * c1, D2, H2, W2);  // grad d2
  relub(a[A_D2], G0, N * c1 * V2);
  NCK(bconv(7, a[A_U2], G0, G1, c3, c1, D2, H2, W2), "backward conv7");  // grad u2
  NCK(cudaMemcpyAsync(m->skip[2], G1, N * c2 * V2 * 4, dd, s), "copy");
  up_bwd_kernel<<<nblk(N * c3 * V3), 256, 0, s>>>(G1, G0, N * c3, D3, H3, W3);  // grad m
  relub(a[A_M], G0, N * c3 * V3);
  NCK(bconv(6, a[A_P2], G0, G1, c2, c3, D3, H3, W3), "backward conv6");  // grad p2
  NCK(cudaMemcpyAsync(G0, m->skip[2], N * c2 * V2 * 4, dd, s), "copy");
  pool_bwd_kernel<<<nblk(N * c2 * V2), 256, 0, s>>>(G1, G0, N * c2, D2, H2, W2, 1);  // grad s2
  relub(a[A_S2], G0, N * c2 * V2);
  NCK(bconv(5, a[A_A2], G0, G1, c2, c2, D2, H2, W2), "backward conv5");
  relub(a[A_A2], G1, N * c2 * V2);
  NCK(bconv(4, a[A_P1], G1, G0, c1, c2, D2, H2, W2), "backward conv4");  // grad p1
  NCK(cudaMemcpyAsync(G1, m->skip[1], N * c1 * V1 * 4, dd, s), "copy");
  pool_bwd_kernel<<<nblk(N * c1 * V1), 256, 0, s>>>(G0, G1, N * c1, D1, H1, W1, 1);  // grad s1
  relub(a[A_S1], G1, N * c1 * V1);
  NCK(bconv(3, a[A_A1], G1, G0, c1, c1, D1, H1, W1), "backward conv3");
  relub(a[A_A1], G0, N * c1 * V1);
  NCK(bconv(2, a[A_P0], G0, G1, c0, c1, D1, H1, W1), "backward conv2");  // grad p0
  NCK(cudaMemcpyAsync(G0, m->skip[0], N * c0 * V0 * 4, dd, s), "copy");
  pool_bwd_kernel<<<nblk(N * c0 * V0), 256, 0, s>>>(G1, G0, N * c0, D, H, W, 1);  // grad s0
  relub(a[A_S0], G0, N * c0 * V0);
  NCK(bconv(1, a[A_A0], G0, G1, c0, c0, D, H, W), "backward conv1");
  relub(a[A_A0], G1, N * c0 * V0);
  NCK(bconv(0, a[A_X], G1, nullptr, m->cin, c0, D, H, W), "backward conv0");
  NCK(cudaGetLastError(), "backward");
  return TP_OK;
}

tp_status tpnn_zero_grad(tpnn* m) {
  if (!m) return TP_ERR_ARG;
  NCK(cudaMemsetAsync(m->gp, 0, m->nparam * 4, m->s), "memset");
  return TP_OK;
}

tp_status tpnn_adam(tpnn* m, float lr, float beta1, float beta2, float eps) {
  if (!m) return TP_ERR_ARG;
  if (!(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
    return nfail(m, TP_ERR_ARG, "Adam needs lr > 0, 0 <= beta < 1, eps > 0");
  m->adam_t++;
  const float c1 = 1.f - (float)std::pow((double)beta1, m->adam_t);
  const float c2 = 1.f - (float)std::pow((double)beta2, m->adam_t);
  adam_kernel<<<nblk(m->nparam), 256, 0, m->s>>>(m->p, m->gp, m->m1, m->m2, m->pb, m->nparam, lr, beta1, beta2, eps,
                                                  c1, c2);
  NCK(cudaGetLastError(), "adam");
  return TP_OK;
}

tp_status tpnn_mse(tpnn* m, const float* y, const void* t_bf16, long long count, float* gy, double* loss) {
  if (!m || !y || !t_bf16 || !gy || count < 1) return nfail(m, TP_ERR_ARG, "bad argument");
  const int nb = nblk(count);
  mse_kernel<<<nb, 256, 0, m->s>>>(y, (const __nv_bfloat16*)t_bf16, gy, m->lpart, count);
  NCK(cudaGetLastError(), "mse");
  if (loss) {
    std::vector<double> h(nb);
    NCK(cudaMemcpyAsync(h.data(), m->lpart, nb * sizeof(double), cudaMemcpyDeviceToHost, m->s), "copy");
    NCK(cudaStreamSynchronize(m->s), "sync");
    double sum = 0.0;
    for (double v : h) sum += v;
    *loss = sum / (double)count;
  }
  return TP_OK;
}

tp_status tpnn_train_step(tpnn* m, const void* x_bf16, const void* t_bf16, int n, int D, int H, int W, float lr,
                          double* loss) {
  if (!m) return TP_ERR_ARG;
  if (n < 1 || D < 8 || H < 8 || W < 8 || D % 8 || H % 8 || W % 8)
    return nfail(m, TP_ERR_ARG, "input must be [n][c_in][D][H][W] with D, H, W >= 8 and divisible by 8");
  tp_status st = tpnn_zero_grad(m);
  if (st == TP_OK) st = ensure_acts(m, n, D, H, W);
  if (st == TP_OK) st = tpnn_forward(m, x_bf16, n, D, H, W, m->ybuf);
  if (st == TP_OK) st = tpnn_mse(m, m->ybuf, t_bf16, (long long)n * m->cout * D * H * W, m->gybuf, loss);
  if (st == TP_OK) st = tpnn_backward(m, m->gybuf);
  if (st == TP_OK) st = tpnn_adam(m, lr, 0.9f, 0.999f, 1e-8f);
  return st;
}

}  // extern "C"
