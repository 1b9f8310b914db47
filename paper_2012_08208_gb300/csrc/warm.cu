// Learned warm start on the problem side: network features, training targets,
// and the energy-scaled start u = alpha * u^ (declared in include/topo_nn.h).
#include <cmath>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "../../include/topo_nn.h"
#include "problem.h"

namespace {

using tp::Grid;

constexpr int kCases = tp::kMaxCases;

struct Scale {
  float v[kCases];
};

__device__ __forceinline__ long long node_of(const Grid& g, int i, int j, int k) {
  return i + (long long)g.nx * (j + (long long)g.ny * k);
}

// Per element: density, fixed-node fraction, load share (3), centre coordinates (3).
__global__ void features_kernel(Grid g, int nc, const double* __restrict__ rho, const uint8_t* __restrict__ mask,
                                const double* __restrict__ f, Scale fs, __nv_bfloat16* __restrict__ out) {
  const long long ne = g.ne;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % g.ex), j = (int)((e / g.ex) % g.ey), k = (int)(e / ((long long)g.ex * g.ey));
    int nfix = 0;
    double fl[kCases][3] = {};
    for (int c8 = 0; c8 < 8; c8++) {
      const long long nd = node_of(g, i + (c8 & 1), j + ((c8 >> 1) & 1), k + (c8 >> 2));
      nfix += mask[nd] != 0;
      for (int c = 0; c < nc; c++)
        for (int d = 0; d < 3; d++) fl[c][d] += f[((long long)c * 3 + d) * g.nn + nd];
    }
    const float r = (float)rho[e];
    const float fx = nfix * 0.125f;
    const float cx = (i + 0.5f) / g.ex, cy = (j + 0.5f) / g.ey, cz = (k + 0.5f) / g.ez;
    for (int c = 0; c < nc; c++) {
      __nv_bfloat16* o = out + (long long)c * TPNN_FEATURES * ne + e;
      const float v[TPNN_FEATURES] = {r, fx, (float)fl[c][0] * fs.v[c], (float)fl[c][1] * fs.v[c],
                                      (float)fl[c][2] * fs.v[c], cx, cy, cz};
#pragma unroll
      for (int ch = 0; ch < TPNN_FEATURES; ch++) o[ch * ne] = __float2bfloat16_rn(v[ch]);
    }
  }
}

// Element means of the displacement (x64 planar [(c*3+d)*nn + node]) into
// mean[c][3][ne]; per-block max |mean| per case into bmax[block][kCases].
__global__ void element_mean_kernel(Grid g, int nc, const double* __restrict__ x64, float* __restrict__ mean,
                                    float* __restrict__ bmax) {
  __shared__ float smax[kCases];
  if (threadIdx.x < kCases) smax[threadIdx.x] = 0.f;
  __syncthreads();
  float lmax[kCases] = {};
  const long long ne = g.ne;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % g.ex), j = (int)((e / g.ex) % g.ey), k = (int)(e / ((long long)g.ex * g.ey));
    for (int c = 0; c < nc; c++)
      for (int d = 0; d < 3; d++) {
        const double* xs = x64 + ((long long)c * 3 + d) * g.nn;
        double s = 0.0;
        for (int c8 = 0; c8 < 8; c8++) s += xs[node_of(g, i + (c8 & 1), j + ((c8 >> 1) & 1), k + (c8 >> 2))];
        const float m = (float)(0.125 * s);
        mean[((long long)c * 3 + d) * ne + e] = m;
        lmax[c] = fmaxf(lmax[c], fabsf(m));
      }
  }
  for (int c = 0; c < nc; c++) {
    float v = lmax[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    // non-negative floats order like their bit patterns
    if ((threadIdx.x & 31) == 0) atomicMax((int*)&smax[c], __float_as_int(v));
  }
  __syncthreads();
  if (threadIdx.x < kCases) bmax[(long long)blockIdx.x * kCases + threadIdx.x] = smax[threadIdx.x];
}

// dst[c][d][e] = mean[c][d][e] / max over blocks of bmax[.][c] (bf16)
__global__ void target_scale_kernel(long long ne, int nc, int nblocks, const float* __restrict__ mean,
                                    const float* __restrict__ bmax, __nv_bfloat16* __restrict__ dst) {
  __shared__ float sinv[kCases];
  if (threadIdx.x < kCases) {
    float m = 0.f;
    for (int b = 0; b < nblocks; b++) m = fmaxf(m, bmax[(long long)b * kCases + threadIdx.x]);
    sinv[threadIdx.x] = m > 0.f ? 1.f / m : 0.f;
  }
  __syncthreads();
  const long long total = (long long)nc * 3 * ne;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x)
    dst[i] = __float2bfloat16_rn(mean[i] * sinv[i / (3 * ne)]);
}

// u^ at each node: mean of the adjacent elements' outputs, 0 on fixed DOFs;
// written in the ABI layout uhat[c][node*3 + d] (FP64).
__global__ void node_average_kernel(Grid g, int nc, const float* __restrict__ y, const uint8_t* __restrict__ mask,
                                    double* __restrict__ uhat) {
  const long long nn = g.nn, ne = g.ne;
  for (long long nd = blockIdx.x * (long long)blockDim.x + threadIdx.x; nd < nn; nd += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(nd % g.nx), j = (int)((nd / g.nx) % g.ny), k = (int)(nd / ((long long)g.nx * g.ny));
    const uint8_t mk = mask[nd];
    for (int c = 0; c < nc; c++) {
      float s[3] = {0.f, 0.f, 0.f};
      int cnt = 0;
      for (int c8 = 0; c8 < 8; c8++) {
        const int ei = i - (c8 & 1), ej = j - ((c8 >> 1) & 1), ek = k - (c8 >> 2);
        if (ei < 0 || ej < 0 || ek < 0 || ei >= g.ex || ej >= g.ey || ek >= g.ez) continue;
        const long long e = ei + (long long)g.ex * (ej + (long long)g.ey * ek);
        for (int d = 0; d < 3; d++) s[d] += y[((long long)c * 3 + d) * ne + e];
        cnt++;
      }
      for (int d = 0; d < 3; d++)
        uhat[(long long)c * nn * 3 + nd * 3 + d] = ((mk >> d) & 1) ? 0.0 : (double)(s[d] / (float)cnt);
    }
  }
}

// Per-block partials of f^T u^ and u^^T (K u^) per case: part[block][2*kCases].
__global__ void warm_dots_kernel(long long nn, int nc, const double* __restrict__ f, const double* __restrict__ uhat,
                                 const double* __restrict__ kuhat, double* __restrict__ part) {
  __shared__ double sred[32 * 2 * kCases];
  double acc[2 * kCases] = {};
  const long long ndof = nn * 3;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)nc * ndof;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i / ndof);
    const long long r = i - c * ndof, nd = r / 3;
    const int d = (int)(r - nd * 3);
    const double u = uhat[i];
    const double fv = f[((long long)c * 3 + d) * nn + nd];
#pragma unroll
    for (int cc = 0; cc < kCases; cc++)
      if (cc == c) {
        acc[cc] += fv * u;
        acc[kCases + cc] += u * kuhat[i];
      }
  }
  tp::block_sum<2 * kCases>(acc, sred);
  if (threadIdx.x < 2 * kCases) part[(long long)blockIdx.x * 2 * kCases + threadIdx.x] = acc[threadIdx.x];
}

// alpha_c = (f^T u^) / (u^^T K u^) from the block partials (fixed order);
// scal[0..kCases) = alpha, scal[kCases..3 kCases) = the two dot products.
__global__ void warm_alpha_kernel(int nblocks, int nc, const double* __restrict__ part, double* __restrict__ scal) {
  const int c = threadIdx.x;
  if (c >= nc) return;
  double a = 0.0, b = 0.0;
  for (int k = 0; k < nblocks; k++) {
    a += part[(long long)k * 2 * kCases + c];
    b += part[(long long)k * 2 * kCases + kCases + c];
  }
  scal[kCases + c] = a;
  scal[2 * kCases + c] = b;
  scal[c] = (b > 0.0 && isfinite(a) && isfinite(b)) ? a / b : 0.0;
}

// x64[(c*3+d)*nn + node] = alpha_c * uhat[c][node*3 + d]
__global__ void warm_apply_kernel(long long nn, int nc, const double* __restrict__ uhat, const double* __restrict__ scal,
                                  double* __restrict__ x64) {
  const long long total = (long long)nc * nn * 3;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long v = i / nn, nd = i - v * nn;
    const int c = (int)(v / 3), d = (int)(v - 3LL * c);
    x64[i] = scal[c] * uhat[(long long)c * nn * 3 + nd * 3 + d];
  }
}

struct Comp {
  double v[kCases];
};

// g[c][node*3 + d] = -(2 alpha_c / comp_c) (f - alpha_c K u^), 0 on fixed DOFs:
// the gradient of the relative energy error 1 - alpha_c f^T u^ / comp_c.
__global__ void energy_grad_node_kernel(long long nn, int nc, const uint8_t* __restrict__ mask,
                                        const double* __restrict__ f, const double* __restrict__ kuhat,
                                        const double* __restrict__ scal, Comp comp, double* __restrict__ g) {
  const long long total = (long long)nc * nn * 3;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i / (nn * 3));
    const long long r = i - c * nn * 3, nd = r / 3;
    const int d = (int)(r - nd * 3);
    const double al = scal[c];
    const double v = -(2.0 * al / comp.v[c]) * (f[((long long)c * 3 + d) * nn + nd] - al * kuhat[i]);
    g[i] = ((mask[nd] >> d) & 1) ? 0.0 : v;
  }
}

// Adjoint of the node averaging: gy[c][d][e] = sum over the element's 8 nodes
// of g[node][d] / (number of elements adjacent to the node).
__global__ void node_average_adjoint_kernel(Grid g, int nc, const double* __restrict__ gn, float* __restrict__ gy) {
  const long long ne = g.ne, nn = g.nn;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % g.ex), j = (int)((e / g.ex) % g.ey), k = (int)(e / ((long long)g.ex * g.ey));
    for (int c = 0; c < nc; c++) {
      double s[3] = {0.0, 0.0, 0.0};
      for (int c8 = 0; c8 < 8; c8++) {
        const int ni = i + (c8 & 1), nj = j + ((c8 >> 1) & 1), nk = k + (c8 >> 2);
        const int cnt = ((ni > 0) + (ni < g.ex)) * ((nj > 0) + (nj < g.ey)) * ((nk > 0) + (nk < g.ez));
        const long long nd = node_of(g, ni, nj, nk);
        for (int d = 0; d < 3; d++) s[d] += gn[(long long)c * nn * 3 + nd * 3 + d] / cnt;
      }
      for (int d = 0; d < 3; d++) gy[((long long)c * 3 + d) * ne + e] = (float)s[d];
    }
  }
}

int blocks_for(long long n) { return (int)std::min<long long>(std::max<long long>((n + 255) / 256, 1), 152 * 8); }

tp_status wfail(tp_problem* p, tp_status s, const std::string& m) {
  if (p) p->err = m;
  return s;
}

#define WCK(call, what)                                                                               \
  do {                                                                                                \
    cudaError_t e_ = (call);                                                                          \
    if (e_ != cudaSuccess) {                                                                          \
      cudaGetLastError();                                                                             \
      return wfail(p, e_ == cudaErrorMemoryAllocation ? TP_ERR_OOM : TP_ERR_CUDA,                     \
                   std::string(what) + ": " + cudaGetErrorString(e_));                                \
    }                                                                                                 \
  } while (0)

tp_status check_grid(tp_problem* p) {
  if (p->dim != 3) return wfail(p, TP_ERR_ARG, "the learned warm start is for 3D problems");
  if (p->g.ex % 8 || p->g.ey % 8 || p->g.ez % 8)
    return wfail(p, TP_ERR_ARG, "the learned warm start needs nelx, nely, nelz to be multiples of 8");
  return TP_OK;
}

tp_status ensure_scratch(tp_problem* p) {
  const long long ne = p->ne;
  if (!p->nn_feat) WCK(cudaMalloc(&p->nn_feat, (size_t)p->nc * TPNN_FEATURES * ne * 2), "alloc features");
  if (!p->nn_out) WCK(cudaMalloc((void**)&p->nn_out, (size_t)p->nc * 3 * ne * 4), "alloc network output");
  if (!p->nn_scal) WCK(cudaMalloc((void**)&p->nn_scal, (size_t)3 * kCases * sizeof(double)), "alloc scalars");
  return TP_OK;
}

tp_status launch_features(tp_problem* p, void* dst) {
  Scale fs;
  for (int c = 0; c < kCases; c++) fs.v[c] = (c < p->nc && p->fmax[c] > 0.0) ? (float)(1.0 / (8.0 * p->fmax[c])) : 0.f;
  features_kernel<<<blocks_for(p->ne), 256, 0, p->stream>>>(p->g, p->nc, p->rho, p->mask, p->f, fs,
                                                           (__nv_bfloat16*)dst);
  p->launches++;
  WCK(cudaGetLastError(), "features kernel");
  return TP_OK;
}

}  // namespace

extern "C" {

tp_status tpnn_features(tp_problem* p, void* dst_bf16) {
  if (!p || !dst_bf16) return wfail(p, TP_ERR_ARG, "null argument");
  tp_status s = check_grid(p);
  if (s != TP_OK) return s;
  if (!p->has_fixed || !p->has_loads || !p->has_density)
    return wfail(p, TP_ERR_STATE, "fixed DOFs, loads and density must be set");
  return launch_features(p, dst_bf16);
}

tp_status tpnn_targets(tp_problem* p, void* dst_bf16) {
  if (!p || !dst_bf16) return wfail(p, TP_ERR_ARG, "null argument");
  tp_status s = check_grid(p);
  if (s != TP_OK) return s;
  if (!p->has_u) return wfail(p, TP_ERR_STATE, "no displacement yet");
  s = ensure_scratch(p);
  if (s != TP_OK) return s;
  const int nb = blocks_for(p->ne);
  // per-block maxima live in the (large enough) CG partial-sum buffer
  element_mean_kernel<<<nb, 256, 0, p->stream>>>(p->g, p->nc, p->x64, p->nn_out, (float*)p->part);
  target_scale_kernel<<<blocks_for((long long)p->nc * 3 * p->ne), 256, 0, p->stream>>>(
      p->ne, p->nc, nb, p->nn_out, (const float*)p->part, (__nv_bfloat16*)dst_bf16);
  p->launches += 2;
  WCK(cudaGetLastError(), "target kernels");
  return TP_OK;
}

tp_status tp_warm_start_nn(tp_problem* p, tpnn* net, double* alpha, double* ms) {
  if (!p || !net) return wfail(p, TP_ERR_ARG, "null argument");
  tp_status s = check_grid(p);
  if (s != TP_OK) return s;
  if (!p->has_fixed || !p->has_loads || !p->has_density)
    return wfail(p, TP_ERR_STATE, "fixed DOFs, loads and density must be set");
  int cin = 0, cout = 0;
  tpnn_info(net, &cin, &cout, nullptr);
  if (cin != TPNN_FEATURES || cout != 3)
    return wfail(p, TP_ERR_ARG, "the warm-start network needs 8 input and 3 output channels");
  s = ensure_scratch(p);
  if (s != TP_OK) return s;
  s = tp_problem_ensure_E(p);
  if (s != TP_OK) return s;
  WCK(cudaEventRecord(p->ev0, p->stream), "event");
  s = launch_features(p, p->nn_feat);
  if (s != TP_OK) return s;
  s = tpnn_forward(net, p->nn_feat, p->nc, p->g.ez, p->g.ey, p->g.ex, p->nn_out);
  if (s != TP_OK) return wfail(p, s, std::string("network forward: ") + tpnn_last_error(net));
  double* uhat = p->abi;
  double* kuhat = (double*)p->w[1];
  node_average_kernel<<<blocks_for(p->nn), 256, 0, p->stream>>>(p->g, p->nc, p->nn_out, p->mask, uhat);
  WCK(cudaGetLastError(), "node average kernel");
  WCK(tp::launch_matvec(p->stream, p->g, p->C.data(), true, p->E64, p->mask, uhat, kuhat, p->nc, p->zlen),
      "matvec");
  const int nb = blocks_for((long long)p->nc * p->ndof);
  warm_dots_kernel<<<nb, 256, 0, p->stream>>>(p->nn, p->nc, p->f, uhat, kuhat, p->part);
  warm_alpha_kernel<<<1, 32, 0, p->stream>>>(nb, p->nc, p->part, p->nn_scal);
  warm_apply_kernel<<<blocks_for((long long)p->nc * p->nn * 3), 256, 0, p->stream>>>(p->nn, p->nc, uhat, p->nn_scal,
                                                                                    p->x64);
  WCK(cudaGetLastError(), "warm-start kernels");
  p->launches += 5;
  WCK(cudaEventRecord(p->ev1, p->stream), "event");
  double h[kCases];
  WCK(cudaMemcpyAsync(h, p->nn_scal, sizeof(h), cudaMemcpyDeviceToHost, p->stream), "copy");
  WCK(cudaStreamSynchronize(p->stream), "sync");
  if (alpha)
    for (int c = 0; c < p->nc; c++) alpha[c] = h[c];
  if (ms) {
    float t = 0.f;
    cudaEventElapsedTime(&t, p->ev0, p->ev1);
    *ms = t;
  }
  p->has_u = true;
  p->has_dc = p->has_dcf = false;
  return TP_OK;
}

tp_status tpnn_energy_grad(tp_problem* p, const float* y, const double* comp, float* gy, double* loss) {
  if (!p || !y || !comp || !gy) return wfail(p, TP_ERR_ARG, "null argument");
  tp_status s = check_grid(p);
  if (s != TP_OK) return s;
  if (!p->has_fixed || !p->has_loads || !p->has_density)
    return wfail(p, TP_ERR_STATE, "fixed DOFs, loads and density must be set");
  Comp cm;
  for (int c = 0; c < kCases; c++) {
    cm.v[c] = c < p->nc ? comp[c] : 1.0;
    if (c < p->nc && !(comp[c] > 0.0)) return wfail(p, TP_ERR_ARG, "compliances must be positive");
  }
  s = ensure_scratch(p);
  if (s != TP_OK) return s;
  s = tp_problem_ensure_E(p);
  if (s != TP_OK) return s;
  double* uhat = p->abi;
  double* kuhat = (double*)p->w[1];
  double* gn = (double*)p->w[2];
  node_average_kernel<<<blocks_for(p->nn), 256, 0, p->stream>>>(p->g, p->nc, y, p->mask, uhat);
  WCK(cudaGetLastError(), "node average kernel");
  WCK(tp::launch_matvec(p->stream, p->g, p->C.data(), true, p->E64, p->mask, uhat, kuhat, p->nc, p->zlen),
      "matvec");
  const int nb = blocks_for((long long)p->nc * p->ndof);
  warm_dots_kernel<<<nb, 256, 0, p->stream>>>(p->nn, p->nc, p->f, uhat, kuhat, p->part);
  warm_alpha_kernel<<<1, 32, 0, p->stream>>>(nb, p->nc, p->part, p->nn_scal);
  energy_grad_node_kernel<<<blocks_for((long long)p->nc * p->ndof), 256, 0, p->stream>>>(
      p->nn, p->nc, p->mask, p->f, kuhat, p->nn_scal, cm, gn);
  node_average_adjoint_kernel<<<blocks_for(p->ne), 256, 0, p->stream>>>(p->g, p->nc, gn, gy);
  WCK(cudaGetLastError(), "energy gradient kernels");
  p->launches += 6;
  if (loss) {
    double h[3 * kCases];
    WCK(cudaMemcpyAsync(h, p->nn_scal, sizeof(h), cudaMemcpyDeviceToHost, p->stream), "copy");
    WCK(cudaStreamSynchronize(p->stream), "sync");
    for (int c = 0; c < p->nc; c++) loss[c] = 1.0 - h[c] * h[kCases + c] / comp[c];
  }
  return TP_OK;
}

}  // extern "C"
