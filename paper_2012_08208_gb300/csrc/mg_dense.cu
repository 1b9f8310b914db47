// Dense FP32 inverse of the coarsest multigrid operator, formed on the GPU at
// every hierarchy build (the moduli change every SIMP step).
//
// The coarsest level is assembled from its per-node coupling blocks into a
// dense n x n matrix (rows and columns of fixed DOFs zero, 1 on their
// diagonal) and inverted in place by a blocked symmetric sweep (Gauss-Jordan
// without pivoting; the matrix is SPD, so every pivot is positive):
//   for each pivot block k (kB rows):  R = A_k: (old row panel),  P = A_kk^-1,
//     W = P R,  A_ij -= R_i^T W_j  for every i, j,  A_k: = W,  A_:k = W^T,  A_kk = -P,
// after which A holds -A^-1.  The sweep keeps A symmetric, so only the upper
// triangle is kept (tiles J >= I; entries below the diagonal are read from
// their mirror), and a last pass negates and mirrors it.  Every step but the
// small pivot inversion is a rank-kB update done by a tiled FP32 kernel.
// (The sweep operator of Beaton and Goodnight, in block form.)
#include <algorithm>

#include "mg.h"

namespace tp {
namespace {

constexpr int kB = 64;    // pivot block
constexpr int kT = 128;   // trailing-update tile (kT x kT outputs per CTA)
constexpr int kQ = 32;    // inner-dimension chunk staged in shared memory

template <int DIM>
__global__ void dense_assemble_kernel(Grid g, const float* __restrict__ S, const uint8_t* __restrict__ mask,
                                      float* __restrict__ A) {
  const int nn = (int)g.nn, n = nn * DIM, nxy = g.nx * g.ny;
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n; row += gridDim.x * blockDim.x) {
    const int nd = row / DIM, r = row - nd * DIM;
    float* Ar = A + (size_t)row * n;
    if ((mask[nd] >> r) & 1) {
      Ar[row] = 1.f;
      continue;
    }
    const int k = DIM == 3 ? nd / nxy : 0, rem = nd - k * nxy, j = rem / g.nx, i = rem - j * g.nx;
    for (int dz = (DIM == 3 ? -1 : 0); dz <= (DIM == 3 ? 1 : 0); dz++) {
      if (k + dz < 0 || k + dz >= g.nz) continue;
      for (int dy = -1; dy <= 1; dy++) {
        if (j + dy < 0 || j + dy >= g.ny) continue;
        for (int dx = -1; dx <= 1; dx++) {
          if (i + dx < 0 || i + dx >= g.nx) continue;
          const int nbr = (dx + 1) + 3 * (dy + 1) + (DIM == 3 ? 9 * (dz + 1) : 0);
          const int n2 = nd + dx + g.nx * dy + nxy * dz;
          for (int s2 = 0; s2 < DIM; s2++) Ar[n2 * DIM + s2] = S[((long long)(nbr * DIM + r) * DIM + s2) * nn + nd];
        }
      }
    }
  }
}

// R[c][j] = A[k0 + c][j] of the symmetric matrix held in its upper triangle
// (the entry at (min, max)); zero rows c >= bk.
__global__ void copy_panel_kernel(const float* __restrict__ A, int n, int k0, int bk, float* __restrict__ R) {
  const long long tot = (long long)n * kB;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(t / n), j = (int)(t - (long long)c * n);
    const int r = k0 + c;
    R[t] = c < bk ? (j >= r ? A[(size_t)r * n + j] : A[(size_t)j * n + r]) : 0.f;
  }
}

// P = A_kk^-1 (A_kk = R[:, k0 .. k0 + bk], padded with the identity); one CTA
// of 256 threads, the block in shared memory.  The block sweep runs over four
// 16 x 16 sub-blocks: warp 0 inverts the diagonal sub-block by an unblocked
// sweep held in registers (8 entries per lane, pivot row and column by warp
// shuffles, no CTA barrier per pivot), then the whole CTA applies that
// sub-block's rank-16 sweep to the 64 x 64 block.  A pivot that is not
// positive and finite sets *flag.
__global__ void __launch_bounds__(256) block_inverse_kernel(const float* __restrict__ R, int n, int k0, int bk,
                                                            float* __restrict__ P, int* flag) {
  constexpr int kS = 16;
  __shared__ float M[kB][kB + 1];
  __shared__ float sQ[kS][kS + 1];  // inverse of the diagonal sub-block
  __shared__ float sV[kB][kS + 1];  // M_:s Q
  __shared__ float sW[kS][kB + 1];  // Q M_s:
  for (int t = threadIdx.x; t < kB * kB; t += blockDim.x) {
    const int c = t / kB, d = t - c * kB;
    M[c][d] = (c < bk && d < bk) ? R[(size_t)c * n + k0 + d] : (c == d ? 1.f : 0.f);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int sb = 0; sb < kB / kS; sb++) {
    const int s0 = sb * kS;
    if (warp == 0) {
      // lane: row lr = lane & 15, columns 8 * (lane >> 4) .. + 8 of the sub-block
      const int lr = lane & 15, half = lane >> 4;
      float m[8];
#pragma unroll
      for (int q = 0; q < 8; q++) m[q] = M[s0 + lr][s0 + 8 * half + q];
      bool bad = false;
#pragma unroll 1
      for (int p = 0; p < kS; p++) {
        float sel = 0.f;  // this lane's entry in column p (meaningful for lanes of column half p >> 3)
#pragma unroll
        for (int q = 0; q < 8; q++)
          if (q == (p & 7)) sel = m[q];
        const float dp = __shfl_sync(0xffffffffu, sel, p + 16 * (p >> 3));    // M[p][p]
        const float colv = __shfl_sync(0xffffffffu, sel, lr + 16 * (p >> 3)); // M[lr][p]
        float rd[8];
#pragma unroll
        for (int q = 0; q < 8; q++) rd[q] = __shfl_sync(0xffffffffu, m[q], p + 16 * half);  // M[p][8 half + q]
        bad |= !(dp > 0.f && isfinite(dp));
        const float inv = 1.f / dp, cr = colv * inv;
#pragma unroll
        for (int q = 0; q < 8; q++) {
          const int d = 8 * half + q;
          float v;
          if (lr == p) v = d == p ? -inv : m[q] * inv;
          else if (d == p) v = cr;
          else v = fmaf(-cr, rd[q], m[q]);
          m[q] = v;
        }
      }
#pragma unroll
      for (int q = 0; q < 8; q++) sQ[lr][8 * half + q] = -m[q];  // the sweep leaves -B^-1
      if (lane == 0 && bad) atomicOr(flag, 1);
    }
    __syncthreads();
    // V = M_:s Q (kB x kS), W = Q M_s: (kS x kB) from the old block
    for (int t = threadIdx.x; t < kB * kS; t += blockDim.x) {
      const int i = t / kS, c = t - i * kS;
      float v = 0.f;
#pragma unroll
      for (int q = 0; q < kS; q++) v = fmaf(M[i][s0 + q], sQ[q][c], v);
      sV[i][c] = v;
      const int c2 = t / kB, j = t - c2 * kB;
      float w = 0.f;
#pragma unroll
      for (int q = 0; q < kS; q++) w = fmaf(sQ[c2][q], M[s0 + q][j], w);
      sW[c2][j] = w;
    }
    __syncthreads();
    // M_ij -= M_is Q M_sj = sV_i M_sj (i, j outside s) and the panels: all new
    // values from the old block first (16 per thread), then the writes
    float nv[kB * kB / 256];
#pragma unroll
    for (int k = 0; k < kB * kB / 256; k++) {
      const int t = threadIdx.x + 256 * k, i = t / kB, j = t - i * kB;
      const bool is = i >= s0 && i < s0 + kS, js = j >= s0 && j < s0 + kS;
      float v;
      if (is && js) v = -sQ[i - s0][j - s0];
      else if (is) v = sW[i - s0][j];
      else if (js) v = sV[i][j - s0];
      else {
        v = M[i][j];
#pragma unroll
        for (int q = 0; q < kS; q++) v = fmaf(-sV[i][q], M[s0 + q][j], v);
      }
      nv[k] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kB * kB / 256; k++) {
      const int t = threadIdx.x + 256 * k;
      M[t / kB][t % kB] = nv[k];
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < kB * kB; t += blockDim.x) P[t] = -M[t / kB][t % kB];  // -A_kk^-1 -> A_kk^-1
}

// W = P R (kB x n); one output per thread.
__global__ void panel_kernel(const float* __restrict__ R, const float* __restrict__ P, int n, float* __restrict__ W) {
  __shared__ float sP[kB][kB + 1];
  for (int t = threadIdx.x; t < kB * kB; t += blockDim.x) sP[t / kB][t % kB] = P[t];
  __syncthreads();
  const long long tot = (long long)n * kB;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(t / n), j = (int)(t - (long long)c * n);
    float s = 0.f;
    for (int q = 0; q < kB; q++) s = fmaf(sP[c][q], R[(size_t)q * n + j], s);
    W[t] = s;
  }
}

// A_ij -= sum_q R[q][i] W[q][j] on the upper-triangular tiles (J >= I): a
// kT x kT tile per CTA (blockIdx.x enumerates the upper tiles row by row), a
// contiguous 8 x 8 block of outputs per thread (rows 8 ty .., columns 8 tx ..),
// so each inner step reads its 16 operands with four 128-bit shared loads; the
// inner dimension in chunks of kQ staged in shared memory.
__global__ void __launch_bounds__(256) trailing_kernel(float* __restrict__ A, int n, int nt, const float* __restrict__ R,
                                                       const float* __restrict__ W) {
  __shared__ __align__(16) float sU[kQ][kT];
  __shared__ __align__(16) float sW[kQ][kT];
  int I = 0, rem = blockIdx.x;  // tile row I holds nt - I tiles
  while (rem >= nt - I) {
    rem -= nt - I;
    I++;
  }
  const int J = I + rem;
  const int i0 = I * kT, j0 = J * kT;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; a++)
#pragma unroll
    for (int b = 0; b < 8; b++) acc[a][b] = 0.f;
  for (int q0 = 0; q0 < kB; q0 += kQ) {
    for (int t = threadIdx.x; t < kT * kQ; t += blockDim.x) {
      const int q = t / kT, c = t - q * kT;  // both panels row-major in q: consecutive columns
      const int i = i0 + c, j = j0 + c;
      sU[q][c] = i < n ? R[(size_t)(q0 + q) * n + i] : 0.f;
      sW[q][c] = j < n ? W[(size_t)(q0 + q) * n + j] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int q = 0; q < kQ; q++) {
      const float4 u0 = *reinterpret_cast<const float4*>(&sU[q][8 * ty]);
      const float4 u1 = *reinterpret_cast<const float4*>(&sU[q][8 * ty + 4]);
      const float4 w0 = *reinterpret_cast<const float4*>(&sW[q][8 * tx]);
      const float4 w1 = *reinterpret_cast<const float4*>(&sW[q][8 * tx + 4]);
      const float u[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
      const float w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
      for (int a = 0; a < 8; a++)
#pragma unroll
        for (int b = 0; b < 8; b++) acc[a][b] = fmaf(u[a], w[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 8; a++) {
    const int i = i0 + 8 * ty + a;
    if (i >= n) continue;
#pragma unroll
    for (int b = 0; b < 8; b++) {
      const int j = j0 + 8 * tx + b;
      if (j < n) A[(size_t)i * n + j] -= acc[a][b];
    }
  }
}

// Upper triangle of rows / columns k0 .. k0 + bk: A_kj = W_j (j >= k0, with
// -P on the diagonal block), A_ik = W_i^T (i < k0).
__global__ void write_panels_kernel(float* __restrict__ A, int n, int k0, int bk, const float* __restrict__ W,
                                    const float* __restrict__ P) {
  const long long tot = (long long)n * bk;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(t / n), j = (int)(t - (long long)c * n);
    if (j >= k0) A[(size_t)(k0 + c) * n + j] = j < k0 + bk ? -P[c * kB + (j - k0)] : W[(size_t)c * n + j];
    else A[(size_t)j * n + k0 + c] = W[(size_t)c * n + j];
  }
}

// A = -A, mirrored from the upper triangle: one thread per pair (i <= j).
__global__ void negate_mirror_kernel(float* A, int n) {
  const long long tot = (long long)n * n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < tot; t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t / n), j = (int)(t - (long long)i * n);
    if (j < i) continue;
    const float v = -A[t];
    A[t] = v;
    A[(size_t)j * n + i] = v;
  }
}

int grid_for(long long n) { return (int)std::min<long long>(std::max<long long>((n + 255) / 256, 1), 152 * 8); }

}  // namespace

size_t dense_scratch_floats(int n) { return (size_t)2 * n * kB + kB * kB; }

cudaError_t dense_coarse_inverse(cudaStream_t s, const Grid& g, const float* S, const uint8_t* mask, float* A,
                                 float* scratch, int* flag, int* nlaunch) {
  const int n = (int)(g.nn * g.dim);
  float* R = scratch;
  float* W = R + (size_t)n * kB;
  float* P = W + (size_t)n * kB;
  cudaError_t e = cudaMemsetAsync(A, 0, (size_t)n * n * sizeof(float), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  if (g.dim == 2) dense_assemble_kernel<2><<<grid_for(n), 256, 0, s>>>(g, S, mask, A);
  else dense_assemble_kernel<3><<<grid_for(n), 256, 0, s>>>(g, S, mask, A);
  int nl = 1;
  const int nt = (n + kT - 1) / kT, ntiles = nt * (nt + 1) / 2;
  for (int k0 = 0; k0 < n; k0 += kB) {
    const int bk = std::min(kB, n - k0);
    copy_panel_kernel<<<grid_for((long long)n * kB), 256, 0, s>>>(A, n, k0, bk, R);
    block_inverse_kernel<<<1, 256, 0, s>>>(R, n, k0, bk, P, flag);
    panel_kernel<<<grid_for((long long)n * kB), 256, 0, s>>>(R, P, n, W);
    trailing_kernel<<<ntiles, 256, 0, s>>>(A, n, nt, R, W);
    write_panels_kernel<<<grid_for((long long)n * bk), 256, 0, s>>>(A, n, k0, bk, W, P);
    nl += 5;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  negate_mirror_kernel<<<grid_for((long long)n * n), 256, 0, s>>>(A, n);
  nl++;
  if (nlaunch) *nlaunch += nl;
  return cudaGetLastError();
}

}  // namespace tp
