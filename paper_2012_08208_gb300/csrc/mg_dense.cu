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
//
// Look-ahead: the row panel of block k + 1 after step k is formed directly
// from the matrix before step k and the panels of step k (next_panel_kernel),
// and the trailing update of step k skips the rows and columns of block k + 1
// (the panel writes of step k + 1 replace them).  So that panel and the pivot
// inversion of block k + 1, a one-CTA kernel, run on a second stream while
// the trailing update of step k runs on the first.  The whole sequence (some
// 380 launches at n = 3952, with the fork and join of the second stream) is
// captured once into a CUDA graph and replayed at every build.
#include <algorithm>

#include "../../include/topo.h"
#include "mg.h"
#include "mg_ops.cuh"

namespace tp {
namespace {

constexpr int kB = 64;    // pivot block
constexpr int kT = 128;   // trailing-update tile (kT x kT outputs per CTA)

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
          for (int s2 = 0; s2 < DIM; s2++) Ar[n2 * DIM + s2] = mgops::sblock<DIM>(S, nn, nd, nbr, n2, r, s2);
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
// sub-block's rank-16 sweep to the 64 x 64 block, each thread owning a 4 x 4
// tile (rows 4 ty .., columns 4 tx ..) so that every inner step is two
// 128-bit shared loads for 16 FMAs.  A pivot that is not positive and finite
// sets *flag.
constexpr int kS = 16;       // sub-block of the pivot-block sweep
constexpr int kLd = kB + 4;  // row stride of the shared block (16-byte rows, rotated banks)
__global__ void __launch_bounds__(256) block_inverse_kernel(const float* __restrict__ R, int n, int k0, int bk,
                                                            float* __restrict__ P, int* flag) {
  __shared__ __align__(16) float M[kB * kLd];
  __shared__ __align__(16) float sQ[kS * (kS + 4)];  // inverse of the diagonal sub-block, stride kS + 4
  __shared__ __align__(16) float sVt[kS * kLd];      // (M_:s Q)^T: sVt[c][i]
  __shared__ __align__(16) float sW[kS * kLd];       // Q M_s:   : sW[c][j]
  constexpr int kQd = kS + 4;
  for (int t = threadIdx.x; t < kB * kB; t += blockDim.x) {
    const int c = t / kB, d = t - c * kB;
    M[c * kLd + d] = (c < bk && d < bk) ? R[(size_t)c * n + k0 + d] : (c == d ? 1.f : 0.f);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int sb = 0; sb < kB / kS; sb++) {
    const int s0 = sb * kS;
    if (warp == 0) {
      // lane: row lr = lane & 15, columns 8 * (lane >> 4) .. + 8 of the sub-block
      const int lr = lane & 15, half = lane >> 4;
      float m[8];
#pragma unroll
      for (int q = 0; q < 8; q++) m[q] = M[(s0 + lr) * kLd + s0 + 8 * half + q];
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
      for (int q = 0; q < 8; q++) sQ[lr * kQd + 8 * half + q] = -m[q];  // the sweep leaves -B^-1
      if (lane == 0 && bad) atomicOr(flag, 1);
    }
    __syncthreads();
    // V = M_:s Q (kB x kS, stored transposed) and W = Q M_s: (kS x kB) from the
    // old block; four outputs per thread each.
    {
      const int i = threadIdx.x >> 2, c4 = 4 * (threadIdx.x & 3);
      float v[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int q = 0; q < kS; q++) {
        const float a = M[i * kLd + s0 + q];
        const float4 b = *reinterpret_cast<const float4*>(&sQ[q * kQd + c4]);
        v[0] = fmaf(a, b.x, v[0]);
        v[1] = fmaf(a, b.y, v[1]);
        v[2] = fmaf(a, b.z, v[2]);
        v[3] = fmaf(a, b.w, v[3]);
      }
#pragma unroll
      for (int e = 0; e < 4; e++) sVt[(c4 + e) * kLd + i] = v[e];
      const int c2 = threadIdx.x >> 4, j4 = 4 * (threadIdx.x & 15);
      float w[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int q = 0; q < kS; q++) {
        const float a = sQ[c2 * kQd + q];
        const float4 b = *reinterpret_cast<const float4*>(&M[(s0 + q) * kLd + j4]);
        w[0] = fmaf(a, b.x, w[0]);
        w[1] = fmaf(a, b.y, w[1]);
        w[2] = fmaf(a, b.z, w[2]);
        w[3] = fmaf(a, b.w, w[3]);
      }
      *reinterpret_cast<float4*>(&sW[c2 * kLd + j4]) = make_float4(w[0], w[1], w[2], w[3]);
    }
    __syncthreads();
    // M_ij -= M_is Q M_sj = V_i M_sj (i, j outside s) and the panels: all new
    // values from the old block first, then the writes.
    const int i0 = 4 * ty, j0 = 4 * tx;
    const bool is = i0 >= s0 && i0 < s0 + kS, js = j0 >= s0 && j0 < s0 + kS;
    float nv[4][4];
    if (is && js) {
#pragma unroll
      for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 4; b++) nv[a][b] = -sQ[(i0 - s0 + a) * kQd + j0 - s0 + b];
    } else if (is) {
#pragma unroll
      for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 4; b++) nv[a][b] = sW[(i0 - s0 + a) * kLd + j0 + b];
    } else if (js) {
#pragma unroll
      for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 4; b++) nv[a][b] = sVt[(j0 - s0 + b) * kLd + i0 + a];
    } else {
#pragma unroll
      for (int a = 0; a < 4; a++) {
        const float4 r = *reinterpret_cast<const float4*>(&M[(i0 + a) * kLd + j0]);
        nv[a][0] = r.x;
        nv[a][1] = r.y;
        nv[a][2] = r.z;
        nv[a][3] = r.w;
      }
#pragma unroll
      for (int q = 0; q < kS; q++) {
        const float4 vv = *reinterpret_cast<const float4*>(&sVt[q * kLd + i0]);
        const float4 mm = *reinterpret_cast<const float4*>(&M[(s0 + q) * kLd + j0]);
        const float va[4] = {vv.x, vv.y, vv.z, vv.w};
        const float mb[4] = {mm.x, mm.y, mm.z, mm.w};
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
          for (int b = 0; b < 4; b++) nv[a][b] = fmaf(-va[a], mb[b], nv[a][b]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 4; a++)
      *reinterpret_cast<float4*>(&M[(i0 + a) * kLd + j0]) = make_float4(nv[a][0], nv[a][1], nv[a][2], nv[a][3]);
    __syncthreads();
  }
  for (int t = threadIdx.x; t < kB * kB; t += blockDim.x) P[t] = -M[(t / kB) * kLd + t % kB];  // -A_kk^-1 -> A_kk^-1
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

// Asynchronous global -> shared copies (cp.async); a zero source size fills
// the destination with zeros and reads nothing.
__device__ __forceinline__ void cp_async16(float* dst, const float* src, bool ok) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(ok ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool ok) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(ok ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

constexpr size_t kTrailingSmem = (size_t)2 * kB * kT * sizeof(float);

// A_ij -= sum_q R[q][i] W[q][j] on the upper-triangular tiles (J >= I): a
// kT x kT tile per CTA (blockIdx.x enumerates the upper tiles row by row).
// Both kB x kT panels are copied to shared memory asynchronously while the
// CTA loads its tile of A into the accumulators; then kB rank-1 steps, each
// thread owning rows 4 ty .. 4 ty + 3 and 64 + 4 ty .. of the tile and the
// same pattern of columns (4 tx ..), so its operands are four 128-bit shared
// loads and its tile rows are read and written as 128-bit words that a warp
// covers contiguously.  V4 (n a multiple of 4: every row starts on a 16-byte
// boundary) selects the 128-bit global accesses; otherwise scalar ones.
// Rows and columns in [x0, x1) (the next pivot block, whose rows the
// look-ahead panel reads concurrently and the next step's panel writes
// replace) are left unwritten; x0 and x1 are multiples of 4 when V4.
template <bool V4>
__global__ void __launch_bounds__(256, 2) trailing_kernel(float* __restrict__ A, int n, int nt,
                                                          const float* __restrict__ R, const float* __restrict__ W,
                                                          int x0, int x1) {
  extern __shared__ __align__(16) float dsm[];
  float* sU = dsm;            // [kB][kT]: R[q][i0 + c]
  float* sW = dsm + kB * kT;  // [kB][kT]: W[q][j0 + c]
  int I = 0, rem = blockIdx.x;  // tile row I holds nt - I tiles
  while (rem >= nt - I) {
    rem -= nt - I;
    I++;
  }
  const int J = I + rem;
  const int i0 = I * kT, j0 = J * kT;
  if (V4) {
    for (int t = threadIdx.x; t < kB * kT / 4; t += blockDim.x) {
      const int q = t / (kT / 4), c = 4 * (t - q * (kT / 4));
      const int i = i0 + c, j = j0 + c;
      cp_async16(sU + q * kT + c, i < n ? R + (size_t)q * n + i : R, i < n);
      cp_async16(sW + q * kT + c, j < n ? W + (size_t)q * n + j : W, j < n);
    }
  } else {
#pragma unroll 1
    for (int t = threadIdx.x; t < kB * kT; t += blockDim.x) {
      const int q = t / kT, c = t - q * kT;
      const int i = i0 + c, j = j0 + c;
      cp_async4(sU + q * kT + c, i < n ? R + (size_t)q * n + i : R, i < n);
      cp_async4(sW + q * kT + c, j < n ? W + (size_t)q * n + j : W, j < n);
    }
  }
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; a++) {
    const int i = i0 + 4 * ty + (a & 3) + (kT / 2) * (a >> 2);
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const int j = j0 + 4 * tx + (kT / 2) * h;
      if (V4) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < n && j < n) v = *reinterpret_cast<const float4*>(A + (size_t)i * n + j);
        acc[a][4 * h] = v.x;
        acc[a][4 * h + 1] = v.y;
        acc[a][4 * h + 2] = v.z;
        acc[a][4 * h + 3] = v.w;
      } else {
#pragma unroll
        for (int e = 0; e < 4; e++) acc[a][4 * h + e] = (i < n && j + e < n) ? A[(size_t)i * n + j + e] : 0.f;
      }
    }
  }
  cp_async_wait_all();
  __syncthreads();
#pragma unroll 2
  for (int q = 0; q < kB; q++) {
    const float4 u0 = *reinterpret_cast<const float4*>(sU + q * kT + 4 * ty);
    const float4 u1 = *reinterpret_cast<const float4*>(sU + q * kT + kT / 2 + 4 * ty);
    const float4 w0 = *reinterpret_cast<const float4*>(sW + q * kT + 4 * tx);
    const float4 w1 = *reinterpret_cast<const float4*>(sW + q * kT + kT / 2 + 4 * tx);
    const float u[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
    const float w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
    for (int a = 0; a < 8; a++)
#pragma unroll
      for (int b = 0; b < 8; b++) acc[a][b] = fmaf(-u[a], w[b], acc[a][b]);
  }
#pragma unroll
  for (int a = 0; a < 8; a++) {
    const int i = i0 + 4 * ty + (a & 3) + (kT / 2) * (a >> 2);
    if (i >= n || (i >= x0 && i < x1)) continue;
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const int j = j0 + 4 * tx + (kT / 2) * h;
      if (V4) {
        if (j < n && !(j >= x0 && j < x1))
          *reinterpret_cast<float4*>(A + (size_t)i * n + j) =
              make_float4(acc[a][4 * h], acc[a][4 * h + 1], acc[a][4 * h + 2], acc[a][4 * h + 3]);
      } else {
#pragma unroll
        for (int e = 0; e < 4; e++)
          if (j + e < n && !(j + e >= x0 && j + e < x1)) A[(size_t)i * n + j + e] = acc[a][4 * h + e];
      }
    }
  }
}

// Row panel of the next pivot block: R1[c][j] = row k1 + c (k1 = k0 + bk,
// c < bk1; zero rows below) of the matrix after step k (trailing update, then
// panel writes), formed from the matrix before step k.  Columns of block k are
// the written panel, W[j - k0][k1 + c]; every other entry is its stored
// (upper-triangle) value minus the rank-kB update, in the order and operand
// pairing of trailing_kernel.  It reads only entries in the rows and columns
// of block k + 1, which the trailing update of step k leaves unwritten, so
// the two run concurrently.  kNP columns per CTA; the panels' columns it
// needs staged in shared memory.
constexpr int kNP = 16;
__global__ void __launch_bounds__(256) next_panel_kernel(const float* __restrict__ A, int n, int k0, int bk, int bk1,
                                                         const float* __restrict__ R, const float* __restrict__ W,
                                                         float* __restrict__ R1) {
  __shared__ float sRr[kB][kB], sWr[kB][kB];     // R[q][k1 + c], W[q][k1 + c]
  __shared__ float sRj[kB][kNP], sWj[kB][kNP];   // R[q][j0 + jj], W[q][j0 + jj]
  const int k1 = k0 + bk, j0 = blockIdx.x * kNP;
  for (int t = threadIdx.x; t < kB * kB; t += blockDim.x) {
    const int q = t / kB, c = t - q * kB;
    const bool ok = c < bk1;
    sRr[q][c] = ok ? R[(size_t)q * n + k1 + c] : 0.f;
    sWr[q][c] = ok ? W[(size_t)q * n + k1 + c] : 0.f;
  }
  for (int t = threadIdx.x; t < kB * kNP; t += blockDim.x) {
    const int q = t / kNP, jj = t - q * kNP, j = j0 + jj;
    sRj[q][jj] = j < n ? R[(size_t)q * n + j] : 0.f;
    sWj[q][jj] = j < n ? W[(size_t)q * n + j] : 0.f;
  }
  __syncthreads();
  const int jj = threadIdx.x % kNP, cg = threadIdx.x / kNP;
  const int j = j0 + jj;
  if (j >= n) return;
  for (int c = cg; c < kB; c += 256 / kNP) {
    float v = 0.f;
    if (c < bk1) {
      const int r = k1 + c;
      if (j >= k0 && j < k1) {
        v = W[(size_t)(j - k0) * n + r];
      } else if (j >= r) {  // stored at (r, j)
        v = A[(size_t)r * n + j];
#pragma unroll 8
        for (int q = 0; q < kB; q++) v = fmaf(-sRr[q][c], sWj[q][jj], v);
      } else {  // stored at (j, r)
        v = A[(size_t)j * n + r];
#pragma unroll 8
        for (int q = 0; q < kB; q++) v = fmaf(-sRj[q][jj], sWr[q][c], v);
      }
    }
    R1[(size_t)c * n + j] = v;
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

size_t dense_scratch_floats(int n) { return (size_t)3 * n * kB + 2 * kB * kB; }

cudaError_t DenseInverter::create() {
  if (side) return cudaSuccess;
  cudaError_t e = cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
  if (e != cudaSuccess) destroy();
  return e;
}

void DenseInverter::destroy() {
  if (exec) cudaGraphExecDestroy(exec);
  if (ready) cudaEventDestroy(ready);
  if (done) cudaEventDestroy(done);
  if (side) cudaStreamDestroy(side);
  if (cap) cudaStreamDestroy(cap);
  exec = nullptr;
  side = cap = nullptr;
  ready = done = nullptr;
  key_n = launches = 0;
}

namespace {

// The launches of the inversion on stream s (captured into the graph).
cudaError_t issue_spd_inverse(cudaStream_t s, const DenseInverter& ds, float* A, int n, float* scratch, int* flag,
                              int* nlaunch) {
  float* Rb[2] = {scratch, scratch + (size_t)n * kB};
  float* W = scratch + (size_t)2 * n * kB;
  float* Pb[2] = {W + (size_t)n * kB, W + (size_t)n * kB + kB * kB};
  const bool v4 = (n & 3) == 0;
  cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  int nl = 0;
  const int nt = (n + kT - 1) / kT, ntiles = nt * (nt + 1) / 2;
  copy_panel_kernel<<<grid_for((long long)n * kB), 256, 0, s>>>(A, n, 0, std::min(kB, n), Rb[0]);
  block_inverse_kernel<<<1, 256, 0, s>>>(Rb[0], n, 0, std::min(kB, n), Pb[0], flag);
  nl += 2;
  for (int k0 = 0, it = 0; k0 < n; k0 += kB, it++) {
    const int cur = it & 1, bk = std::min(kB, n - k0), k1 = k0 + bk;
    const int bk1 = k1 < n ? std::min(kB, n - k1) : 0;
    panel_kernel<<<grid_for((long long)n * kB), 256, 0, s>>>(Rb[cur], Pb[cur], n, W);
    nl++;
    if (bk1 > 0) {
      cudaStream_t sb = s;
      if (ds.side) {
        e = cudaEventRecord(ds.ready, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ds.side, ds.ready, 0);
        if (e != cudaSuccess) return e;
        sb = ds.side;
      }
      next_panel_kernel<<<(n + kNP - 1) / kNP, 256, 0, sb>>>(A, n, k0, bk, bk1, Rb[cur], W, Rb[cur ^ 1]);
      block_inverse_kernel<<<1, 256, 0, sb>>>(Rb[cur ^ 1], n, k1, bk1, Pb[cur ^ 1], flag);
      nl += 2;
      if (ds.side) e = cudaEventRecord(ds.done, ds.side);
      if (e != cudaSuccess) return e;
    }
    if (v4) trailing_kernel<true><<<ntiles, 256, kTrailingSmem, s>>>(A, n, nt, Rb[cur], W, k1, k1 + bk1);
    else trailing_kernel<false><<<ntiles, 256, kTrailingSmem, s>>>(A, n, nt, Rb[cur], W, k1, k1 + bk1);
    write_panels_kernel<<<grid_for((long long)n * bk), 256, 0, s>>>(A, n, k0, bk, W, Pb[cur]);
    nl += 2;
    if (bk1 > 0 && ds.side) e = cudaStreamWaitEvent(s, ds.done, 0);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  negate_mirror_kernel<<<grid_for((long long)n * n), 256, 0, s>>>(A, n);
  nl++;
  if (nlaunch) *nlaunch += nl;
  return cudaGetLastError();
}


// Replays ds's graph on s, capturing `issue` (launches on the stream it is
// given) first when the key differs from the captured one.
template <class F>
cudaError_t replay(cudaStream_t s, DenseInverter& ds, const void* const (&key)[5], int n, int* nlaunch, F issue) {
  bool same = ds.exec && ds.key_n == n;
  for (int i = 0; i < 5 && same; i++) same = ds.key[i] == key[i];
  if (!same) {
    if (ds.exec) cudaGraphExecDestroy(ds.exec);
    ds.exec = nullptr;
    cudaError_t e = cudaFuncSetAttribute((n & 3) == 0 ? (const void*)trailing_kernel<true>
                                                      : (const void*)trailing_kernel<false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrailingSmem);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(ds.cap, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return e;
    int nl = 0;
    e = issue(ds.cap, &nl);
    cudaGraph_t gr = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(ds.cap, &gr);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ds.exec, gr, 0);
    if (gr) cudaGraphDestroy(gr);
    if (e != cudaSuccess) {
      ds.exec = nullptr;
      return e;
    }
    for (int i = 0; i < 5; i++) ds.key[i] = key[i];
    ds.key_n = n;
    ds.launches = nl;
  }
  const cudaError_t e = cudaGraphLaunch(ds.exec, s);
  if (e == cudaSuccess && nlaunch) *nlaunch += ds.launches;
  return e;
}

}  // namespace

cudaError_t dense_spd_inverse(cudaStream_t s, DenseInverter& ds, float* A, int n, float* scratch, int* flag,
                              int* nlaunch) {
  const void* const key[5] = {A, nullptr, nullptr, scratch, flag};
  return replay(s, ds, key, n, nlaunch,
                [&](cudaStream_t cs, int* nl) { return issue_spd_inverse(cs, ds, A, n, scratch, flag, nl); });
}

cudaError_t dense_coarse_inverse(cudaStream_t s, DenseInverter& ds, const Grid& g, const float* S,
                                 const uint8_t* mask, float* A, float* scratch, int* flag, int* nlaunch) {
  const int n = (int)(g.nn * g.dim);
  const void* const key[5] = {A, S, mask, scratch, flag};
  return replay(s, ds, key, n, nlaunch, [&](cudaStream_t cs, int* nl) {
    cudaError_t e = cudaMemsetAsync(A, 0, (size_t)n * n * sizeof(float), cs);
    if (e != cudaSuccess) return e;
    if (g.dim == 2) dense_assemble_kernel<2><<<grid_for(n), 256, 0, cs>>>(g, S, mask, A);
    else dense_assemble_kernel<3><<<grid_for(n), 256, 0, cs>>>(g, S, mask, A);
    (*nl)++;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return issue_spd_inverse(cs, ds, A, n, scratch, flag, nl);
  });
}

}  // namespace tp

extern "C" tp_status tp_spd_inverse_f32(const float* a, float* ainv, int n, void* cuda_stream) {
  if (!a || !ainv || n < 1 || n > TP_SPD_INVERSE_MAX_N) return TP_ERR_ARG;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const size_t bytes = (size_t)n * n * sizeof(float);
  float *dA = nullptr, *scr = nullptr;
  int* flag = nullptr;
  tp::DenseInverter ds;
  cudaError_t e = cudaMalloc((void**)&dA, bytes);
  if (e == cudaSuccess) e = cudaMalloc((void**)&scr, tp::dense_scratch_floats(n) * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&flag, sizeof(int));
  const bool oom = e == cudaErrorMemoryAllocation;
  if (e == cudaSuccess) e = ds.create();
  if (e == cudaSuccess) e = cudaMemcpyAsync(dA, a, bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = tp::dense_spd_inverse(s, ds, dA, n, scr, flag, nullptr);
  int hflag = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(ainv, dA, bytes, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  ds.destroy();
  for (void* q : {(void*)dA, (void*)scr, (void*)flag})
    if (q) cudaFree(q);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return oom ? TP_ERR_OOM : TP_ERR_CUDA;
  }
  return hflag ? TP_ERR_BREAKDOWN : TP_OK;
}
