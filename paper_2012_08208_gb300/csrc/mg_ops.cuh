// Per-item device bodies of the multigrid V-cycle below the finest level:
// Chebyshev step / residual on an assembled level, restriction, prolongation,
// and the dense coarsest solve.  The standalone kernels (mg.cu) and the
// persistent multigrid PCG kernel (mg_pcg.cu) call the same bodies, so both
// compute identical values.
//
// Vectors are [case][node * DIM + comp] (the ABI layout); `off` is the case's
// offset case * n_dof of the level.  With CG = true, vector loads go through
// L2 only (__ldcg): in the persistent kernel they were written by other CTAs of
// the same launch, and L1 is not coherent across CTAs.  The standalone kernels
// (CG = false) read data written by earlier launches and keep L1 reuse between
// neighbouring nodes.  Operator data (stencils, scales, masks, the dense
// inverse) is read-only and may be cached anywhere.
#pragma once
#include "common.cuh"
#include "strain.cuh"

namespace tp {
namespace mgops {

__device__ __forceinline__ long long node_index(const Grid& g, int i, int j, int k) {
  return i + (long long)g.nx * (j + (long long)g.ny * k);
}

template <bool CG>
__device__ __forceinline__ float ldv(const float* p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}

// Assembled levels store their coupling blocks once per symmetric pair: node
// nd's DIM x DIM block to neighbour nbr = (dx+1) + 3 (dy+1) [+ 9 (dz+1)] is
// kept for the forward half nbr >= kSelf (the node itself and the 4 / 13
// neighbours after it) in slot h = nbr - kSelf,
//   S[((h * DIM + r) * DIM + s) * n_nodes + nd],
// and a backward block (nbr < kSelf) is the transpose of the forward block that
// the neighbour n2 holds for the opposite direction, slot kSelf - nbr.  The
// operator is symmetric by construction, and a sweep reads half the bytes.
template <int DIM>
struct Sym {
  static constexpr int kSelf = DIM == 2 ? 4 : 13;      // slot 0: the node itself
  static constexpr int kSlots = kSelf + 1;             // stored blocks per node
};
template <int DIM>
__device__ __forceinline__ float sblock(const float* __restrict__ S, int nn, int nd, int nbr, int n2, int r, int s) {
  constexpr int C = Sym<DIM>::kSelf;
  return nbr >= C ? S[((long long)((nbr - C) * DIM + r) * DIM + s) * nn + nd]
                  : S[((long long)((C - nbr) * DIM + s) * DIM + r) * nn + n2];
}

// 1D multilinear weight of coarse corner offset `o` (0 or 1) at fine position t in [0, f].
__device__ __forceinline__ float w1(int o, int t, int f) { return o ? (float)t / f : 1.f - (float)t / f; }

// Node nd of a level with assembled blocks S (symmetric storage, sblock):
//   mode 1: y = ca u + cc w + om D^-1 (b - A u)   (Chebyshev step; w may be null)
//   mode 2: y = b - A u                            (residual)
// A u with fixed entries of u read as 0 (their rows and columns of S are
// zero); y = 0 on fixed DOFs.  w is read at the node's own DOFs only, so y may
// alias w.
template <int DIM, bool CG>
__device__ __forceinline__ void stencil_node(const Grid& g, const float* __restrict__ S,
                                             const uint8_t* __restrict__ mask, const float* __restrict__ invd,
                                             const float* u, const float* w, const float* b, float* y, int mode,
                                             float ca, float cc, float om, int nd, long long off) {
  const int nn = (int)g.nn, nxy = g.nx * g.ny;
  const int k = DIM == 3 ? nd / nxy : 0, rem = nd - k * nxy, j = rem / g.nx, i = rem - j * g.nx;
  float acc[DIM];
#pragma unroll
  for (int r = 0; r < DIM; r++) acc[r] = 0.f;
#pragma unroll
  for (int dz = (DIM == 3 ? -1 : 0); dz <= (DIM == 3 ? 1 : 0); dz++) {
    if (k + dz < 0 || k + dz >= g.nz) continue;
#pragma unroll
    for (int dy = -1; dy <= 1; dy++) {
      if (j + dy < 0 || j + dy >= g.ny) continue;
#pragma unroll
      for (int dx = -1; dx <= 1; dx++) {
        if (i + dx < 0 || i + dx >= g.nx) continue;
        const int nbr = (dx + 1) + 3 * (dy + 1) + (DIM == 3 ? 9 * (dz + 1) : 0);
        const int n2 = nd + dx + g.nx * dy + nxy * dz;
#pragma unroll
        for (int s2 = 0; s2 < DIM; s2++) {
          const float v = ldv<CG>(u + off + (long long)n2 * DIM + s2);
#pragma unroll
          for (int r = 0; r < DIM; r++) acc[r] = fmaf(sblock<DIM>(S, nn, nd, nbr, n2, r, s2), v, acc[r]);
        }
      }
    }
  }
  const uint8_t mk = mask[nd];
#pragma unroll
  for (int r = 0; r < DIM; r++) {
    const long long idx = (long long)nd * DIM + r;
    const float res = ldv<CG>(b + off + idx) - acc[r];
    float out = res;
    if (mode == 1) {
      out = fmaf(ca, ldv<CG>(u + off + idx), om * invd[idx] * res);
      if (w) out = fmaf(cc, ldv<CG>(w + off + idx), out);
    }
    y[off + idx] = ((mk >> r) & 1) ? 0.f : out;
  }
}

// Coarse node nd: b_c = P^T r_f for f = 2 (3^dim fine neighbours; fine fixed
// DOFs read as 0, coarse fixed DOFs set to 0).  With x0 given, also the
// coarse level's first smoothing step from zero, x0 = omega D^-1 b_c.
// offf / offc: the case's offsets on the fine and coarse levels.
template <int DIM, bool CG>
__device__ __forceinline__ void restrict2_node(const Grid& gf, const Grid& gc, const uint8_t* __restrict__ mf,
                                               const uint8_t* __restrict__ mc, const float* rf, float* bc, float* x0,
                                               const float* __restrict__ invd, float omega, int nd, long long offf,
                                               long long offc) {
  const int nxy = gc.nx * gc.ny;
  const int Kz = nd / nxy, rem = nd - Kz * nxy, J = rem / gc.nx, I = rem - J * gc.nx;
  float acc[DIM];
#pragma unroll
  for (int s2 = 0; s2 < DIM; s2++) acc[s2] = 0.f;
#pragma unroll
  for (int dz = (DIM == 3 ? -1 : 0); dz <= (DIM == 3 ? 1 : 0); dz++) {
    const int fk = 2 * Kz + dz;
    if (fk < 0 || fk >= gf.nz) continue;
#pragma unroll
    for (int dy = -1; dy <= 1; dy++) {
      const int fj = 2 * J + dy;
      if (fj < 0 || fj >= gf.ny) continue;
#pragma unroll
      for (int dx = -1; dx <= 1; dx++) {
        const int fi = 2 * I + dx;
        if (fi < 0 || fi >= gf.nx) continue;
        const float wgt = (dx ? 0.5f : 1.f) * (dy ? 0.5f : 1.f) * (dz ? 0.5f : 1.f);
        const long long n2 = node_index(gf, fi, fj, fk);
        const uint8_t m2 = mf[n2];
#pragma unroll
        for (int s2 = 0; s2 < DIM; s2++)
          if (!((m2 >> s2) & 1)) acc[s2] = fmaf(wgt, ldv<CG>(rf + offf + n2 * DIM + s2), acc[s2]);
      }
    }
  }
  const uint8_t mk = mc[nd];
#pragma unroll
  for (int s2 = 0; s2 < DIM; s2++) {
    const long long idx = (long long)nd * DIM + s2;
    const float v = ((mk >> s2) & 1) ? 0.f : acc[s2];
    bc[offc + idx] = v;
    if (x0) x0[offc + idx] = omega * invd[idx] * v;
  }
}

// The same for a coarsening factor f > 2: the warp's lanes split the
// (2f - 1)^dim fine neighbours of coarse node nd and the sum is reduced in a
// fixed order; lane 0 stores.  All 32 lanes must call it.
template <int DIM, bool CG>
__device__ __forceinline__ void restrict_warp(const Grid& gf, const Grid& gc, int f, const uint8_t* __restrict__ mf,
                                              const uint8_t* __restrict__ mc, const float* rf, float* bc, float* x0,
                                              const float* __restrict__ invd, float omega, int nd, long long offf,
                                              long long offc, int lane) {
  const int nxy = gc.nx * gc.ny;
  const int w = 2 * f - 1, nz = DIM == 3 ? w : 1, tot = w * w * nz;
  const int Kz = nd / nxy, rem = nd - Kz * nxy, J = rem / gc.nx, I = rem - J * gc.nx;
  float acc[DIM];
#pragma unroll
  for (int s2 = 0; s2 < DIM; s2++) acc[s2] = 0.f;
  for (int q = lane; q < tot; q += 32) {
    const int dx = q % w - (f - 1), dy = (q / w) % w - (f - 1), dz = DIM == 3 ? q / (w * w) - (f - 1) : 0;
    const int fi = f * I + dx, fj = f * J + dy, fk = f * Kz + dz;
    if (fi < 0 || fi >= gf.nx || fj < 0 || fj >= gf.ny || fk < 0 || fk >= gf.nz) continue;
    float wgt = (1.f - fabsf((float)dx) / f) * (1.f - fabsf((float)dy) / f);
    if (DIM == 3) wgt *= 1.f - fabsf((float)dz) / f;
    const long long n2 = node_index(gf, fi, fj, fk);
    const uint8_t m2 = mf[n2];
#pragma unroll
    for (int s2 = 0; s2 < DIM; s2++)
      if (!((m2 >> s2) & 1)) acc[s2] = fmaf(wgt, ldv<CG>(rf + offf + n2 * DIM + s2), acc[s2]);
  }
#pragma unroll
  for (int s2 = 0; s2 < DIM; s2++)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[s2] += __shfl_xor_sync(0xffffffffu, acc[s2], o);
  if (lane == 0) {
    const uint8_t mk = mc[nd];
#pragma unroll
    for (int s2 = 0; s2 < DIM; s2++) {
      const long long idx = (long long)nd * DIM + s2;
      const float v = ((mk >> s2) & 1) ? 0.f : acc[s2];
      bc[offc + idx] = v;
      if (x0) x0[offc + idx] = omega * invd[idx] * v;
    }
  }
}

// Fine node nd: x_f += P x_c on its free DOFs.
template <int DIM, bool CG>
__device__ __forceinline__ void prolong_node(const Grid& gf, const Grid& gc, int f, const uint8_t* __restrict__ mf,
                                             const float* xc, float* xf, int nd, long long offf, long long offc) {
  constexpr int NC = DIM == 2 ? 4 : 8;
  const int nxy = gf.nx * gf.ny;
  const int k = nd / nxy, rem = nd - k * nxy, j = rem / gf.nx, i = rem - j * gf.nx;
  const int I = min(i / f, gc.ex - 1), J = min(j / f, gc.ey - 1), Kz = DIM == 3 ? min(k / f, gc.ez - 1) : 0;
  const int tx = i - f * I, ty = j - f * J, tz = k - f * Kz;
  float acc[DIM];
#pragma unroll
  for (int s = 0; s < DIM; s++) acc[s] = 0.f;
#pragma unroll
  for (int C = 0; C < NC; C++) {
    float wgt = w1(cofs(C, 0), tx, f) * w1(cofs(C, 1), ty, f);
    if (DIM == 3) wgt *= w1(cofs(C, 2), tz, f);
    if (wgt == 0.f) continue;
    const long long n2 = node_index(gc, I + cofs(C, 0), J + cofs(C, 1), Kz + (DIM == 3 ? cofs(C, 2) : 0));
#pragma unroll
    for (int s = 0; s < DIM; s++) acc[s] = fmaf(wgt, ldv<CG>(xc + offc + n2 * DIM + s), acc[s]);
  }
  const uint8_t mk = mf[nd];
#pragma unroll
  for (int s = 0; s < DIM; s++)
    if (!((mk >> s) & 1)) {
      const long long idx = offf + (long long)nd * DIM + s;
      xf[idx] = ldv<CG>(xf + idx) + acc[s];
    }
}

// Coarsest solve, row i for every case: x_c,i = sum_j Ainv_ij b_c,j (case
// stride n); one warp per row (all lanes call it), the matrix read once for
// all cases; lane 0 stores.  When n is a multiple of 4 (rows and case vectors
// then start on 16-byte boundaries: the buffers are whole allocations) each
// lane reads 128-bit words (four in flight in the standalone kernel, one in
// the register-bound persistent kernel); the row is otherwise read one float
// per lane.
template <bool CG>
__device__ __forceinline__ void dense_row(int n, int nc, const float* __restrict__ Ainv, const float* b, float* x,
                                          int i, int lane) {
  constexpr int kCases = 8;
  float acc[kCases];
#pragma unroll
  for (int c = 0; c < kCases; c++) acc[c] = 0.f;
  const float* Ar = Ainv + (long long)i * n;
  if ((n & 3) == 0) {
    const float4* A4 = reinterpret_cast<const float4*>(Ar);
    const int n4 = n >> 2;
#pragma unroll(CG ? 1 : 4)
    for (int j = lane; j < n4; j += 32) {
      const float4 a = __ldg(A4 + j);
#pragma unroll
      for (int c = 0; c < kCases; c++)
        if (c < nc) {
          const float4* bp = reinterpret_cast<const float4*>(b + (long long)c * n) + j;
          const float4 v = CG ? __ldcg(bp) : *bp;
          acc[c] = fmaf(a.x, v.x, fmaf(a.y, v.y, fmaf(a.z, v.z, fmaf(a.w, v.w, acc[c]))));
        }
    }
  } else {
    for (int j = lane; j < n; j += 32) {
      const float a = Ar[j];
#pragma unroll
      for (int c = 0; c < kCases; c++)
        if (c < nc) acc[c] = fmaf(a, ldv<CG>(b + (long long)c * n + j), acc[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < kCases; c++) {
    if (c >= nc) break;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
    if (lane == 0) x[(long long)c * n + i] = acc[c];
  }
}

}  // namespace mgops
}  // namespace tp
