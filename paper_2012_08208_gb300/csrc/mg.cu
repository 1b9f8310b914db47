// Geometric multigrid preconditioner for the CG solve (not in the paper, which
// factorises K directly): nested structured grids, Galerkin coarse operators
// held as per-element matrices, Chebyshev smoothing on the l1-Jacobi scaling,
// and a dense FP32 inverse of the coarsest grid (at most 4096 DOFs, formed on
// the device; mg_dense.cu).
//
// Level 0 is the problem's grid with element matrices E_e K0.  A coarse
// element of level l + 1 covers f^dim elements of level l (f = 2 while every
// element count is even, in 3D f = 4 first when every count divides by 4, then
// the smallest odd factor common to all counts);
// with the multilinear interpolation P of the coarse element's corner values
// onto the fine nodes inside it, the coarse element matrix is the Galerkin sum
//   K_E = sum_{children c} P_c^T (M K_c M) P_c,
// M zeroing the fine fixed DOFs.  A coarse DOF is fixed when the fine DOF at the
// same place is; its rows and columns are zeroed and the operator is the
// identity there.  Restriction is P^T.  All vectors are [case][node * dim + comp]
// (the ABI layout), FP32 inside the V-cycle.
#include <algorithm>
#include <type_traits>
#include <cmath>
#include <cstring>
#include <vector>

#include "mg.h"
#include "mg_dots.cuh"
#include "mg_ops.cuh"

namespace tp {
namespace {

template <int DIM>
struct MgC {
  static constexpr int NC = DIM == 2 ? 4 : 8;  // element corners
  static constexpr int ND = NC * DIM;          // element DOFs
};

__constant__ float c_K0[24 * 24];  // level-0 element matrix (unit modulus), row-major
__constant__ float c_K0abs[24];    // its l1 row sums, sum_b |K0[a][b]|

using mgops::node_index;
using mgops::w1;

// Element matrix entry (row a, column b) of element e on a level.
template <int DIM>
__device__ __forceinline__ float kentry(const float* K, const float* E, long long e, int a, int b) {
  constexpr int ND = MgC<DIM>::ND;
  return K ? K[e * ND * ND + a * ND + b] : E[e] * c_K0[a * ND + b];
}

// Assembled form of a level: per node, the DIM x DIM coupling blocks to itself
// and to its forward neighbours (symmetric storage, mgops::sblock; structure of
// arrays: one coalesced load per entry), with the rows and columns of fixed
// DOFs zeroed.
template <int DIM>
__global__ void stencil_kernel(Grid g, const float* __restrict__ K, const float* __restrict__ E,
                               const uint8_t* __restrict__ mask, float* __restrict__ S) {
  constexpr int NC = MgC<DIM>::NC, ND = MgC<DIM>::ND, NB = DIM == 2 ? 9 : 27, C0 = mgops::Sym<DIM>::kSelf;
  const int nn = (int)g.nn, nxy = g.nx * g.ny;
  for (int nd = blockIdx.x * blockDim.x + threadIdx.x; nd < nn; nd += gridDim.x * blockDim.x) {
    const int k = DIM == 3 ? nd / nxy : 0, rem = nd - k * nxy, j = rem / g.nx, i = rem - j * g.nx;
    const uint8_t mk = mask[nd];
    for (int nbr = C0; nbr < NB; nbr++) {  // one DIM x DIM block at a time, summed in registers
      const int dx = nbr % 3 - 1, dy = (nbr / 3) % 3 - 1, dz = DIM == 3 ? nbr / 9 - 1 : 0;
      float acc[DIM * DIM];
#pragma unroll
      for (int q = 0; q < DIM * DIM; q++) acc[q] = 0.f;
      const int i2 = i + dx, j2 = j + dy, k2 = k + dz;
      if (i2 >= 0 && i2 < g.nx && j2 >= 0 && j2 < g.ny && k2 >= 0 && k2 < g.nz) {
        const uint8_t m2 = mask[node_index(g, i2, j2, k2)];
        for (int c = 0; c < NC; c++) {  // elements holding this node as corner c ...
          const int ei = i - cofs(c, 0), ej = j - cofs(c, 1), ek = k - (DIM == 3 ? cofs(c, 2) : 0);
          if (ei < 0 || ej < 0 || ek < 0 || ei >= g.ex || ej >= g.ey || ek >= g.ez) continue;
          // ... and the neighbour as corner cc
          const int ox = cofs(c, 0) + dx, oy = cofs(c, 1) + dy, oz = (DIM == 3 ? cofs(c, 2) : 0) + dz;
          if (ox < 0 || ox > 1 || oy < 0 || oy > 1 || oz < 0 || oz > 1) continue;
          const int cc = h8_corner(ox, oy, DIM == 3 ? oz : 0);
          const long long e = ei + (long long)g.ex * (ej + (long long)g.ey * ek);
          const float* Ke = K ? K + e * ND * ND : c_K0;
          const float sc = K ? 1.f : E[e];
#pragma unroll
          for (int r = 0; r < DIM; r++)
#pragma unroll
            for (int s2 = 0; s2 < DIM; s2++) acc[r * DIM + s2] = fmaf(sc, Ke[(c * DIM + r) * ND + cc * DIM + s2], acc[r * DIM + s2]);
        }
#pragma unroll
        for (int r = 0; r < DIM; r++)
#pragma unroll
          for (int s2 = 0; s2 < DIM; s2++)
            if (((mk >> r) & 1) || ((m2 >> s2) & 1)) acc[r * DIM + s2] = 0.f;
      }
#pragma unroll
      for (int q = 0; q < DIM * DIM; q++) S[((long long)(nbr - C0) * DIM * DIM + q) * nn + nd] = acc[q];
    }
  }
}

// Chebyshev step / residual on an assembled coarse level (mgops::stencil_node);
// one thread per node and case (blockIdx.y = case).
template <int DIM>
__global__ void apply_stencil_kernel(Grid g, const float* __restrict__ S, const uint8_t* __restrict__ mask,
                                     const float* __restrict__ invd, const float* u, const float* w, const float* b,
                                     float* y, int mode, float ca, float cc, float om, const int* __restrict__ stop) {
  if (halted(stop)) return;
  const int nn = (int)g.nn;
  const long long off = (long long)blockIdx.y * nn * DIM;
  for (int nd = blockIdx.x * blockDim.x + threadIdx.x; nd < nn; nd += gridDim.x * blockDim.x)
    mgops::stencil_node<DIM, false>(g, S, mask, invd, u, w, b, y, mode, ca, cc, om, nd, off);
}

// The same step on a small assembled 3D level with G lanes per node (G = 2,
// 4, 8, 16): lane g of a group takes neighbours g, g + G, ... < 27, the
// partial rows are summed by a fixed xor butterfly over the group, and lanes
// 0..2 finish one component each with mgops::stencil_node's formula.  A small
// level has too few nodes for one thread per node to keep its ~300 loads in
// flight; a warp per node would leave five lanes idle and take a wave of
// warps per 9,728 nodes.  Every lane runs the same trip count (the stride is
// uniform over the grid), so the shuffles always see the whole warp.
template <int G>
__global__ void __launch_bounds__(256) apply_stencil_group_kernel(Grid g, const float* __restrict__ S,
                                                                  const uint8_t* __restrict__ mask,
                                                                  const float* __restrict__ invd, const float* u,
                                                                  const float* w, const float* b, float* y, int mode,
                                                                  float ca, float cc, float om,
                                                                  const int* __restrict__ stop) {
  static_assert(G >= 2 && G <= 16 && (G & (G - 1)) == 0, "a power of two up to 16");
  constexpr int kNbr = (27 + G - 1) / G;
  if (halted(stop)) return;
  const int nn = (int)g.nn, nxy = g.nx * g.ny;
  const long long off = (long long)blockIdx.y * nn * 3;
  const int sub = threadIdx.x & (G - 1);
  const int groups = (gridDim.x * blockDim.x) / G;
  for (int base = 0; base < nn; base += groups) {
    const int nd = base + (int)((blockIdx.x * blockDim.x + threadIdx.x) / G);
    const bool active = nd < nn;
    const int k = nd / nxy, rem = nd - k * nxy, j = rem / g.nx, i = rem - j * g.nx;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
    for (int q = 0; q < kNbr; q++) {
      const int nbr = sub + G * q;
      const int dx = nbr % 3 - 1, dy = (nbr / 3) % 3 - 1, dz = nbr / 9 - 1;
      if (active && nbr < 27 && i + dx >= 0 && i + dx < g.nx && j + dy >= 0 && j + dy < g.ny && k + dz >= 0 &&
          k + dz < g.nz) {
        const int n2 = nd + dx + g.nx * dy + nxy * dz;
#pragma unroll
        for (int s2 = 0; s2 < 3; s2++) {
          const float v = u[off + (long long)n2 * 3 + s2];
          a0 = fmaf(mgops::sblock<3>(S, nn, nd, nbr, n2, 0, s2), v, a0);
          a1 = fmaf(mgops::sblock<3>(S, nn, nd, nbr, n2, 1, s2), v, a1);
          a2 = fmaf(mgops::sblock<3>(S, nn, nd, nbr, n2, 2, s2), v, a2);
        }
      }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      a0 += __shfl_xor_sync(0xffffffffu, a0, o);
      a1 += __shfl_xor_sync(0xffffffffu, a1, o);
      a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    }
    if (active && sub < 3) {
      const float acc = sub == 0 ? a0 : (sub == 1 ? a1 : a2);
      const long long idx = (long long)nd * 3 + sub;
      const float res = b[off + idx] - acc;
      float out = res;
      if (mode == 1) {
        out = fmaf(ca, u[off + idx], om * invd[idx] * res);
        if (w) out = fmaf(cc, w[off + idx], out);
      }
      y[off + idx] = ((mask[nd] >> sub) & 1) ? 0.f : out;
    }
  }
}

// 3D levels with at most this many nodes run their stencil steps with 8 lanes
// per node; above, one thread per node (a warp then reads 32 consecutive
// nodes of each stored coupling entry in one request).
constexpr long long kWarpNodes = 65536;
// 3D coarse levels with at most this many nodes are restricted one warp per
// coarse node (too few nodes for one thread each to keep loads in flight).
constexpr long long kWarpRestrictNodes = 8192;

// Inverse l1 row sums from the assembled form (see diag_kernel).
template <int DIM>
__global__ void diag_stencil_kernel(Grid g, const float* __restrict__ S, const uint8_t* __restrict__ mask,
                                    float* __restrict__ invd) {
  const int nn = (int)g.nn, nxy = g.nx * g.ny;
  for (int nd = blockIdx.x * blockDim.x + threadIdx.x; nd < nn; nd += gridDim.x * blockDim.x) {
    const int k = DIM == 3 ? nd / nxy : 0, rem = nd - k * nxy, j = rem / g.nx, i = rem - j * g.nx;
    const uint8_t mk = mask[nd];
    float d[DIM];
#pragma unroll
    for (int r = 0; r < DIM; r++) d[r] = 0.f;
    for (int dz = (DIM == 3 ? -1 : 0); dz <= (DIM == 3 ? 1 : 0); dz++) {
      if (k + dz < 0 || k + dz >= g.nz) continue;
      for (int dy = -1; dy <= 1; dy++) {
        if (j + dy < 0 || j + dy >= g.ny) continue;
        for (int dx = -1; dx <= 1; dx++) {
          if (i + dx < 0 || i + dx >= g.nx) continue;
          const int nbr = (dx + 1) + 3 * (dy + 1) + (DIM == 3 ? 9 * (dz + 1) : 0);
          const int n2 = nd + dx + g.nx * dy + nxy * dz;
#pragma unroll
          for (int r = 0; r < DIM; r++)
#pragma unroll
            for (int s2 = 0; s2 < DIM; s2++) d[r] += fabsf(mgops::sblock<DIM>(S, nn, nd, nbr, n2, r, s2));
        }
      }
    }
#pragma unroll
    for (int r = 0; r < DIM; r++) invd[(long long)nd * DIM + r] = ((mk >> r) & 1) || !(d[r] > 0.f) ? 1.f : 1.f / d[r];
  }
}

// Inverse l1 row sums of a level, 1 / sum_j |A_ij| (1 on fixed DOFs): the
// l1-Jacobi smoother x += omega D_l1^-1 (b - A x) contracts in the A-norm for
// any SPD A and any weight 0 < omega < 2 (the eigenvalues of D_l1^-1 A lie in
// (0, 1]).
template <int DIM>
__global__ void diag_kernel(Grid g, const float* __restrict__ K, const float* __restrict__ E,
                            const uint8_t* __restrict__ mask, float* __restrict__ invd) {
  constexpr int NC = MgC<DIM>::NC;
  const int nn = (int)g.nn, nxy = g.nx * g.ny;
  for (int nd = blockIdx.x * blockDim.x + threadIdx.x; nd < nn; nd += gridDim.x * blockDim.x) {
    const int k = DIM == 3 ? nd / nxy : 0, rem = nd - k * nxy, j = rem / g.nx, i = rem - j * g.nx;
    float d[DIM];
#pragma unroll
    for (int r = 0; r < DIM; r++) d[r] = 0.f;
#pragma unroll
    for (int c = 0; c < NC; c++) {
      const int ei = i - cofs(c, 0), ej = j - cofs(c, 1), ek = k - (DIM == 3 ? cofs(c, 2) : 0);
      if (ei < 0 || ej < 0 || ek < 0 || ei >= g.ex || ej >= g.ey || ek >= g.ez) continue;
      const long long e = ei + (long long)g.ex * (ej + (long long)g.ey * ek);
      constexpr int ND = MgC<DIM>::ND;
      if (!K) {  // level 0: with no fixed node in the element, row (c, r) sums to E_e sum_b |K0|
        uint8_t any = 0;
#pragma unroll
        for (int n = 0; n < NC; n++)
          any |= mask[node_index(g, ei + cofs(n, 0), ej + cofs(n, 1), ek + (DIM == 3 ? cofs(n, 2) : 0))];
        if (!any) {
          const float Ee = E[e];
#pragma unroll
          for (int r = 0; r < DIM; r++) d[r] = fmaf(Ee, c_K0abs[c * DIM + r], d[r]);
          continue;
        }
      }
#pragma unroll
      for (int r = 0; r < DIM; r++)
        for (int b = 0; b < ND; b++) {
          const int n2c = b / DIM, s2 = b % DIM;
          const long long n2 = node_index(g, ei + cofs(n2c, 0), ej + cofs(n2c, 1), ek + (DIM == 3 ? cofs(n2c, 2) : 0));
          if ((mask[n2] >> s2) & 1) continue;  // fixed columns do not couple
          d[r] += fabsf(kentry<DIM>(K, E, e, c * DIM + r, b));
        }
    }
    const uint8_t mk = mask[nd];
#pragma unroll
    for (int r = 0; r < DIM; r++) invd[nd * DIM + r] = ((mk >> r) & 1) || !(d[r] > 0.f) ? 1.f : 1.f / d[r];
  }
}

// Corner index of the offsets (x, y, z) in the order of cofs.
__host__ __device__ constexpr int corner_of(int x, int y, int z) { return (y ? (x ? 2 : 3) : (x ? 1 : 0)) + 4 * z; }

// Inverse l1 row sums of the assembled 3D level-0 operator, sum_j |A_ij| over
// the free columns j, where the 3 x 3 block A_ij = sum over the elements
// holding both nodes of E_e K0 (formed here, never stored).  Assembly cancels
// part of the element-level sums of diag_kernel: these are at most those (0.67
// to 0.75 of them inside a solid region of the H8 cantilever, equal beside
// void), and Gershgorin on the assembled rows keeps the spectrum of D^-1 A in
// (0, 1], so the same Chebyshev interval applies and smooths harder.  The
// neighbour and corner loops unroll to the 64 (corner, corner) pairs of the 8
// elements, K0 entries as constant-bank operands.
__global__ void diag_assembled_kernel(Grid g, const float* __restrict__ E, const uint8_t* __restrict__ mask,
                                      float* __restrict__ invd) {
  constexpr int ND = MgC<3>::ND;
  const int nn = (int)g.nn, nxy = g.nx * g.ny;
  for (int nd = blockIdx.x * blockDim.x + threadIdx.x; nd < nn; nd += gridDim.x * blockDim.x) {
    const int k = nd / nxy, rem = nd - k * nxy, j = rem / g.nx, i = rem - j * g.nx;
    // moduli of the 8 elements around the node (0 outside the grid); the node
    // is corner c of element c
    float Ee[8];
#pragma unroll
    for (int c = 0; c < 8; c++) {
      const int ei = i - cofs(c, 0), ej = j - cofs(c, 1), ek = k - cofs(c, 2);
      const bool in = ei >= 0 && ej >= 0 && ek >= 0 && ei < g.ex && ej < g.ey && ek < g.ez;
      Ee[c] = in ? E[ei + (long long)g.ex * (ej + (long long)g.ey * ek)] : 0.f;
    }
    float d[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int o = 0; o < 27; o++) {
      const int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = o / 9 - 1;
      if (i + ox < 0 || j + oy < 0 || k + oz < 0 || i + ox >= g.nx || j + oy >= g.ny || k + oz >= g.nz) continue;
      const uint8_t m2 = mask[nd + ox + g.nx * oy + nxy * oz];
      float blk[3][3] = {};
#pragma unroll
      for (int c = 0; c < 8; c++) {
        const int x2 = cofs(c, 0) + ox, y2 = cofs(c, 1) + oy, z2 = cofs(c, 2) + oz;
        if (x2 < 0 || x2 > 1 || y2 < 0 || y2 > 1 || z2 < 0 || z2 > 1) continue;  // resolved at compile time
        const int c2 = corner_of(x2, y2, z2);
#pragma unroll
        for (int r = 0; r < 3; r++)
#pragma unroll
          for (int s2 = 0; s2 < 3; s2++) blk[r][s2] = fmaf(Ee[c], c_K0[(c * 3 + r) * ND + c2 * 3 + s2], blk[r][s2]);
      }
#pragma unroll
      for (int r = 0; r < 3; r++)
#pragma unroll
        for (int s2 = 0; s2 < 3; s2++)
          if (!((m2 >> s2) & 1)) d[r] += fabsf(blk[r][s2]);
    }
    const uint8_t mk = mask[nd];
#pragma unroll
    for (int r = 0; r < 3; r++) invd[(long long)nd * 3 + r] = ((mk >> r) & 1) || !(d[r] > 0.f) ? 1.f : 1.f / d[r];
  }
}

// Coarse mask: a coarse node takes the fixed bits of the fine node at its place.
__global__ void coarse_mask_kernel(Grid gf, Grid gc, int f, const uint8_t* __restrict__ mf, uint8_t* __restrict__ mc) {
  const int nn = (int)gc.nn, nxy = gc.nx * gc.ny;
  for (int nd = blockIdx.x * blockDim.x + threadIdx.x; nd < nn; nd += gridDim.x * blockDim.x) {
    const int k = nd / nxy, rem = nd - k * nxy, j = rem / gc.nx, i = rem - j * gc.nx;
    mc[nd] = mf[node_index(gf, f * i, f * j, f * k)];
  }
}


// Galerkin coarse element matrices: one CTA per coarse element, one thread per
// entry.  For each child c (fine DOFs masked), with Phi_c[n][C] the weight of
// coarse corner C at the child's node n, in two separable stages:
//   T = K_c (Phi_c x I),   K_E += (Phi_c x I)^T T.
// The children are taken kGalChunk at a time: their matrices and fine-node
// fixed bits are loaded together (all loads of a thread in flight at once),
// then both stages run over the staged children between three barriers.  The
// sums keep the order child by child, corner by corner.  With a list, the CTAs
// stride over the coarse elements list[0 .. *list_count) instead of taking
// element blockIdx.x.
constexpr int kGalChunk = 8;

template <int DIM>
__global__ void __launch_bounds__(MgC<DIM>::ND * MgC<DIM>::ND, DIM == 3 ? 3 : 16) galerkin_kernel(Grid gf, Grid gc, int f, const float* __restrict__ Kf, const float* __restrict__ Ef,
                                const float* __restrict__ K0g, const uint8_t* __restrict__ mf,
                                const uint8_t* __restrict__ mc, float* __restrict__ Kc,
                                const int* __restrict__ list = nullptr, const int* __restrict__ list_count = nullptr) {
  constexpr int NC = MgC<DIM>::NC, ND = MgC<DIM>::ND, NE = ND * ND;
  __shared__ float sK[kGalChunk * NE];
  __shared__ float sT[kGalChunk * NE];
  __shared__ float sPhi[kGalChunk * NC * NC];
  __shared__ uint8_t sM[kGalChunk * NC];
  const int t = threadIdx.x;  // blockDim.x == ND * ND
  const float k0t = Kf ? 0.f : K0g[t];
  const long long nlist = list ? (long long)*list_count : (long long)gridDim.x;
  for (long long li = blockIdx.x; li < nlist; li += gridDim.x) {
  const long long ec = list ? (long long)list[li] : li;
  const int I = (int)(ec % gc.ex), J = (int)((ec / gc.ex) % gc.ey), Kz = (int)(ec / ((long long)gc.ex * gc.ey));
  const int a = t / ND, b = t % ND;
  float acc = 0.f;
  const int nch = DIM == 2 ? f * f : f * f * f;
  for (int ch0 = 0; ch0 < nch; ch0 += kGalChunk) {
    const int m = min(kGalChunk, nch - ch0);
    float kv[kGalChunk];
#pragma unroll
    for (int q = 0; q < kGalChunk; q++) {
      kv[q] = 0.f;
      if (q < m) {
        const int ch = ch0 + q;
        const int cx = ch % f, cy = (ch / f) % f, cz = DIM == 3 ? ch / (f * f) : 0;
        const long long e = (f * I + cx) + (long long)gf.ex * ((f * J + cy) + (long long)gf.ey * (DIM == 3 ? f * Kz + cz : 0));
        kv[q] = Kf ? Kf[e * NE + t] : Ef[e] * k0t;
      }
    }
    if (t < m * NC) {
      const int ch = ch0 + t / NC, n = t % NC;
      const int cx = ch % f, cy = (ch / f) % f, cz = DIM == 3 ? ch / (f * f) : 0;
      sM[t] = mf[node_index(gf, f * I + cx + cofs(n, 0), f * J + cy + cofs(n, 1),
                            DIM == 3 ? f * Kz + cz + cofs(n, 2) : 0)];
    }
    for (int i = t; i < m * NC * NC; i += blockDim.x) {
      const int ch = ch0 + i / (NC * NC), n = (i / NC) % NC, C = i % NC;
      const int cx = ch % f, cy = (ch / f) % f, cz = DIM == 3 ? ch / (f * f) : 0;
      float w = w1(cofs(C, 0), cx + cofs(n, 0), f) * w1(cofs(C, 1), cy + cofs(n, 1), f);
      if (DIM == 3) w *= w1(cofs(C, 2), cz + cofs(n, 2), f);
      sPhi[i] = w;
    }
    __syncthreads();  // fixed bits and weights staged; the previous chunk's sT is no longer read
#pragma unroll
    for (int q = 0; q < kGalChunk; q++)
      if (q < m) {
        const bool fa = (sM[q * NC + a / DIM] >> (a % DIM)) & 1, fb = (sM[q * NC + b / DIM] >> (b % DIM)) & 1;
        sK[q * NE + t] = (fa || fb) ? 0.f : kv[q];
      }
    __syncthreads();
    {  // T_q[a][(C, s)] = sum_n K_q[a][(n, s)] Phi_q[n][C]
      const int C = b / DIM, s2 = b % DIM;
      for (int q = 0; q < m; q++) {
        float v = 0.f;
#pragma unroll
        for (int n = 0; n < NC; n++) v = fmaf(sK[q * NE + a * ND + n * DIM + s2], sPhi[(q * NC + n) * NC + C], v);
        sT[q * NE + t] = v;
      }
    }
    __syncthreads();
    {  // K_E[(C1, r)][b] += sum_n Phi_q[n][C1] T_q[(n, r)][b], child by child
      const int C1 = a / DIM, r = a % DIM;
      for (int q = 0; q < m; q++)
#pragma unroll
        for (int n = 0; n < NC; n++) acc = fmaf(sPhi[(q * NC + n) * NC + C1], sT[q * NE + (n * DIM + r) * ND + b], acc);
    }
    __syncthreads();  // sK, sPhi and sM are restaged by the next chunk
  }
  // zero rows and columns of fixed coarse DOFs
  const int Ca = a / DIM, ra = a % DIM, Cb = b / DIM, rb = b % DIM;
  const uint8_t ma = mc[node_index(gc, I + cofs(Ca, 0), J + cofs(Ca, 1), Kz + (DIM == 3 ? cofs(Ca, 2) : 0))];
  const uint8_t mb = mc[node_index(gc, I + cofs(Cb, 0), J + cofs(Cb, 1), Kz + (DIM == 3 ? cofs(Cb, 2) : 0))];
  if (((ma >> ra) & 1) || ((mb >> rb) & 1)) acc = 0.f;
  Kc[ec * NE + t] = acc;
  }
}

// The same Galerkin product for f = 2 (every coarsening of the 2:1 levels):
// the child offsets are bit fields, the element coordinates 32-bit, and the
// interpolation weights (the same for every element) are formed once per CTA
// and stored transposed, Phi_q[C][n], so a thread reads its weight column as
// 128-bit words.  The CTAs stride over the coarse elements (or the list).  The
// sums are those of galerkin_kernel, term by term in the same order, so the
// values are identical; this form issues about a third of the instructions
// (galerkin_kernel: about 1,900 per thread at level 2 of the 240 x 80 x 80
// hierarchy, issue slots 72 % busy, 0.93 ms).
template <int DIM>
__global__ void __launch_bounds__(MgC<DIM>::ND * MgC<DIM>::ND, DIM == 3 ? 3 : 16)
    galerkin2_kernel(Grid gf, Grid gc, const float* __restrict__ Kf, const float* __restrict__ Ef,
                     const float* __restrict__ K0g, const uint8_t* __restrict__ mf, const uint8_t* __restrict__ mc,
                     float* __restrict__ Kc, const int* __restrict__ list, const int* __restrict__ list_count) {
  constexpr int NC = MgC<DIM>::NC, ND = MgC<DIM>::ND, NE = ND * ND, NCH = NC;  // 2^dim children
  __shared__ float sK[NCH * NE];
  __shared__ float sT[NCH * NE];
  __shared__ __align__(16) float sPt[NCH * NC * NC];  // [child][C][n]
  __shared__ uint8_t sM[NCH * NC];
  const int t = threadIdx.x;  // blockDim.x == NE
  for (int i = t; i < NCH * NC * NC; i += blockDim.x) {
    const int q = i / (NC * NC), C = (i / NC) % NC, n = i % NC;
    const int cx = q & 1, cy = (q >> 1) & 1, cz = q >> 2;
    auto w2 = [](int o, int p) { return o ? 0.5f * (float)p : 1.f - 0.5f * (float)p; };  // w1 for f = 2
    float w = w2(cofs(C, 0), cx + cofs(n, 0)) * w2(cofs(C, 1), cy + cofs(n, 1));
    if (DIM == 3) w *= w2(cofs(C, 2), cz + cofs(n, 2));
    sPt[i] = w;
  }
  const float k0t = Kf ? 0.f : K0g[t];
  const int a = t / ND, b = t % ND;
  const int C = b / DIM, s2 = b % DIM;   // stage 1 column
  const int C1 = a / DIM, r = a % DIM;   // stage 2 row
  const unsigned ex = (unsigned)gc.ex, ey = (unsigned)gc.ey;
  const int nlist = list ? *list_count : (int)gc.ne;
  for (int li = blockIdx.x; li < nlist; li += gridDim.x) {
    const unsigned ec = list ? (unsigned)list[li] : (unsigned)li;
    const int I = (int)(ec % ex), J = (int)((ec / ex) % ey), Kz = DIM == 3 ? (int)(ec / (ex * ey)) : 0;
    float kv[NCH];
#pragma unroll
    for (int q = 0; q < NCH; q++) {
      const long long e = (2 * I + (q & 1)) + (long long)gf.ex * ((2 * J + ((q >> 1) & 1)) +
                                                                 (long long)gf.ey * (DIM == 3 ? 2 * Kz + (q >> 2) : 0));
      kv[q] = Kf ? Kf[e * NE + t] : Ef[e] * k0t;
    }
    if (t < NCH * NC) {
      const int q = t / NC, n = t % NC;
      sM[t] = mf[node_index(gf, 2 * I + (q & 1) + cofs(n, 0), 2 * J + ((q >> 1) & 1) + cofs(n, 1),
                            DIM == 3 ? 2 * Kz + (q >> 2) + cofs(n, 2) : 0)];
    }
    __syncthreads();  // weights and fixed bits staged; the previous element's stage 2 is done
#pragma unroll
    for (int q = 0; q < NCH; q++) {
      const bool fa = (sM[q * NC + a / DIM] >> (a % DIM)) & 1, fb = (sM[q * NC + b / DIM] >> (b % DIM)) & 1;
      sK[q * NE + t] = (fa || fb) ? 0.f : kv[q];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NCH; q++) {  // T_q[a][(C, s)] = sum_n K_q[a][(n, s)] Phi_q[n][C]
      float ph[NC];
#pragma unroll
      for (int n4 = 0; n4 < NC; n4 += 4) {
        const float4 v = *reinterpret_cast<const float4*>(&sPt[(q * NC + C) * NC + n4]);
        ph[n4] = v.x;
        ph[n4 + 1] = v.y;
        ph[n4 + 2] = v.z;
        ph[n4 + 3] = v.w;
      }
      float v = 0.f;
#pragma unroll
      for (int n = 0; n < NC; n++) v = fmaf(sK[q * NE + a * ND + n * DIM + s2], ph[n], v);
      sT[q * NE + t] = v;
    }
    __syncthreads();
    float acc = 0.f;
#pragma unroll
    for (int q = 0; q < NCH; q++) {  // K_E[(C1, r)][b] += sum_n Phi_q[n][C1] T_q[(n, r)][b]
      float ph[NC];
#pragma unroll
      for (int n4 = 0; n4 < NC; n4 += 4) {
        const float4 v = *reinterpret_cast<const float4*>(&sPt[(q * NC + C1) * NC + n4]);
        ph[n4] = v.x;
        ph[n4 + 1] = v.y;
        ph[n4 + 2] = v.z;
        ph[n4 + 3] = v.w;
      }
#pragma unroll
      for (int n = 0; n < NC; n++) acc = fmaf(ph[n], sT[q * NE + (n * DIM + r) * ND + b], acc);
    }
    const int Ca = a / DIM, ra = a % DIM, Cb = b / DIM, rb = b % DIM;
    const uint8_t ma = mc[node_index(gc, I + cofs(Ca, 0), J + cofs(Ca, 1), Kz + (DIM == 3 ? cofs(Ca, 2) : 0))];
    const uint8_t mb = mc[node_index(gc, I + cofs(Cb, 0), J + cofs(Cb, 1), Kz + (DIM == 3 ? cofs(Cb, 2) : 0))];
    if (((ma >> ra) & 1) || ((mb >> rb) & 1)) acc = 0.f;
    Kc[(long long)ec * NE + t] = acc;
  }
}

// Coarse elements whose footprint holds a fixed fine DOF: touched[ec] = 1
// when any of the (f + 1)^dim fine nodes inside coarse element ec has a fixed
// bit (its children's matrices are masked); those elements are also appended
// to list[0 .. *count) (*count zeroed before the launch).
template <int DIM>
__global__ void touched_kernel(Grid gf, Grid gc, int f, const uint8_t* __restrict__ mf, uint8_t* __restrict__ touched,
                               int* __restrict__ list, int* __restrict__ count) {
  const long long ne = gc.ne;
  for (long long ec = blockIdx.x * (long long)blockDim.x + threadIdx.x; ec < ne;
       ec += (long long)gridDim.x * blockDim.x) {
    const int I = (int)(ec % gc.ex), J = (int)((ec / gc.ex) % gc.ey), Kz = (int)(ec / ((long long)gc.ex * gc.ey));
    uint8_t any = 0;
    for (int z = 0; z <= (DIM == 3 ? f : 0); z++)
      for (int y = 0; y <= f; y++)
        for (int x = 0; x <= f; x++) any |= mf[node_index(gf, f * I + x, f * J + y, DIM == 3 ? f * Kz + z : 0)];
    touched[ec] = any ? 1 : 0;
    if (any) list[atomicAdd(count, 1)] = (int)ec;  // list order is free: each element is computed alone
  }
}

// The untouched elements of level 1 (K_E = sum_ch E_ch A_ch), one warp per
// element: the element's coordinates and its children's moduli are formed
// once per warp (child ch's modulus in lane ch mod 32 of one of two registers,
// broadcast by shuffle), and each lane sums ND^2 / 32 entries, child by child
// (coalesced stores).  The child matrices are staged in shared memory once per
// CTA.  Touched elements are left to galerkin_kernel (list mode).  Needs f^dim <= 64;
// shared memory (dynamic): f^dim ND^2 floats.
constexpr int kG1Threads = 1024;  // 32 warps share one staged table (it fills most of shared memory at f = 4)

template <int DIM>
__global__ void __launch_bounds__(kG1Threads) galerkin1_flat_kernel(Grid gf, Grid gc, int f, const float* __restrict__ Ef,
                                                             const float* __restrict__ A,
                                                             const uint8_t* __restrict__ touched,
                                                             float* __restrict__ Kc) {
  constexpr int ND = MgC<DIM>::ND, NE = ND * ND, kPer = NE / 32;
  static_assert(NE % 32 == 0, "whole entries per lane");
  extern __shared__ __align__(16) float sA[];  // [nch][NE]
  const int nch = DIM == 2 ? f * f : f * f * f;
  for (int i = threadIdx.x; i < nch * NE; i += blockDim.x) sA[i] = A[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long ec = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); ec < gc.ne; ec += nw) {
    if (touched[ec]) continue;  // uniform over the warp
    const unsigned e32 = (unsigned)ec;
    const int I = (int)(e32 % (unsigned)gc.ex), J = (int)((e32 / (unsigned)gc.ex) % (unsigned)gc.ey);
    const int Kz = DIM == 3 ? (int)(e32 / ((unsigned)gc.ex * (unsigned)gc.ey)) : 0;
    float ev[2] = {0.f, 0.f};
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const int ch = lane + 32 * h;
      if (ch < nch) {
        const int cx = ch % f, cy = (ch / f) % f, cz = DIM == 3 ? ch / (f * f) : 0;
        ev[h] = Ef[(f * I + cx) + (long long)gf.ex * ((f * J + cy) + (long long)gf.ey * (DIM == 3 ? f * Kz + cz : 0))];
      }
    }
    float acc[kPer];
#pragma unroll
    for (int q = 0; q < kPer; q++) acc[q] = 0.f;
    for (int ch = 0; ch < nch; ch++) {
      const float ech = __shfl_sync(0xffffffffu, ch < 32 ? ev[0] : ev[1], ch & 31);
      const float* a = sA + ch * NE + lane;
#pragma unroll
      for (int q = 0; q < kPer; q++) acc[q] = fmaf(ech, a[32 * q], acc[q]);
    }
    float* out = Kc + ec * NE + lane;
#pragma unroll
    for (int q = 0; q < kPer; q++) out[32 * q] = acc[q];
  }
}

// Restriction (mgops::restrict2_node, restrict_warp) with the coarse level's
// first smoothing step when x0 is given; blockIdx.y = case.
template <int DIM>
__global__ void restrict2_kernel(Grid gf, Grid gc, const uint8_t* __restrict__ mf, const uint8_t* __restrict__ mc,
                                 const float* rf, float* bc, float* x0, const float* __restrict__ invd, float omega,
                                 const int* __restrict__ stop) {
  if (halted(stop)) return;
  const long long offf = (long long)blockIdx.y * gf.nn * DIM, offc = (long long)blockIdx.y * gc.nn * DIM;
  const int nn = (int)gc.nn;
  for (int nd = blockIdx.x * blockDim.x + threadIdx.x; nd < nn; nd += gridDim.x * blockDim.x)
    mgops::restrict2_node<DIM, false>(gf, gc, mf, mc, rf, bc, x0, invd, omega, nd, offf, offc);
}

template <int DIM>
__global__ void restrict_kernel(Grid gf, Grid gc, int f, const uint8_t* __restrict__ mf, const uint8_t* __restrict__ mc,
                                const float* rf, float* bc, float* x0, const float* __restrict__ invd, float omega,
                                const int* __restrict__ stop) {
  if (halted(stop)) return;
  const long long offf = (long long)blockIdx.y * gf.nn * DIM, offc = (long long)blockIdx.y * gc.nn * DIM;
  const int nn = (int)gc.nn, lane = threadIdx.x & 31;
  for (int nd = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; nd < nn; nd += (gridDim.x * blockDim.x) >> 5)
    mgops::restrict_warp<DIM, false>(gf, gc, f, mf, mc, rf, bc, x0, invd, omega, nd, offf, offc, lane);
}

// x_f += P x_c on free fine DOFs (mgops::prolong_node); blockIdx.y = case.
template <int DIM>
__global__ void prolong_kernel(Grid gf, Grid gc, int f, const uint8_t* __restrict__ mf, const float* xc, float* xf,
                               const int* __restrict__ stop) {
  if (halted(stop)) return;
  const long long offf = (long long)blockIdx.y * gf.nn * DIM, offc = (long long)blockIdx.y * gc.nn * DIM;
  const int nn = (int)gf.nn;
  for (int nd = blockIdx.x * blockDim.x + threadIdx.x; nd < nn; nd += gridDim.x * blockDim.x)
    mgops::prolong_node<DIM, false>(gf, gc, f, mf, xc, xf, nd, offf, offc);
}

// Restriction and prolongation for f = 2 (prolongation also f = 4) in 3D, one thread per node on a 3D
// grid (x by threads, y by blockIdx.y, z and the case by blockIdx.z), so the
// node coordinates need no division and the weights are constants.  They form
// the sums of restrict2_node and prolong_node term by term in the same order
// (a skipped term there is an exact +0 here), so the values are identical.
// Every load of a thread is unconditional within the grid and independent of
// the fixed bits, which select afterwards: all of them are in flight at once.
constexpr int kT2X = 128;  // threads per block along x

__global__ void __launch_bounds__(kT2X)
    restrict2x_kernel(Grid gf, Grid gc, const uint8_t* __restrict__ mf, const uint8_t* __restrict__ mc,
                      const float* __restrict__ rf, float* __restrict__ bc, float* __restrict__ x0,
                      const float* __restrict__ invd, float omega, const int* __restrict__ stop) {
  if (halted(stop)) return;
  const int I = blockIdx.x * kT2X + threadIdx.x, J = blockIdx.y, K = blockIdx.z % gc.nz, c = blockIdx.z / gc.nz;
  if (I >= gc.nx) return;
  const long long offf = (long long)c * gf.nn * 3, offc = (long long)c * gc.nn * 3;
  float acc[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int dz = -1; dz <= 1; dz++) {
    const int fk = 2 * K + dz;
    if (fk < 0 || fk >= gf.nz) continue;  // uniform over the block
#pragma unroll
    for (int dy = -1; dy <= 1; dy++) {
      const int fj = 2 * J + dy;
      if (fj < 0 || fj >= gf.ny) continue;  // uniform over the block
      const long long row = (long long)gf.nx * (fj + (long long)gf.ny * fk);
      float v[3][3];
      uint8_t m[3];
#pragma unroll
      for (int dx = -1; dx <= 1; dx++) {
        const int fi = 2 * I + dx;
        const bool in = fi >= 0 && fi < gf.nx;
        const long long n2 = row + (in ? fi : 0);
        m[dx + 1] = in ? mf[n2] : (uint8_t)7;
#pragma unroll
        for (int s2 = 0; s2 < 3; s2++) v[dx + 1][s2] = in ? rf[offf + n2 * 3 + s2] : 0.f;
      }
#pragma unroll
      for (int dx = -1; dx <= 1; dx++) {
        const float wgt = (dx ? 0.5f : 1.f) * (dy ? 0.5f : 1.f) * (dz ? 0.5f : 1.f);
#pragma unroll
        for (int s2 = 0; s2 < 3; s2++)
          acc[s2] = fmaf(wgt, ((m[dx + 1] >> s2) & 1) ? 0.f : v[dx + 1][s2], acc[s2]);
      }
    }
  }
  const long long nd = I + (long long)gc.nx * (J + (long long)gc.ny * K);
  const uint8_t mk = mc[nd];
#pragma unroll
  for (int s2 = 0; s2 < 3; s2++) {
    const long long idx = nd * 3 + s2;
    const float v = ((mk >> s2) & 1) ? 0.f : acc[s2];
    bc[offc + idx] = v;
    if (x0) x0[offc + idx] = omega * invd[idx] * v;
  }
}

// Restriction for f = 4 in 3D in two passes.  The weight of fine node
// (4I + dx, 4J + dy, 4K + dz) in coarse node (I, J, K) is the product of
// (1 - |d| / 4) over the axes, so the 343-node sum separates: pass 1 sums x
// and y over the 7 x 7 fine nodes around each (coarse x, coarse y, fine z),
// fine fixed DOFs read as 0, into r4; pass 2 sums z, zeroes the coarse fixed
// DOFs and forms the coarse level's first smoothing step.  One thread per
// output node on a 3D grid (no divisions); the sums of restrict_warp in
// another order.  A warp per coarse node over the 343 fine nodes took about
// 60 us at 240 x 80 x 80.
__device__ __forceinline__ float w4(int d) { return 1.f - 0.25f * (float)(d < 0 ? -d : d); }

__global__ void __launch_bounds__(kT2X)
    restrict4_xy_kernel(Grid gf, Grid gc, const uint8_t* __restrict__ mf, const float* __restrict__ rf,
                        float* __restrict__ r4, const int* __restrict__ stop) {
  if (halted(stop)) return;
  const int I = blockIdx.x * kT2X + threadIdx.x, J = blockIdx.y, k = blockIdx.z % gf.nz, c = blockIdx.z / gf.nz;
  if (I >= gc.nx) return;
  const long long offf = (long long)c * gf.nn * 3;
  float acc[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int dy = -3; dy <= 3; dy++) {
    const int fj = 4 * J + dy;
    if (fj < 0 || fj >= gf.ny) continue;  // uniform over the block
    const long long row = (long long)gf.nx * (fj + (long long)gf.ny * k);
    float rs[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int dx = -3; dx <= 3; dx++) {
      const int fi = 4 * I + dx;
      const bool in = fi >= 0 && fi < gf.nx;
      const long long n2 = row + (in ? fi : 0);
      const uint8_t m = in ? mf[n2] : (uint8_t)7;
#pragma unroll
      for (int s2 = 0; s2 < 3; s2++) {
        const float v = in ? rf[offf + n2 * 3 + s2] : 0.f;
        rs[s2] = fmaf(w4(dx), ((m >> s2) & 1) ? 0.f : v, rs[s2]);
      }
    }
#pragma unroll
    for (int s2 = 0; s2 < 3; s2++) acc[s2] = fmaf(w4(dy), rs[s2], acc[s2]);
  }
  float* out = r4 + ((((long long)c * gf.nz + k) * gc.ny + J) * gc.nx + I) * 3;
#pragma unroll
  for (int s2 = 0; s2 < 3; s2++) out[s2] = acc[s2];
}

__global__ void __launch_bounds__(kT2X)
    restrict4_z_kernel(Grid gf, Grid gc, const float* __restrict__ r4, const uint8_t* __restrict__ mc,
                       float* __restrict__ bc, float* __restrict__ x0, const float* __restrict__ invd, float omega,
                       const int* __restrict__ stop) {
  if (halted(stop)) return;
  const int I = blockIdx.x * kT2X + threadIdx.x, J = blockIdx.y, K = blockIdx.z % gc.nz, c = blockIdx.z / gc.nz;
  if (I >= gc.nx) return;
  float acc[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int dz = -3; dz <= 3; dz++) {
    const int fk = 4 * K + dz;
    if (fk < 0 || fk >= gf.nz) continue;  // uniform over the block
    const float* in = r4 + ((((long long)c * gf.nz + fk) * gc.ny + J) * gc.nx + I) * 3;
#pragma unroll
    for (int s2 = 0; s2 < 3; s2++) acc[s2] = fmaf(w4(dz), in[s2], acc[s2]);
  }
  const long long offc = (long long)c * gc.nn * 3;
  const long long nd = I + (long long)gc.nx * (J + (long long)gc.ny * K);
  const uint8_t mk = mc[nd];
#pragma unroll
  for (int s2 = 0; s2 < 3; s2++) {
    const long long idx = nd * 3 + s2;
    const float v = ((mk >> s2) & 1) ? 0.f : acc[s2];
    bc[offc + idx] = v;
    if (x0) x0[offc + idx] = omega * invd[idx] * v;
  }
}

// The prolongation takes F = 2 or 4 (the weights t / F are exact in FP32).
template <int F>
__global__ void __launch_bounds__(kT2X)
    prolongfx_kernel(Grid gf, Grid gc, const uint8_t* __restrict__ mf, const float* __restrict__ xc,
                     float* __restrict__ xf, const int* __restrict__ stop) {
  static_assert(F == 2 || F == 4, "power-of-two factors");
  constexpr float kInvF = 1.f / F;
  if (halted(stop)) return;
  const int i = blockIdx.x * kT2X + threadIdx.x, j = blockIdx.y, k = blockIdx.z % gf.nz, c = blockIdx.z / gf.nz;
  if (i >= gf.nx) return;
  const long long offf = (long long)c * gf.nn * 3, offc = (long long)c * gc.nn * 3;
  const long long nd = i + (long long)gf.nx * (j + (long long)gf.ny * k);
  const uint8_t mk = mf[nd];
  float xv[3];
#pragma unroll
  for (int s = 0; s < 3; s++) xv[s] = xf[offf + nd * 3 + s];
  // corner 0 of the coarse element holding the node, and the node's position in it
  const int I = min(i / F, gc.ex - 1), J = min(j / F, gc.ey - 1), Kz = min(k / F, gc.ez - 1);
  const int tx = i - F * I, ty = j - F * J, tz = k - F * Kz;
  float cv[8][3];
#pragma unroll
  for (int C = 0; C < 8; C++) {
    const long long n2 = (I + cofs(C, 0)) + (long long)gc.nx * ((J + cofs(C, 1)) + (long long)gc.ny * (Kz + cofs(C, 2)));
#pragma unroll
    for (int s = 0; s < 3; s++) cv[C][s] = xc[offc + n2 * 3 + s];
  }
  float acc[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int C = 0; C < 8; C++) {
    const float wgt = (cofs(C, 0) ? kInvF * tx : 1.f - kInvF * tx) * (cofs(C, 1) ? kInvF * ty : 1.f - kInvF * ty) *
                      (cofs(C, 2) ? kInvF * tz : 1.f - kInvF * tz);
    if (wgt == 0.f) continue;
#pragma unroll
    for (int s = 0; s < 3; s++) acc[s] = fmaf(wgt, cv[C][s], acc[s]);
  }
#pragma unroll
  for (int s = 0; s < 3; s++)
    if (!((mk >> s) & 1)) xf[offf + nd * 3 + s] = xv[s] + acc[s];
}

// Coarsest solve: x = A^-1 b with the dense inverse (mgops::dense_row), all
// cases per row; one warp per row.
__global__ void dense_solve_kernel(int n, int nc, const float* __restrict__ Ainv, const float* b, float* x,
                                   const int* __restrict__ stop) {
  if (halted(stop)) return;
  const int lane = threadIdx.x & 31;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += (gridDim.x * blockDim.x) >> 5)
    mgops::dense_row<false>(n, nc, Ainv, b, x, i, lane);
}

int blocks(long long n) { return (int)std::min<long long>(std::max<long long>((n + 255) / 256, 1), 152 * 16); }

// Smallest factor f >= 2 dividing every element count (2 first), or 0.
int common_factor(const Grid& g) {
  for (int f : {2, 3, 5, 7}) {
    if (g.ex % f || g.ey % f || (g.dim == 3 && g.ez % f)) continue;
    if (g.ex / f < 1 || g.ey / f < 1 || (g.dim == 3 && g.ez / f < 1)) continue;
    return f;
  }
  return 0;
}

Grid coarsen(const Grid& g, int f) {
  Grid c = g;
  c.ex = g.ex / f;
  c.ey = g.ey / f;
  c.ez = g.dim == 3 ? g.ez / f : 1;
  c.nx = c.ex + 1;
  c.ny = c.ey + 1;
  c.nz = g.dim == 3 ? c.ez + 1 : 1;
  c.nn = (long long)c.nx * c.ny * c.nz;
  c.ne = (long long)c.ex * c.ey * c.ez;
  return c;
}

}  // namespace

// ---------------------------------------------------------------------------

double MgHierarchy::vcycle_bytes() const {
  const int dim = lv[0].g.dim, L = (int)lv.size();
  // stored coupling entries per node of an assembled level (symmetric storage)
  const double nbr = dim == 2 ? mgops::Sym<2>::kSlots * 4.0 : mgops::Sym<3>::kSlots * 9.0;
  double total = 0.0;
  for (int li = 0; li + 1 < L; li++) {
    const MgLevel& l = lv[li];
    const double nodes = (double)l.g.nn, vals = (double)nc * nodes * dim;
    // operator data of one sweep: moduli (finest) or assembled blocks, plus the scale
    const double op = (li == 0 ? 4.0 * l.g.ne : 4.0 * nbr * nodes) + 4.0 * nodes * dim;
    // Chebyshev steps before (degree - 1), residual, after (degree): u, b read, y
    // written; w read by the steps that use x_{k-2}
    const int nl = degree_at(li);
    const int steps = 2 * nl, w_reads = std::max(0, nl - 2) + (nl - 1);
    total += steps * (op + 12.0 * vals) + w_reads * 4.0 * vals;
    const MgLevel& c = lv[li + 1];
    const double cvals = (double)nc * c.g.nn * dim;
    total += 4.0 * vals + 8.0 * cvals;   // restriction: r read, b (and x0) written
    total += 8.0 * vals + 4.0 * cvals;   // prolongation: x read and written, coarse x read
  }
  total += 4.0 * (double)cn * cn + 8.0 * nc * cn;  // dense coarsest solve
  return total;
}

double MgHierarchy::fine_bytes() const {
  const MgLevel& l = lv[0];
  // finest-level sweep: moduli and the l1 scale once per launch; per case u
  // and b read, y written
  return (double)l.g.ne * 4.0 + (double)l.g.nn * l.g.dim * 4.0 * (1 + 3 * nc);
}

void MgHierarchy::collect_sweeps(int npairs) {
  for (int k = 0; k < npairs && 2 * k + 1 < (int)sweep_ev.size(); k++) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, sweep_ev[2 * k], sweep_ev[2 * k + 1]) == cudaSuccess) {
      timed_ms += ms;
      timed_launches++;
      timed_bytes += fine_bytes();
    }
  }
  cudaGetLastError();
}

double MgHierarchy::iter_bytes() const {
  const MgLevel& l = lv[0];
  const double vals = (double)nc * l.g.nn * l.g.dim;
  // operator phase: moduli, z and p_old read, q and p_new written; update: d,
  // p, q, r read, d, r, x0 written, the scale once
  return vcycle_bytes() + (4.0 * l.g.ne + 16.0 * vals) + (28.0 * vals + 4.0 * l.g.nn * l.g.dim);
}

void MgHierarchy::drop_graphs() {
  for (auto& row : gx)
    for (auto& g : row) {
      if (g) cudaGraphExecDestroy(g);
      g = nullptr;
    }
}

void MgHierarchy::release() {
  drop_graphs();
  if (cap) cudaStreamDestroy(cap);
  cap = nullptr;
  if (side) cudaStreamDestroy(side);
  side = nullptr;
  for (cudaEvent_t* e : {&fork, &join}) {
    if (*e) cudaEventDestroy(*e);
    *e = nullptr;
  }
  for (auto& e : ev) {
    if (e) cudaEventDestroy(e);
    e = nullptr;
  }
  for (auto& e : sweep_ev) cudaEventDestroy(e);
  sweep_ev.clear();
  ev_used = 0;
  for (auto& l : lv) {
    void* ptrs[] = {l.K, l.S, l.mask_own ? (void*)l.mask : nullptr, l.invd, l.x[0], l.x[1], l.b, l.t, l.r4};
    for (void* q : ptrs)
      if (q) cudaFree(q);
  }
  lv.clear();
  for (void* q : {(void*)A1, (void*)touched1, (void*)touched_list}) if (q) cudaFree(q);
  A1 = nullptr;
  touched1 = nullptr;
  touched_list = nullptr;
  for (void* q : {(void*)cinv, (void*)K0d, (void*)ctl, (void*)p32, (void*)q32, (void*)d32, (void*)p32b,
                  (void*)dscratch, (void*)dflag})
    if (q) cudaFree(q);
  if (ctl_h) cudaFreeHost(ctl_h);
  cinv = nullptr;
  K0d = nullptr;
  ctl = nullptr;
  ctl_h = nullptr;
  p32 = q32 = d32 = p32b = dscratch = nullptr;
  dflag = nullptr;
  dinv.destroy();
  built = false;
}

// Chebyshev coefficients for the interval [1 / ratio, 1] (centre theta,
// half-width delta, sigma = theta / delta): with rho_1 = 1 / sigma and
// rho_k = 1 / (2 sigma - rho_{k-1}), the step direction d_k = rho_k rho_{k-1}
// d_{k-1} + (2 rho_k / delta) D^-1 r_k gives the three-term form above.
void MgHierarchy::set_smoother(int degree, float ratio) {
  nu = std::max(1, std::min(degree, 7));
  cheb_ratio = ratio;
  const double lo = 1.0 / ratio, theta = 0.5 * (1.0 + lo), delta = 0.5 * (1.0 - lo), sigma = theta / delta;
  omega = (float)(1.0 / theta);
  double rho_prev = 1.0 / sigma;
  for (int k = 2; k <= nu; k++) {
    const double rho = 1.0 / (2.0 * sigma - rho_prev);
    ca[k] = (float)(1.0 + rho * rho_prev);
    cc[k] = (float)(-rho * rho_prev);
    cw[k] = (float)(2.0 * rho / delta);
    rho_prev = rho;
  }
}

cudaError_t MgHierarchy::plan(const Grid& g0, const uint8_t* mask0, int nc_, int max_coarse_dofs) {
  release();
  nc = nc_;
  set_smoother(nu, cheb_ratio);
  nu0 = g0.nn > (g0.dim == 3 ? kDegree1Nodes3D : kDegree1Nodes) ? 1 : nu;
  MgLevel l0;
  l0.g = g0;
  l0.f = 1;
  l0.mask = const_cast<uint8_t*>(mask0);
  l0.mask_own = false;
  lv.push_back(l0);
  // coarsen until the first level with at most max_coarse_dofs DOFs (the
  // largest coarsest grid the dense inverse takes), at least once
  while ((int)lv.size() < 12 && (lv.size() < 2 || lv.back().g.nn * g0.dim > max_coarse_dofs)) {
    int f = common_factor(lv.back().g);
    if (!f) break;
    // 3D: the first coarsening is 4:1 when every element count allows it.
    // It drops the level 8x finer than level 2, whose assembled blocks and
    // Galerkin element matrices are the largest of the hierarchy; at
    // 240 x 80 x 80 the SIMP step took 37.8 ms against 40.1 ms with 2:1, the
    // iterations growing by about 4 % (12 % at 120 x 40 x 40).  In 2D it was
    // neutral at 600 x 200 (10 % more iterations), so 2D keeps 2:1.
    if (lv.size() == 1 && f == 2 && g0.dim == 3 && g0.ex % 4 == 0 && g0.ey % 4 == 0 && g0.ez % 4 == 0) f = 4;
    MgLevel l;
    l.g = coarsen(lv.back().g, f);
    l.f = f;
    lv.push_back(l);
  }
  if (lv.back().g.nn * g0.dim > max_coarse_dofs || lv.size() < 2) return cudaErrorInvalidValue;
  cudaError_t e = cudaSuccess;
  for (size_t i = 0; i < lv.size() && e == cudaSuccess; i++) {
    MgLevel& l = lv[i];
    const long long ndof = l.g.nn * g0.dim, nd = g0.dim == 2 ? 8 : 24;
    if (i > 0) {
      e = cudaMalloc((void**)&l.K, l.g.ne * nd * nd * sizeof(float));
      if (e == cudaSuccess) e = cudaMalloc((void**)&l.mask, l.g.nn);
      l.mask_own = true;
    }
    if (e == cudaSuccess && i > 0) {
      const long long nb = g0.dim == 2 ? mgops::Sym<2>::kSlots * 4 : mgops::Sym<3>::kSlots * 9;
      e = cudaMalloc((void**)&l.S, l.g.nn * nb * sizeof(float));
    }
    if (e == cudaSuccess) e = cudaMalloc((void**)&l.invd, ndof * sizeof(float));
    for (int k = 0; k < 2 && e == cudaSuccess; k++) e = cudaMalloc((void**)&l.x[k], nc * ndof * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void**)&l.b, nc * ndof * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void**)&l.t, nc * ndof * sizeof(float));
    if (e == cudaSuccess && i > 0 && l.f == 4 && g0.dim == 3)
      e = cudaMalloc((void**)&l.r4, (size_t)nc * lv[i - 1].g.nz * l.g.ny * l.g.nx * 3 * sizeof(float));
  }
  {
    const int f1 = lv[1].f, nd = g0.dim == 2 ? 8 : 24;
    const long long nch = g0.dim == 2 ? f1 * f1 : f1 * f1 * f1;
    if (e == cudaSuccess) e = cudaMalloc((void**)&A1, nch * nd * nd * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void**)&touched1, std::max<long long>(lv[1].g.ne, 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)&touched_list, (lv[1].g.ne + 1) * sizeof(int));
  }
  cn = (int)(lv.back().g.nn * g0.dim);
  if (e == cudaSuccess) e = cudaMalloc((void**)&cinv, (size_t)cn * cn * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&dscratch, dense_scratch_floats(cn) * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&dflag, sizeof(int));
  const size_t nv = (size_t)nc * g0.nn * g0.dim;
  if (e == cudaSuccess) e = cudaMalloc((void**)&p32, nv * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&q32, nv * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&d32, nv * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&p32b, nv * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&ctl, sizeof(MgCtl));
  if (e == cudaSuccess) e = cudaMemset(ctl, 0, sizeof(MgCtl));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&ctl_h, sizeof(MgCtl));
  return e;
}

cudaError_t MgHierarchy::build(cudaStream_t s, const double* K0, const float* E32, int* nlaunch) {
  const int dim = lv[0].g.dim, nd = dim == 2 ? 8 : 24;
  std::vector<float> k0f(nd * nd);
  for (int i = 0; i < nd * nd; i++) k0f[i] = (float)K0[i];
  cudaError_t e = cudaMemcpyToSymbolAsync(c_K0, k0f.data(), nd * nd * sizeof(float), 0, cudaMemcpyHostToDevice, s);
  k0abs.assign(nd, 0.f);
  for (int a = 0; a < nd; a++) {
    double r = 0.0;
    for (int b = 0; b < nd; b++) r += std::fabs((double)k0f[a * nd + b]);
    k0abs[a] = (float)r;
  }
  if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_K0abs, k0abs.data(), nd * sizeof(float), 0, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !K0d) e = cudaMalloc((void**)&K0d, nd * nd * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpyAsync(K0d, k0f.data(), nd * nd * sizeof(float), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  E0 = E32;
  int nl = 0;
  {  // level-1 child matrices A_ch = P_ch^T K0 P_ch (FP64 sums, stored in FP32)
    const int f = lv[1].f, NC = dim == 2 ? 4 : 8;
    const int nch = dim == 2 ? f * f : f * f * f;
    std::vector<float> Ah((size_t)nch * nd * nd);
    for (int ch = 0; ch < nch; ch++) {
      const int cxyz[3] = {ch % f, (ch / f) % f, dim == 3 ? ch / (f * f) : 0};
      double phi[8][8];
      for (int n = 0; n < NC; n++)
        for (int C = 0; C < NC; C++) {
          double w = 1.0;
          for (int ax = 0; ax < dim; ax++) {
            const double t = (double)(cxyz[ax] + cofs(n, ax)) / f;
            w *= cofs(C, ax) ? t : 1.0 - t;
          }
          phi[n][C] = w;
        }
      for (int a = 0; a < nd; a++)
        for (int b = 0; b < nd; b++) {
          const int C1 = a / dim, r = a % dim, C2 = b / dim, s2 = b % dim;
          double v = 0.0;
          for (int n = 0; n < NC; n++)
            for (int m = 0; m < NC; m++) v += phi[n][C1] * phi[m][C2] * K0[(n * dim + r) * nd + m * dim + s2];
          Ah[((size_t)ch * nd + a) * nd + b] = (float)v;
        }
    }
    e = cudaMemcpyAsync(A1, Ah.data(), Ah.size() * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
  }
  for (size_t i = 0; i < lv.size(); i++) {
    MgLevel& l = lv[i];
    if (i > 0) {
      const MgLevel& fl = lv[i - 1];
      coarse_mask_kernel<<<blocks(l.g.nn), 256, 0, s>>>(fl.g, l.g, l.f, fl.mask, l.mask);
      // Level 1: K_E = sum_ch E_ch A_ch for the coarse elements that no fixed
      // fine DOF touches (warp per element, child matrices staged in shared
      // memory, f^dim <= 64); the touched ones by the masked triple product of
      // galerkin_kernel over their list.  Otherwise galerkin_kernel for all.
      const int nch1 = dim == 2 ? l.f * l.f : l.f * l.f * l.f;
      const size_t smf = (size_t)nch1 * nd * nd * sizeof(float);
      if (i == 1 && nch1 <= 64 && smf <= 160 * 1024) {
        e = cudaMemsetAsync(touched_list, 0, sizeof(int), s);
        if (e != cudaSuccess) return e;
        const unsigned g1grid =
            (unsigned)std::max<long long>(1, std::min<long long>((l.g.ne + 31) / 32, 152 * 2));  // warp per element
        if (dim == 2) {
          touched_kernel<2><<<blocks(l.g.ne), 256, 0, s>>>(fl.g, l.g, l.f, fl.mask, touched1, touched_list + 1,
                                                           touched_list);
          e = cudaFuncSetAttribute(galerkin1_flat_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smf);
          if (e != cudaSuccess) return e;
          galerkin1_flat_kernel<2><<<g1grid, kG1Threads, smf, s>>>(fl.g, l.g, l.f, E32, A1, touched1, l.K);
          if (l.f == 2)
            galerkin2_kernel<2><<<152 * 16, 64, 0, s>>>(fl.g, l.g, nullptr, E32, K0d, fl.mask, l.mask, l.K,
                                                        touched_list + 1, touched_list);
          else
            galerkin_kernel<2><<<152 * 16, 64, 0, s>>>(fl.g, l.g, l.f, nullptr, E32, K0d, fl.mask, l.mask, l.K,
                                                       touched_list + 1, touched_list);
        } else {
          touched_kernel<3><<<blocks(l.g.ne), 256, 0, s>>>(fl.g, l.g, l.f, fl.mask, touched1, touched_list + 1,
                                                           touched_list);
          e = cudaFuncSetAttribute(galerkin1_flat_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smf);
          if (e != cudaSuccess) return e;
          galerkin1_flat_kernel<3><<<g1grid, kG1Threads, smf, s>>>(fl.g, l.g, l.f, E32, A1, touched1, l.K);
          if (l.f == 2)
            galerkin2_kernel<3><<<152 * 3, 576, 0, s>>>(fl.g, l.g, nullptr, E32, K0d, fl.mask, l.mask, l.K,
                                                        touched_list + 1, touched_list);
          else
            galerkin_kernel<3><<<152 * 3, 576, 0, s>>>(fl.g, l.g, l.f, nullptr, E32, K0d, fl.mask, l.mask, l.K,
                                                       touched_list + 1, touched_list);
        }
        nl += 2;  // the touched-element flags and the flat kernel (the list launch is counted below)
      } else if (l.f == 2) {  // CTAs striding over the elements (weights formed once per CTA)
        const unsigned gr2 = (unsigned)std::min<long long>(l.g.ne, dim == 2 ? 152 * 16 * 4 : 152 * 3 * 8);
        if (dim == 2)
          galerkin2_kernel<2><<<gr2, 64, 0, s>>>(fl.g, l.g, fl.K, i == 1 ? E32 : nullptr, K0d, fl.mask, l.mask, l.K,
                                                 nullptr, nullptr);
        else
          galerkin2_kernel<3><<<gr2, 576, 0, s>>>(fl.g, l.g, fl.K, i == 1 ? E32 : nullptr, K0d, fl.mask, l.mask, l.K,
                                                  nullptr, nullptr);
      } else if (dim == 2)
        galerkin_kernel<2><<<(unsigned)l.g.ne, 64, 0, s>>>(fl.g, l.g, l.f, fl.K, i == 1 ? E32 : nullptr, K0d, fl.mask,
                                                            l.mask, l.K);
      else
        galerkin_kernel<3><<<(unsigned)l.g.ne, 576, 0, s>>>(fl.g, l.g, l.f, fl.K, i == 1 ? E32 : nullptr, K0d, fl.mask,
                                                             l.mask, l.K);
      nl += 2;
    }
    if (l.S) {
      if (dim == 2) {
        stencil_kernel<2><<<blocks(l.g.nn), 256, 0, s>>>(l.g, l.K, i == 0 ? E32 : nullptr, l.mask, l.S);
        diag_stencil_kernel<2><<<blocks(l.g.nn), 256, 0, s>>>(l.g, l.S, l.mask, l.invd);
      } else {
        stencil_kernel<3><<<blocks(l.g.nn), 256, 0, s>>>(l.g, l.K, i == 0 ? E32 : nullptr, l.mask, l.S);
        diag_stencil_kernel<3><<<blocks(l.g.nn), 256, 0, s>>>(l.g, l.S, l.mask, l.invd);
      }
      nl += 2;
    } else {
      if (dim == 2) diag_kernel<2><<<blocks(l.g.nn), 256, 0, s>>>(l.g, l.K, i == 0 ? E32 : nullptr, l.mask, l.invd);
      else if (i == 0) diag_assembled_kernel<<<blocks(l.g.nn), 256, 0, s>>>(l.g, E32, l.mask, l.invd);
      else diag_kernel<3><<<blocks(l.g.nn), 256, 0, s>>>(l.g, l.K, nullptr, l.mask, l.invd);
      nl++;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  // coarsest: dense FP32 inverse on the device (blocked Gauss-Jordan sweep)
  const MgLevel& c = lv.back();
  e = dinv.create();
  if (e == cudaSuccess) e = dense_coarse_inverse(s, dinv, c.g, c.S, c.mask, cinv, dscratch, dflag, &nl);
  int flag = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, dflag, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (nlaunch) *nlaunch += nl;
  if (e != cudaSuccess) return e;
  coarse_ok = flag == 0;
  built = true;
  return cudaSuccess;
}

// One V-cycle on level li (see mg.h for the entry state).  Sweeps alternate
// between x[0] and x[1]; with nu sweeps before and after, the result lands in
// a buffer fixed by nu, which *out names.
cudaError_t MgHierarchy::vcycle(cudaStream_t s, int li, int* nlaunch, const int* stop, float** out) {
  MgLevel& l = lv[li];
  const int dim = l.g.dim;
  const long long ndof = l.g.nn * dim;
  if (li == (int)lv.size() - 1) {
    dense_solve_kernel<<<(cn + 7) / 8, 256, 0, s>>>(cn, nc, cinv, l.b, l.x[0], stop);
    (*nlaunch)++;
    *out = l.x[0];
    return cudaGetLastError();
  }
  auto sweep = [&](const float* u, const float* w, float* y, int mode, float a, float c, float om,
                   int dots = -1) -> cudaError_t {
    const bool tm = capture_events && li == 0 && ev_used + 2 <= (int)sweep_ev.size();
    if (tm) cudaEventRecordWithFlags(sweep_ev[ev_used], s, cudaEventRecordExternal);
    cudaError_t e;
    if (li == 0) {
      e = fine_op_fn(fine_ctx, s, u, w, l.b, l.invd, y, mode, a, c, om, stop, dots);
    } else {
      dim3 grid(blocks(l.g.nn), nc);
      if (dim == 2)
        apply_stencil_kernel<2><<<grid, 256, 0, s>>>(l.g, l.S, l.mask, l.invd, u, w, l.b, y, mode, a, c, om, stop);
      else if (l.g.nn <= kWarpNodes)
        apply_stencil_group_kernel<8><<<dim3(blocks(l.g.nn * 8), nc), 256, 0, s>>>(l.g, l.S, l.mask, l.invd, u, w, l.b,
                                                                                 y, mode, a, c, om, stop);
      else
        apply_stencil_kernel<3><<<grid, 256, 0, s>>>(l.g, l.S, l.mask, l.invd, u, w, l.b, y, mode, a, c, om, stop);
      e = cudaGetLastError();
    }
    if (tm) {
      cudaEventRecordWithFlags(sweep_ev[ev_used + 1], s, cudaEventRecordExternal);
      ev_used += 2;
    }
    (*nlaunch)++;
    return e;
  };
  // pre-smoothing from zero: x[0] already holds step 1, omega D^-1 b; step k
  // needs x_{k-2}, which is 0 for k = 2
  int cur = 0;
  const int nuL = degree_at(li);
  for (int k = 2; k <= nuL; k++) {
    cudaError_t e = sweep(l.x[cur], k == 2 ? nullptr : l.x[cur ^ 1], l.x[cur ^ 1], 1, ca[k], cc[k], cw[k]);
    if (e != cudaSuccess) return e;
    cur ^= 1;
  }
  cudaError_t e = sweep(l.x[cur], nullptr, l.t, 2, 0.f, 0.f, 0.f);  // residual
  if (e != cudaSuccess) return e;
  MgLevel& c = lv[li + 1];
  const bool coarsest = li + 1 == (int)lv.size() - 1;
  float* cx0 = coarsest ? nullptr : c.x[0];  // the dense solve needs no first sweep
  if (c.f == 4 && dim == 3 && c.r4 && c.g.ny <= 65535 && l.g.nz * nc <= 65535 && c.g.nz * nc <= 65535) {
    restrict4_xy_kernel<<<dim3((c.g.nx + kT2X - 1) / kT2X, c.g.ny, l.g.nz * nc), kT2X, 0, s>>>(l.g, c.g, l.mask, l.t,
                                                                                              c.r4, stop);
    restrict4_z_kernel<<<dim3((c.g.nx + kT2X - 1) / kT2X, c.g.ny, c.g.nz * nc), kT2X, 0, s>>>(l.g, c.g, c.r4, c.mask,
                                                                                             c.b, cx0, c.invd, omega,
                                                                                             stop);
    (*nlaunch)++;  // the second pass (the restriction's launch is counted below)
  } else if (c.f == 2 && dim == 3 && c.g.nn > kWarpRestrictNodes && c.g.ny <= 65535 && c.g.nz * nc <= 65535) {
    dim3 gr((c.g.nx + kT2X - 1) / kT2X, c.g.ny, c.g.nz * nc);
    restrict2x_kernel<<<gr, kT2X, 0, s>>>(l.g, c.g, l.mask, c.mask, l.t, c.b, cx0, c.invd, omega, stop);
  } else if (c.f == 2 && !(dim == 3 && c.g.nn <= kWarpNodes)) {
    dim3 gr(blocks(c.g.nn), nc);
    if (dim == 2) restrict2_kernel<2><<<gr, 256, 0, s>>>(l.g, c.g, l.mask, c.mask, l.t, c.b, cx0, c.invd, omega, stop);
    else restrict2_kernel<3><<<gr, 256, 0, s>>>(l.g, c.g, l.mask, c.mask, l.t, c.b, cx0, c.invd, omega, stop);
  } else {
    dim3 gr(blocks(c.g.nn * 32), nc);
    if (dim == 2)
      restrict_kernel<2><<<gr, 256, 0, s>>>(l.g, c.g, c.f, l.mask, c.mask, l.t, c.b, cx0, c.invd, omega, stop);
    else
      restrict_kernel<3><<<gr, 256, 0, s>>>(l.g, c.g, c.f, l.mask, c.mask, l.t, c.b, cx0, c.invd, omega, stop);
  }
  (*nlaunch)++;
  float* xc = nullptr;
  e = vcycle(s, li + 1, nlaunch, stop, &xc);
  if (e != cudaSuccess) return e;
  dim3 gp(blocks(l.g.nn), nc);
  const dim3 gx((l.g.nx + kT2X - 1) / kT2X, l.g.ny, l.g.nz * nc);
  if (dim == 3 && c.f == 2 && l.g.ny <= 65535 && l.g.nz * nc <= 65535)
    prolongfx_kernel<2><<<gx, kT2X, 0, s>>>(l.g, c.g, l.mask, xc, l.x[cur], stop);
  else if (dim == 3 && c.f == 4 && l.g.ny <= 65535 && l.g.nz * nc <= 65535)
    prolongfx_kernel<4><<<gx, kT2X, 0, s>>>(l.g, c.g, l.mask, xc, l.x[cur], stop);
  else if (dim == 2) prolong_kernel<2><<<gp, 256, 0, s>>>(l.g, c.g, c.f, l.mask, xc, l.x[cur], stop);
  else prolong_kernel<3><<<gp, 256, 0, s>>>(l.g, c.g, c.f, l.mask, xc, l.x[cur], stop);
  (*nlaunch)++;
  // post-smoothing with the same polynomial from the corrected iterate
  for (int k = 1; k <= nuL; k++) {
    const int dots = li == 0 && k == nuL ? fine_dots : -1;  // the step that produces z
    e = k == 1 ? sweep(l.x[cur], nullptr, l.x[cur ^ 1], 1, 1.f, 0.f, omega, dots)
               : sweep(l.x[cur], l.x[cur ^ 1], l.x[cur ^ 1], 1, ca[k], cc[k], cw[k], dots);
    if (e != cudaSuccess) return e;
    cur ^= 1;
  }
  *out = l.x[cur];
  return cudaGetLastError();
}

}  // namespace tp

// ---------------------------------------------------------------------------
// FP64 outer-PCG vector kernels.
namespace tp {
namespace {

struct FF {
  double v[8];
};

// Per-case partial dot products: block (b, c) sums chunk b of case c;
// part[(c * nb + b) * 2 + k] for the two products k.
__global__ void dot2_kernel(long long n, const double* __restrict__ a1, const double* __restrict__ b1,
                            const double* __restrict__ a2, const double* __restrict__ b2, double* __restrict__ part) {
  __shared__ double sred[32 * 2];
  const int c = blockIdx.y, nb = gridDim.x;
  const long long base = (long long)c * n;
  double acc[2] = {0.0, 0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)nb * blockDim.x) {
    acc[0] = fma(a1[base + i], b1[base + i], acc[0]);
    if (a2) acc[1] = fma(a2[base + i], b2[base + i], acc[1]);
  }
  block_sum<2>(acc, sred);
  if (threadIdx.x < 2) part[((long long)c * nb + blockIdx.x) * 2 + threadIdx.x] = acc[threadIdx.x];
}

// Sums the partials (one warp per (case, product), fixed order) and forms the
// PCG scalars of each case.
__global__ void scalars_kernel(int nb, int nc, const double* __restrict__ part, int what, double* sc) {
  __shared__ double tot[16];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int pr = warp; pr < 2 * nc; pr += blockDim.x >> 5) {
    const int c = pr >> 1, k = pr & 1;
    double sum = 0.0;
    for (int b = lane; b < nb; b += 32) sum += part[((long long)c * nb + b) * 2 + k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) tot[pr] = sum;
  }
  __syncthreads();
  const int c = threadIdx.x;
  if (c >= 8) return;
  if (c >= nc) {
    sc[c] = sc[8 + c] = 0.0;
    return;
  }
  const double s1 = tot[2 * c], s2 = tot[2 * c + 1];
  if (what == 0) {  // alpha = rz / pq
    sc[24 + c] = s1;
    sc[c] = (s1 > 0.0 && isfinite(s1)) ? sc[16 + c] / s1 : 0.0;
  } else if (what == 1) {  // beta = rz_new / rz
    sc[8 + c] = sc[16 + c] != 0.0 ? s1 / sc[16 + c] : 0.0;
    sc[16 + c] = s1;
    sc[32 + c] = s2;
  } else {  // start
    sc[16 + c] = s1;
    sc[32 + c] = s2;
    sc[8 + c] = 0.0;
  }
}

__global__ void residual_abi_kernel(long long n, const double* __restrict__ f, const double* __restrict__ Ax,
                                    const uint8_t* __restrict__ mask, int dim, double* r) {
  const int c = blockIdx.y, nn = (int)n;
  const long long base = (long long)c * n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += gridDim.x * blockDim.x) {
    const int node = i / dim, comp = i - node * dim;
    r[base + i] = ((mask[node] >> comp) & 1) ? 0.0 : f[base + i] - Ax[base + i];
  }
}

// ---- graph-captured iteration ----------------------------------------------

__global__ void seg_init_kernel(MgCtl* ctl, int nc, double tol2, FF ff, int it_limit, int use64) {
  const int c = threadIdx.x;
  if (c < 8) {
    ctl->ff[c] = c < nc ? ff.v[c] : 0.0;
    ctl->rr_start[c] = 0.0;
  }
  if (c == 0) {
    ctl->tol2 = tol2;
    ctl->best = 0.0;
    ctl->it = 0;
    ctl->best_it = 0;
    ctl->it_limit = it_limit;
    ctl->stop = 0;
    ctl->reason = 0;
    ctl->use64 = use64;
    ctl->nc = nc;
    ctl->ticket = 0u;
  }
}

// r32 = (float) r, x0 = omega D^-1 r32 (blockIdx.y = case).
__global__ void prep_kernel(long long n, const double* __restrict__ r, float* __restrict__ r32, float* __restrict__ x0,
                            const float* __restrict__ invd, float omega) {
  const int nn = (int)n;
  const long long base = (long long)blockIdx.y * n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += gridDim.x * blockDim.x) {
    const float v = (float)r[base + i];
    r32[base + i] = v;
    x0[base + i] = omega * invd[i] * v;
  }
}

template <typename TB>
__device__ __forceinline__ double as_f64(TB v) {
  return (double)v;
}
// Per-thread partial sums: FP64 when either operand is FP64, else FP32 (a
// thread sums about ten products; the block and grid totals are FP64).
template <typename TA, typename TB>
using acc_t = typename std::conditional<sizeof(TA) == 8 || sizeof(TB) == 8, double, float>::type;

// Fused dot products and PCG scalars.  Block (b, c) sums chunk b of case c in
// FP64 and stores its partials; the last block to finish (ticket) sums every
// case's partials in a fixed order, so the result does not depend on the
// order in which blocks finish, and then does the scalar work (one thread per
// case) and, for what 1, the stopping rule of the segment.
template <typename TA, typename TB>
__global__ void dotscal_kernel(long long n, const TA* __restrict__ a1, const TB* __restrict__ b1,
                               const TA* __restrict__ a2, const TA* __restrict__ b2, double* part, MgCtl* ctl,
                               int what) {
  if (what != 2 && ctl->stop) return;  // uniform: the flag changes only in the last block of this kernel
  const int c = blockIdx.y, nb = gridDim.x;
  const long long base = (long long)c * n;
  using A = acc_t<TA, TB>;
  // four independent partial sums per thread; the loads of a pass are
  // predicated rather than left to a remainder loop, so every thread issues
  // all of them at once (a grid of 8 CTAs per SM covers the vector in one pass
  // of 128-bit loads)
  A t0[4] = {A(0), A(0), A(0), A(0)}, t1[4] = {A(0), A(0), A(0), A(0)};
  const int nn = (int)n, stride = nb * blockDim.x, i0 = blockIdx.x * blockDim.x + threadIdx.x;
  const bool sq = a2 != nullptr && (const void*)a2 == (const void*)a1 && b2 == a2;  // second product a1 . a1
  int done = 0;  // elements covered by the vector pass
  if constexpr (sizeof(TA) == 4 && sizeof(TB) == 4) {
    auto al = [](const void* p) { return ((uintptr_t)p & 15u) == 0; };
    if (al(a1 + base) && al(b1 + base) && (a2 == nullptr || sq || (al(a2 + base) && al(b2 + base)))) {
      const int n4 = nn >> 2;
      const float4* A1 = reinterpret_cast<const float4*>(a1 + base);
      const float4* B1 = reinterpret_cast<const float4*>(b1 + base);
      for (int i = i0; i < n4; i += 4 * stride) {
        float4 x[4], y[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
          const bool in = i + k * stride < n4;
          x[k] = in ? A1[i + k * stride] : make_float4(0.f, 0.f, 0.f, 0.f);
          y[k] = in ? B1[i + k * stride] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int k = 0; k < 4; k++)
          t0[k] = fmaf(x[k].w, y[k].w, fmaf(x[k].z, y[k].z, fmaf(x[k].y, y[k].y, fmaf(x[k].x, y[k].x, t0[k]))));
        if (sq) {
#pragma unroll
          for (int k = 0; k < 4; k++)
            t1[k] = fmaf(x[k].w, x[k].w, fmaf(x[k].z, x[k].z, fmaf(x[k].y, x[k].y, fmaf(x[k].x, x[k].x, t1[k]))));
        } else if (a2) {
          const float4* A2 = reinterpret_cast<const float4*>(a2 + base);
          const float4* B2 = reinterpret_cast<const float4*>(b2 + base);
#pragma unroll
          for (int k = 0; k < 4; k++) {
            const bool in = i + k * stride < n4;
            x[k] = in ? A2[i + k * stride] : make_float4(0.f, 0.f, 0.f, 0.f);
            y[k] = in ? B2[i + k * stride] : make_float4(0.f, 0.f, 0.f, 0.f);
          }
#pragma unroll
          for (int k = 0; k < 4; k++)
            t1[k] = fmaf(x[k].w, y[k].w, fmaf(x[k].z, y[k].z, fmaf(x[k].y, y[k].y, fmaf(x[k].x, y[k].x, t1[k]))));
        }
      }
      done = n4 << 2;
    }
  }
  for (int i = done + i0; i < nn; i += 4 * stride) {
    A x[4], y[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const bool in = i + k * stride < nn;
      x[k] = in ? (A)a1[base + i + k * stride] : A(0);
      y[k] = in ? (A)b1[base + i + k * stride] : A(0);
    }
#pragma unroll
    for (int k = 0; k < 4; k++) t0[k] = fma(x[k], y[k], t0[k]);
    if (sq) {
#pragma unroll
      for (int k = 0; k < 4; k++) t1[k] = fma(x[k], x[k], t1[k]);
    } else if (a2) {
#pragma unroll
      for (int k = 0; k < 4; k++) {
        const bool in = i + k * stride < nn;
        x[k] = in ? (A)a2[base + i + k * stride] : A(0);
        y[k] = in ? (A)b2[base + i + k * stride] : A(0);
      }
#pragma unroll
      for (int k = 0; k < 4; k++) t1[k] = fma(x[k], y[k], t1[k]);
    }
  }
  double acc[2] = {((double)t0[0] + (double)t0[1]) + ((double)t0[2] + (double)t0[3]),
                   ((double)t1[0] + (double)t1[1]) + ((double)t1[2] + (double)t1[3])};
  pcg_dots_complete(acc, part, ctl, what);
}

// x += alpha p, r -= alpha q, r32 = (float) r, x0 = omega D^-1 r32.
template <typename TQ>
__global__ void update_xr_kernel(long long n, const MgCtl* __restrict__ ctl, double* x, const double* __restrict__ p,
                                 double* r, const TQ* __restrict__ q, float* __restrict__ r32, float* __restrict__ x0,
                                 const float* __restrict__ invd, float omega) {
  if (ctl->stop) return;
  const int c = blockIdx.y, nn = (int)n;
  const double a = ctl->sc[c];
  const long long base = (long long)c * n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += gridDim.x * blockDim.x) {
    x[base + i] = fma(a, p[base + i], x[base + i]);
    const double rv = fma(-a, as_f64(q[base + i]), r[base + i]);
    r[base + i] = rv;
    const float v = (float)rv;
    r32[base + i] = v;
    x0[base + i] = omega * invd[i] * v;
  }
}

// FP32 inner iteration (correction d of the segment): d += alpha p,
// r -= alpha q, x0 = omega D^-1 r (r is the V-cycle's right-hand side).
__global__ void update32_kernel(long long n, const MgCtl* __restrict__ ctl, float* d, const float* __restrict__ p,
                                float* r, const float* __restrict__ q, float* __restrict__ x0,
                                const float* __restrict__ invd, float omega) {
  if (ctl->stop) return;
  const int c = blockIdx.y, nn = (int)n;
  const float a = (float)ctl->sc[c];
  const long long base = (long long)c * n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += gridDim.x * blockDim.x) {
    d[base + i] = fmaf(a, p[base + i], d[base + i]);
    const float v = fmaf(-a, q[base + i], r[base + i]);
    r[base + i] = v;
    x0[base + i] = omega * invd[i] * v;
  }
}

// p = z + beta p in FP32 (p = z when beta = 0).
__global__ void update_p32_kernel(long long n, const MgCtl* __restrict__ ctl, float* p, const float* __restrict__ z) {
  if (ctl->stop) return;
  const int c = blockIdx.y, nn = (int)n;
  const float b = (float)ctl->sc[8 + c];
  const long long base = (long long)c * n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += gridDim.x * blockDim.x)
    p[base + i] = b != 0.f ? fmaf(b, p[base + i], z[base + i]) : z[base + i];
}

// x += (double) d (end of an FP32 segment).
__global__ void merge_kernel(long long n, double* x, const float* __restrict__ d) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] += (double)d[i];
}

// p = z + beta p (p = z at a segment start, beta = 0), p32 = (float) p.
__global__ void update_p_kernel(long long n, const MgCtl* __restrict__ ctl, double* p, float* __restrict__ p32,
                                const float* __restrict__ z) {
  if (ctl->stop) return;
  const int c = blockIdx.y, nn = (int)n;
  const double b = ctl->sc[8 + c];
  const long long base = (long long)c * n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += gridDim.x * blockDim.x) {
    const double v = b != 0.0 ? fma(b, p[base + i], (double)z[base + i]) : (double)z[base + i];
    p[base + i] = v;
    p32[base + i] = (float)v;
  }
}

int vblocks(long long n) { return (int)std::min<long long>(std::max<long long>((n + 255) / 256, 1), 152 * 8); }

}  // namespace

cudaError_t pcg_dot2(cudaStream_t s, long long n, int nc, const double* a1, const double* b1, const double* a2,
                     const double* b2, double* part, int* nblocks) {
  // up to 8 CTAs of 256 threads per SM (all cases together), each thread
  // summing at least 8 products
  const int nb = (int)std::min<long long>(std::max<long long>((n + 2047) / 2048, 1), 8 * 152 / nc);
  dot2_kernel<<<dim3(nb, nc), 256, 0, s>>>(n, a1, b1, a2, b2, part);
  *nblocks = nb;
  return cudaGetLastError();
}
cudaError_t pcg_scalars(cudaStream_t s, int nblocks, int nc, const double* part, int what, double* sc) {
  scalars_kernel<<<1, 512, 0, s>>>(nblocks, nc, part, what, sc);
  return cudaGetLastError();
}
cudaError_t pcg_residual(cudaStream_t s, long long n, int nc, const double* f, const double* Ax, const uint8_t* mask,
                         int dim, double* r) {
  residual_abi_kernel<<<dim3(vblocks(n), nc), 256, 0, s>>>(n, f, Ax, mask, dim, r);
  return cudaGetLastError();
}
cudaError_t mg_seg_init(cudaStream_t s, MgCtl* ctl, int nc, double tol2, const double* ff, int it_limit, int use64) {
  FF f{};
  for (int c = 0; c < nc && c < 8; c++) f.v[c] = ff[c];
  seg_init_kernel<<<1, 32, 0, s>>>(ctl, nc, tol2, f, it_limit, use64);
  return cudaGetLastError();
}
cudaError_t mg_prep(cudaStream_t s, long long n, int nc, const double* r, float* r32, float* x0, const float* invd,
                    float omega) {
  prep_kernel<<<dim3(vblocks(n), nc), 256, 0, s>>>(n, r, r32, x0, invd, omega);
  return cudaGetLastError();
}
cudaError_t mg_dotscal(cudaStream_t s, long long n, int nc, const void* a1, bool a_f32, const void* b1, bool b1_f32,
                       const void* a2, const void* b2, double* part, MgCtl* ctl, int what, int* nblocks) {
  // the CTAs of 256 threads that are resident at once on the device (all
  // cases together), each thread summing at least 8 products
  static int resident[3] = {0, 0, 0};
  const int kind = a_f32 && b1_f32 ? 0 : (b1_f32 ? 1 : 2);
  if (!resident[kind]) {
    int dev = 0, nsm = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = kind == 0   ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dotscal_kernel<float, float>, 256, 0)
          : kind == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dotscal_kernel<double, float>, 256, 0)
                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dotscal_kernel<double, double>, 256, 0);
    if (e != cudaSuccess) return e;
    resident[kind] = std::max(nsm * per_sm, 1);
  }
  const int nb = (int)std::min<long long>(std::max<long long>((n + 2047) / 2048, 1), std::max(resident[kind] / nc, 1));
  const dim3 grid(nb, nc);
  if (a_f32 && b1_f32)
    dotscal_kernel<float, float><<<grid, 256, 0, s>>>(n, (const float*)a1, (const float*)b1, (const float*)a2,
                                                      (const float*)b2, part, ctl, what);
  else if (a_f32)
    return cudaErrorInvalidValue;
  else if (b1_f32)
    dotscal_kernel<double, float><<<grid, 256, 0, s>>>(n, (const double*)a1, (const float*)b1, (const double*)a2,
                                                       (const double*)b2, part, ctl, what);
  else
    dotscal_kernel<double, double><<<grid, 256, 0, s>>>(n, (const double*)a1, (const double*)b1, (const double*)a2,
                                                        (const double*)b2, part, ctl, what);
  if (nblocks) *nblocks = nb;
  return cudaGetLastError();
}
cudaError_t mg_update32(cudaStream_t s, long long n, int nc, MgCtl* ctl, float* d, const float* p, float* r,
                        const float* q, float* x0, const float* invd, float omega) {
  update32_kernel<<<dim3(vblocks(n), nc), 256, 0, s>>>(n, ctl, d, p, r, q, x0, invd, omega);
  return cudaGetLastError();
}
cudaError_t mg_update_p32(cudaStream_t s, long long n, int nc, MgCtl* ctl, float* p, const float* z) {
  update_p32_kernel<<<dim3(vblocks(n), nc), 256, 0, s>>>(n, ctl, p, z);
  return cudaGetLastError();
}
cudaError_t mg_merge(cudaStream_t s, long long n, double* x, const float* d) {
  merge_kernel<<<vblocks(n), 256, 0, s>>>(n, x, d);
  return cudaGetLastError();
}
cudaError_t mg_update_xr(cudaStream_t s, long long n, int nc, MgCtl* ctl, double* x, const double* p, double* r,
                         const void* q, bool q_f32, float* r32, float* x0, const float* invd, float omega) {
  if (q_f32)
    update_xr_kernel<float><<<dim3(vblocks(n), nc), 256, 0, s>>>(n, ctl, x, p, r, (const float*)q, r32, x0, invd, omega);
  else
    update_xr_kernel<double><<<dim3(vblocks(n), nc), 256, 0, s>>>(n, ctl, x, p, r, (const double*)q, r32, x0, invd,
                                                                  omega);
  return cudaGetLastError();
}
cudaError_t mg_update_p(cudaStream_t s, long long n, int nc, MgCtl* ctl, double* p, float* p32, const float* z) {
  update_p_kernel<<<dim3(vblocks(n), nc), 256, 0, s>>>(n, ctl, p, p32, z);
  return cudaGetLastError();
}

}  // namespace tp
