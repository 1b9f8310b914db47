// Node-tile machinery shared by the operator, CG and sensitivity kernels:
// element-corner geometry, tile maps, shared-memory tile loaders and the
// per-node application of the element stiffness.
#pragma once
#include "host.h"

namespace tp {

// ---------------------------------------------------------------------------
// Geometry of an element's corners and of the node tiles.

__host__ __device__ constexpr int cofs(int c, int axis) {
  return axis == 0 ? (((c & 3) == 1 || (c & 3) == 2) ? 1 : 0)
                   : (axis == 1 ? (((c & 3) >= 2) ? 1 : 0) : (c >= 4 ? 1 : 0));
}

template <int DIM>
struct TileGeom {
  static constexpr int NCORN = DIM == 2 ? 4 : 8;
  static constexpr int ND = DIM * NCORN;
  static constexpr int TX = 32;
  static constexpr int TY = DIM == 2 ? 8 : 4;
  static constexpr int TZ = DIM == 2 ? 1 : 4;
  static constexpr int HX = TX + 2, HY = TY + 2, HZ = DIM == 3 ? TZ + 2 : 1;
  static constexpr int EX = TX + 1, EY = TY + 1, EZ = DIM == 3 ? TZ + 1 : 1;
  static constexpr int HN = HX * HY * HZ;
  static constexpr int EN = EX * EY * EZ;
  static constexpr int TN = TX * TY * TZ;
};

template <int DIM, typename T>
struct KMat {
  T k[TileGeom<DIM>::ND * TileGeom<DIM>::ND];
};

template <int DIM>
struct TileMap {
  int tiles_x, tiles_y, tiles_z, ntiles;
};


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

template <int DIM>
static TileMap<DIM> tile_map(const Grid& g) {
  using G = TileGeom<DIM>;
  TileMap<DIM> m;
  m.tiles_x = (g.nx + G::TX - 1) / G::TX;
  m.tiles_y = (g.ny + G::TY - 1) / G::TY;
  m.tiles_z = DIM == 3 ? (g.nz + G::TZ - 1) / G::TZ : 1;
  m.ntiles = m.tiles_x * m.tiles_y * m.tiles_z;
  return m;
}

template <int DIM>
__device__ __forceinline__ void tile_origin(const TileMap<DIM>& m, int t, int& x0, int& y0, int& z0) {
  using G = TileGeom<DIM>;
  x0 = (t % m.tiles_x) * G::TX;
  y0 = ((t / m.tiles_x) % m.tiles_y) * G::TY;
  z0 = (t / (m.tiles_x * m.tiles_y)) * G::TZ;
}

// Moduli of the (TX+1)(TY+1)(TZ+1) elements touching a node tile; 0 outside the mesh.
template <int DIM, typename T>
__device__ __forceinline__ void load_E(const Grid& g, int x0, int y0, int z0, const T* __restrict__ E,
                                       T* sE) {
  using G = TileGeom<DIM>;
  for (int i = threadIdx.x; i < G::EN; i += blockDim.x) {
    const int ex = i % G::EX, ey = (i / G::EX) % G::EY, ez = i / (G::EX * G::EY);
    const int gx = x0 - 1 + ex, gy = y0 - 1 + ey, gz = DIM == 3 ? z0 - 1 + ez : 0;
    T v = T(0);
    if (gx >= 0 && gx < g.ex && gy >= 0 && gy < g.ey && gz >= 0 && gz < g.ez)
      v = __ldg(E + gx + (long long)g.ex * (gy + (long long)g.ey * gz));
    sE[i] = v;
  }
}

// Node values of the tile plus a one-node halo; fn(node, v, own) supplies the
// value of component v (case-major inside the node) of an in-mesh node.
template <int DIM, typename T, typename F>
__device__ __forceinline__ void load_halo(const Grid& g, int x0, int y0, int z0, int nv, T* sP, F fn) {
  using G = TileGeom<DIM>;
  const int total = G::HN * nv;
  for (int i = threadIdx.x; i < total; i += blockDim.x) {
    const int hn = i / nv, v = i - hn * nv;
    const int hx = hn % G::HX, hy = (hn / G::HX) % G::HY, hz = hn / (G::HX * G::HY);
    const int gx = x0 - 1 + hx, gy = y0 - 1 + hy, gz = DIM == 3 ? z0 - 1 + hz : 0;
    T val = T(0);
    if (gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny && gz >= 0 && gz < g.nz) {
      const bool own = hx >= 1 && hx <= G::TX && hy >= 1 && hy <= G::TY &&
                       (DIM == 2 || (hz >= 1 && hz <= G::TZ));
      const long long node = gx + (long long)g.nx * (gy + (long long)g.ny * gz);
      val = fn(node, v, own);
    }
    sP[i] = val;
  }
}

// (K u) at one node for one load case: sum over the elements that share the
// node of E_e * (rows of K0 belonging to the node's corner) * u_e.
template <int DIM, typename T, typename KT>
__device__ __forceinline__ void node_apply(const T* sP, const T* sE, int nv, int cs, int tx, int ty,
                                           int tz, const KT& K, T (&acc)[DIM]) {
  using G = TileGeom<DIM>;
#pragma unroll
  for (int r = 0; r < DIM; r++) acc[r] = T(0);
#pragma unroll
  for (int cn = 0; cn < G::NCORN; cn++) {
    const int ex = tx + 1 - cofs(cn, 0), ey = ty + 1 - cofs(cn, 1);
    const int ez = DIM == 3 ? tz + 1 - cofs(cn, 2) : 0;
    const T Ee = sE[(ez * G::EY + ey) * G::EX + ex];
    T t[DIM];
#pragma unroll
    for (int r = 0; r < DIM; r++) t[r] = T(0);
#pragma unroll
    for (int m = 0; m < G::NCORN; m++) {
      const int hx = ex + cofs(m, 0), hy = ey + cofs(m, 1), hz = DIM == 3 ? ez + cofs(m, 2) : 0;
      const T* pu = sP + ((hz * G::HY + hy) * G::HX + hx) * nv + cs * DIM;
#pragma unroll
      for (int s = 0; s < DIM; s++) {
        const T us = pu[s];
#pragma unroll
        for (int r = 0; r < DIM; r++) t[r] = fma(K.k[(DIM * cn + r) * G::ND + DIM * m + s], us, t[r]);
      }
    }
#pragma unroll
    for (int r = 0; r < DIM; r++) acc[r] = fma(Ee, t[r], acc[r]);
  }
}

template <int DIM>
__device__ __forceinline__ bool own_node(const Grid& g, int ln, int x0, int y0, int z0, int& tx,
                                         int& ty, int& tz, long long& node) {
  using G = TileGeom<DIM>;
  tx = ln % G::TX;
  ty = (ln / G::TX) % G::TY;
  tz = ln / (G::TX * G::TY);
  const int gx = x0 + tx, gy = y0 + ty, gz = DIM == 3 ? z0 + tz : 0;
  if (gx >= g.nx || gy >= g.ny || gz >= g.nz) return false;
  node = gx + (long long)g.nx * (gy + (long long)g.ny * gz);
  return true;
}

template <int DIM, typename T>
inline void fill_k(KMat<DIM, T>& km, const double* K0) {
  constexpr int n = TileGeom<DIM>::ND * TileGeom<DIM>::ND;
  for (int i = 0; i < n; i++) km.k[i] = (T)K0[i];
}

inline int grid_for(long long n, int threads = 256) {
  long long b = (n + threads - 1) / threads;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace tp
