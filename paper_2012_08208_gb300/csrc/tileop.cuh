// Tile operators: apply y = sum_e E_e K0 u_e over one tile of output nodes.
//
// Both operators read their input through a functor load(node, v, own), v =
// case * DIM + component (masking, or forming p = z + beta p_old on the fly, is
// the caller's business) and hand every output node to
// emit(node, case, y[DIM], u_self[DIM]).  Each output
// node is owned by exactly one tile; elements on tile borders are recomputed by
// the neighbouring tile, so there are no atomics and the summation order of
// every node is fixed (bitwise deterministic results).
//
//   TileOp<2,T>: 32 x 16 node tile, two nodes per thread (256 threads), all load
//     cases in one pass.  Each node evaluates the strains of its four elements
//     from a shared-memory halo tile and sums its own corner forces.
//   TileOp<3,T>: 32 x 8 node columns x zlen planes, 320 threads, streamed along z.
//     Per element layer the 33 x 9 elements touching the columns compute all
//     eight corner forces once (element-centric); each node then sums the lower
//     corners of layer k and the upper corners of layer k-1 in a fixed order.
//     Node planes live in a three-plane ring in shared memory.
#pragma once
#include "strain.cuh"

namespace tp {

template <typename T>
struct V4 {
  T x, y, z, w;
};

struct TileMapG {
  int tiles_x, tiles_y, tiles_z, ntiles, zlen;
};

template <int DIM, typename T>
struct TileOp;

// ---------------------------------------------------------------------------
template <typename T, int TY_ = 16>
struct Q4Tile {
  static constexpr int THREADS = 256;
  static constexpr int TX = 32, TY = TY_, HX = TX + 2, HY = TY + 2, EX = TX + 1, EY = TY + 1;
  static constexpr int NPT = TX * TY / THREADS;  // output nodes per thread

  static __host__ TileMapG map(const Grid& g, int /*zlen*/) {
    TileMapG m;
    m.tiles_x = (g.nx + TX - 1) / TX;
    m.tiles_y = (g.ny + TY - 1) / TY;
    m.tiles_z = 1;
    m.ntiles = m.tiles_x * m.tiles_y;
    m.zlen = 1;
    return m;
  }
  // shared memory for up to NCM load cases
  static __host__ __device__ constexpr size_t smem_bytes(int ncm = 1) {
    return (size_t)(HX * HY * 2 * ncm + EX * EY) * sizeof(T);
  }

  // Calls fn(node) for every output node of tile t, with the thread / node
  // assignment of apply (the thread that emitted a node visits it).
  template <class Fn>
  __device__ static void for_each_own(const Grid& g, const TileMapG& m, int t, Fn fn) {
    const int x0 = (t % m.tiles_x) * TX, y0 = (t / m.tiles_x) * TY;
#pragma unroll
    for (int k = 0; k < (NPT > 0 ? NPT : 1); k++) {
      const int ln = threadIdx.x + k * THREADS;
      if (ln >= TX * TY) break;
      const int gx = x0 + ln % TX, gy = y0 + ln / TX;
      if (gx < g.nx && gy < g.ny) fn(gx + (long long)g.nx * gy);
    }
  }

  // All `nc` cases of the tile in one pass: load(node, v, own) supplies value v
  // (v = case * 2 + comp) of a node; emit(node, case, y[2], u_self[2]).
  template <int NCM, class Load, class Emit>
  __device__ static void apply(const Grid& g, const TileMapG& m, int t, const T* __restrict__ E,
                               const CMat<2, T>& C, unsigned char* smem, int nc, Load load, Emit emit) {
    const int nv = 2 * nc;
    T* sU = reinterpret_cast<T*>(smem);  // [nv][HY][HX]
    T* sE = sU + HX * HY * nv;           // [EY][EX]
    const int x0 = (t % m.tiles_x) * TX, y0 = (t / m.tiles_x) * TY;
    for (int i = threadIdx.x; i < EX * EY; i += blockDim.x) {
      const int ex = x0 - 1 + i % EX, ey = y0 - 1 + i / EX;
      sE[i] = (ex >= 0 && ex < g.ex && ey >= 0 && ey < g.ey) ? __ldg(E + ex + (long long)g.ex * ey) : T(0);
    }
    // planar halo [v][HY][HX]: consecutive threads load consecutive nodes of a row
    const int total = HX * HY * nv;
#pragma unroll 8
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
      const int v = i / (HX * HY), hn = i - v * (HX * HY);
      const int hx = hn % HX, hy = hn / HX;
      const int gx = x0 - 1 + hx, gy = y0 - 1 + hy;
      T val = T(0);
      if (gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny) {
        const bool own = hx >= 1 && hx <= TX && hy >= 1 && hy <= TY;
        val = load(gx + (long long)g.nx * gy, v, own);
      }
      sU[i] = val;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < (NPT > 0 ? NPT : 1); k++) {
      const int ln = threadIdx.x + k * THREADS;
      if (ln >= TX * TY) break;
      const int tx = ln % TX, ty = ln / TX;
      const int gx = x0 + tx, gy = y0 + ty;
      if (gx >= g.nx || gy >= g.ny) continue;
      const long long node = gx + (long long)g.nx * gy;
      for (int cs = 0; cs < nc; cs++) {
        T yx = T(0), yy = T(0);
        // element in which this node is corner c: tile coords (tx+1-cx, ty+1-cy)
        auto elem = [&](auto cc) {
          constexpr int c = decltype(cc)::value;
          constexpr int cx = (c == 1 || c == 2) ? 1 : 0, cy = c >= 2 ? 1 : 0;
          const int ex = tx + 1 - cx, ey = ty + 1 - cy;
          const T Ee = sE[ey * EX + ex];
          T ux[4], uy[4];
#pragma unroll
          for (int q = 0; q < 4; q++) {
            const int qx = (q == 1 || q == 2) ? 1 : 0, qy = q >= 2 ? 1 : 0;
            const T* p = sU + (2 * cs) * (HX * HY) + (ey + qy) * HX + ex + qx;
            ux[q] = p[0];
            uy[q] = p[HX * HY];
          }
          T gg[5], sg[5];
          q4_strain(ux, uy, gg);
          q4_stress(gg, Ee, C, sg);
          T fx, fy;
          q4_corner_force<c>(sg, fx, fy);
          yx += fx;
          yy += fy;
        };
        elem(std::integral_constant<int, 0>());
        elem(std::integral_constant<int, 1>());
        elem(std::integral_constant<int, 2>());
        elem(std::integral_constant<int, 3>());
        const T* ps = sU + (2 * cs) * (HX * HY) + (ty + 1) * HX + tx + 1;
        T y[2] = {yx, yy};
        T us[2] = {ps[0], ps[HX * HY]};
        emit(node, cs, y, us);
      }
    }
    __syncthreads();
  }
};

template <typename T>
struct TileOp<2, T> : Q4Tile<T, 16> {};

// ---------------------------------------------------------------------------
template <typename T>
struct TileOp<3, T> {
  static constexpr int THREADS = 320;
  static constexpr int TX = 32, TY = 8, HX = TX + 2, HY = TY + 2, EX = TX + 1, EY = TY + 1;
  static constexpr int NEL = EX * EY;  // 297 elements per layer
  static constexpr int PLANE = HX * HY;

  static __host__ TileMapG map(const Grid& g, int zlen) {
    TileMapG m;
    if (zlen < 1) zlen = 1;
    if (zlen > g.nz) zlen = g.nz;
    m.tiles_x = (g.nx + TX - 1) / TX;
    m.tiles_y = (g.ny + TY - 1) / TY;
    m.tiles_z = (g.nz + zlen - 1) / zlen;
    m.ntiles = m.tiles_x * m.tiles_y * m.tiles_z;
    m.zlen = zlen;
    return m;
  }
  static __host__ __device__ constexpr size_t smem_bytes() {
    return (size_t)(3 * PLANE + 3 * 4 * NEL) * sizeof(V4<T>);
  }

  static __host__ __device__ constexpr size_t smem_bytes(int) { return smem_bytes(); }

  // Calls fn(node) for every output node of tile t, with the thread / node
  // assignment of the node phase of apply1.
  template <class Fn>
  __device__ static void for_each_own(const Grid& g, const TileMapG& m, int t, Fn fn) {
    const int x0 = (t % m.tiles_x) * TX;
    const int y0 = ((t / m.tiles_x) % m.tiles_y) * TY;
    const int z0 = (t / (m.tiles_x * m.tiles_y)) * m.zlen;
    const int z1 = min(z0 + m.zlen, g.nz);
    if (threadIdx.x >= TX * TY) return;
    const int gx = x0 + threadIdx.x % TX, gy = y0 + threadIdx.x / TX;
    if (gx >= g.nx || gy >= g.ny) return;
    for (int kz = z0; kz < z1; kz++) fn(gx + (long long)g.nx * (gy + (long long)g.ny * kz));
  }

  // All `nc` cases, one streaming pass per case: load(node, v, own) with
  // v = case * 3 + comp; emit(node, case, y[3], u_self[3]).
  template <int NCM, class Load, class Emit>
  __device__ static void apply(const Grid& g, const TileMapG& m, int t, const T* __restrict__ E,
                               const CMat<3, T>& C, unsigned char* smem, int nc, Load load, Emit emit) {
    for (int cs = 0; cs < nc; cs++)
      apply1(
          g, m, t, E, C, smem, [&](long long node, int comp, bool own) -> T { return load(node, cs * 3 + comp, own); },
          [&](long long node, const T(&y)[3], const T(&us)[3]) { emit(node, cs, y, us); });
  }

  template <class Load, class Emit>
  __device__ static void apply1(const Grid& g, const TileMapG& m, int t, const T* __restrict__ E,
                                const CMat<3, T>& C, unsigned char* smem, Load load, Emit emit) {
    V4<T>* ring = reinterpret_cast<V4<T>*>(smem);  // [3][HY][HX]
    V4<T>* flo = ring + 3 * PLANE;                 // [4][NEL]   lower corners, current layer
    V4<T>* fhi = flo + 4 * NEL;                    // [2][4][NEL] upper corners, by layer parity
    const int x0 = (t % m.tiles_x) * TX;
    const int y0 = ((t / m.tiles_x) % m.tiles_y) * TY;
    const int z0 = (t / (m.tiles_x * m.tiles_y)) * m.zlen;
    const int z1 = min(z0 + m.zlen, g.nz);  // owned planes [z0, z1)
    const int tid = threadIdx.x;

    auto slot = [](int kz) { return ((kz % 3) + 3) % 3; };
    auto load_plane = [&](int kz) {
      T* dst = reinterpret_cast<T*>(ring + slot(kz) * PLANE);
      for (int i = tid; i < PLANE * 3; i += blockDim.x) {
        const int comp = i / PLANE, hn = i - comp * PLANE;
        const int hx = hn % HX, hy = hn / HX;
        const int gx = x0 - 1 + hx, gy = y0 - 1 + hy;
        T v = T(0);
        if (kz >= 0 && kz < g.nz && gx >= 0 && gx < g.nx && gy >= 0 && gy < g.ny) {
          const bool own = hx >= 1 && hx <= TX && hy >= 1 && hy <= TY && kz >= z0 && kz < z1;
          v = load(gx + (long long)g.nx * (gy + (long long)g.ny * kz), comp, own);
        }
        dst[hn * 4 + comp] = v;
      }
    };

    load_plane(z0 - 1);
    for (int kz = z0 - 1; kz < z1; kz++) {  // element layer kz spans node planes kz, kz+1
      load_plane(kz + 1);
      __syncthreads();
      if (tid < NEL) {
        const int ex_t = tid % EX, ey_t = tid / EX;
        const int gex = x0 - 1 + ex_t, gey = y0 - 1 + ey_t;
        V4<T> out[8];
        const bool valid = gex >= 0 && gex < g.ex && gey >= 0 && gey < g.ey && kz >= 0 && kz < g.ez;
        if (valid) {
          const T Ee = __ldg(E + gex + (long long)g.ex * (gey + (long long)g.ey * kz));
          T u[8][3];
#pragma unroll
          for (int c = 0; c < 8; c++) {
            const int cx = cofs(c, 0), cy = cofs(c, 1), cz = cofs(c, 2);
            const V4<T> v = ring[slot(kz + cz) * PLANE + (ey_t + cy) * HX + ex_t + cx];
            u[c][0] = v.x;
            u[c][1] = v.y;
            u[c][2] = v.z;
          }
          T f[8][3];
          h8_element_forces(u, Ee, C, f);
#pragma unroll
          for (int c = 0; c < 8; c++) out[c] = V4<T>{f[c][0], f[c][1], f[c][2], T(0)};
        } else {
#pragma unroll
          for (int c = 0; c < 8; c++) out[c] = V4<T>{T(0), T(0), T(0), T(0)};
        }
#pragma unroll
        for (int c = 0; c < 4; c++) {
          flo[c * NEL + tid] = out[c];
          fhi[((kz & 1) * 4 + c) * NEL + tid] = out[4 + c];
        }
      }
      __syncthreads();
      if (kz >= z0 && tid < TX * TY) {
        const int tx = tid % TX, ty = tid / TX;
        const int gx = x0 + tx, gy = y0 + ty;
        if (gx < g.nx && gy < g.ny) {
          T y[3] = {T(0), T(0), T(0)};
          const int prev = (kz - 1) & 1;
#pragma unroll
          for (int c = 0; c < 4; c++) {  // node is corner c (lower) of layer kz, corner c+4 of layer kz-1
            const int ex_t = tx + 1 - cofs(c, 0), ey_t = ty + 1 - cofs(c, 1);
            const int e = ey_t * EX + ex_t;
            const V4<T> a = flo[c * NEL + e];
            const V4<T> b = fhi[(prev * 4 + c) * NEL + e];
            y[0] += a.x + b.x;
            y[1] += a.y + b.y;
            y[2] += a.z + b.z;
          }
          const V4<T> s = ring[slot(kz) * PLANE + (ty + 1) * HX + tx + 1];
          T us[3] = {s.x, s.y, s.z};
          emit(gx + (long long)g.nx * (gy + (long long)g.ny * kz), y, us);
        }
      }
    }
    __syncthreads();
  }
};

}  // namespace tp
