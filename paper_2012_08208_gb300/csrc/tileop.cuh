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
//   TileOp<3,T>: 32 x 8 element columns streamed along z (256 threads), each
//     thread computing its element's eight corner forces once per layer; node
//     sums by registers (z), warp shuffles (x) and a shared exchange (y).
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

  // Input value v of the tile-local output node (tx, ty) as staged by the last
  // apply on this shared memory (valid until the next apply writes it).
  __device__ static T staged(const unsigned char* smem, int v, int tx, int ty) {
    return reinterpret_cast<const T*>(smem)[v * (HX * HY) + (ty + 1) * HX + tx + 1];
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
// H8: element columns streamed along z.
//
// A tile is 32 x 8 element columns (one thread each: lane = x, warp = y),
// elements ex = x0 - 1 + lane, ey = y0 - 1 + warp, and owns the 31 x 7 node
// columns x0 <= x < x0 + 31, y0 <= y < y0 + 7 (thread (lane, warp) owns node
// (ex, ey) when lane >= 1 and warp >= 1) over the planes z0 <= z < z1.  Per
// element layer kz (between node planes kz and kz + 1) each thread
//   - reads the four new corners (plane kz + 1) from a double-buffered shared
//     plane; the four old corners are kept in registers from the previous layer;
//   - issues the global loads of plane kz + 2 before its element arithmetic and
//     stores them into the free plane buffer afterwards;
//   - computes its element's eight corner forces (strain form);
//   - sums, for its own node of plane kz, the lower corners of layer kz and the
//     upper corners of layer kz - 1 (kept in registers): its own column's by
//     addition, the x-neighbour's by a warp shuffle, the y-neighbours' through
//     one double-buffered shared exchange.
// One __syncthreads per layer.  The summation order of every node is fixed.
template <typename T>
struct TileOp<3, T> {
  static constexpr int THREADS = 256;
  static constexpr int LX = 32, LY = 8;          // element columns per tile
  static constexpr int OX = LX - 1, OY = LY - 1;  // owned node columns per tile
  static constexpr int PX = LX + 1, PY = LY + 1;  // nodes per staged plane
  static constexpr int PLANE = PX * PY;           // 297

  static __host__ TileMapG map(const Grid& g, int zlen) {
    TileMapG m;
    if (zlen < 1) zlen = 1;
    if (zlen > g.nz) zlen = g.nz;
    const int nzt = (g.nz + zlen - 1) / zlen;  // balance the z chunks
    m.zlen = (g.nz + nzt - 1) / nzt;
    m.tiles_x = (g.nx + OX - 1) / OX;
    m.tiles_y = (g.ny + OY - 1) / OY;
    m.tiles_z = (g.nz + m.zlen - 1) / m.zlen;
    m.ntiles = m.tiles_x * m.tiles_y * m.tiles_z;
    return m;
  }
  static __host__ __device__ constexpr size_t smem_bytes() {
    return (size_t)(2 * PLANE + 2 * THREADS) * sizeof(V4<T>);
  }
  static __host__ __device__ constexpr size_t smem_bytes(int) { return smem_bytes(); }

  __device__ static void origin(const Grid& g, const TileMapG& m, int t, int& x0, int& y0, int& z0, int& z1) {
    x0 = (t % m.tiles_x) * OX;
    y0 = ((t / m.tiles_x) % m.tiles_y) * OY;
    z0 = (t / (m.tiles_x * m.tiles_y)) * m.zlen;
    z1 = min(z0 + m.zlen, g.nz);
  }

  // Calls fn(node) for every output node of tile t, with the thread / node
  // assignment of apply1's output.
  template <class Fn>
  __device__ static void for_each_own(const Grid& g, const TileMapG& m, int t, Fn fn) {
    int x0, y0, z0, z1;
    origin(g, m, t, x0, y0, z0, z1);
    const int lane = threadIdx.x & 31, row = threadIdx.x >> 5;
    if (lane == 0 || row == 0) return;
    const int gx = x0 - 1 + lane, gy = y0 - 1 + row;
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
    apply1_pre(
        g, m, t, E, C, smem, load, [](long long) { return 0; },
        [&](long long node, const T(&y)[3], const T(&us)[3], int) { emit(node, y, us); });
  }

  // The same with a pre-load: pre(node) is called for this thread's output
  // node of plane kz before the element arithmetic of that layer, and its
  // result reaches emit(node, y, us, pre_result), so the global loads the
  // emitter needs (a right-hand side, a scale, the fixed bits) overlap the
  // arithmetic instead of following the barrier.
  template <class Load, class Pre, class Emit>
  __device__ static void apply1_pre(const Grid& g, const TileMapG& m, int t, const T* __restrict__ E,
                                    const CMat<3, T>& C, unsigned char* smem, Load load, Pre pre, Emit emit) {
    V4<T>* P = reinterpret_cast<V4<T>*>(smem);  // [2][PY][PX] staged node planes
    V4<T>* X = P + 2 * PLANE;                   // [2][LY][LX] y-exchange of corner sums
    int x0, y0, z0, z1;
    origin(g, m, t, x0, y0, z0, z1);
    const int tid = threadIdx.x, lane = tid & 31, row = tid >> 5;
    const int ex = x0 - 1 + lane, ey = y0 - 1 + row;
    const bool col_ok = ex >= 0 && ex < g.ex && ey >= 0 && ey < g.ey;
    const bool owner = lane >= 1 && row >= 1 && ex < g.nx && ey < g.ny;
    const long long nplane = (long long)g.nx * g.ny;
    // Staging: every thread loads its own column's node (plane slot (row, lane));
    // threads 0..40 also load one of the 41 nodes of the last plane row and
    // column (never owned by the tile).
    const bool main_ok = ex >= 0 && ex < g.nx && ey >= 0 && ey < g.ny;
    const long long main_off = main_ok ? ex + (long long)g.nx * ey : 0;
    const int xs_slot = tid < PX ? (PY - 1) * PX + tid : (tid - PX) * PX + PX - 1;
    const int xs_x = tid < PX ? x0 - 1 + tid : x0 + LX - 1;
    const int xs_y = tid < PX ? y0 + LY - 1 : y0 - 1 + (tid - PX);
    const bool has_xs = tid < PX + LY;
    const bool xs_ok = has_xs && xs_x >= 0 && xs_x < g.nx && xs_y >= 0 && xs_y < g.ny;
    const long long xs_off = xs_ok ? xs_x + (long long)g.nx * xs_y : 0;

    auto prefetch = [&](int kz, T (&v)[6]) {
      const bool zin = kz >= 0 && kz < g.nz;
      const bool own = owner && kz >= z0 && kz < z1;
#pragma unroll
      for (int r = 0; r < 3; r++) v[r] = (zin && main_ok) ? load(main_off + nplane * kz, r, own) : T(0);
#pragma unroll
      for (int r = 0; r < 3; r++) v[3 + r] = (zin && xs_ok) ? load(xs_off + nplane * kz, r, false) : T(0);
    };
    auto stage = [&](V4<T>* dst, const T (&v)[6]) {
      dst[row * PX + lane] = V4<T>{v[0], v[1], v[2], T(0)};
      if (has_xs) dst[xs_slot] = V4<T>{v[3], v[4], v[5], T(0)};
    };
    auto corners = [&](const V4<T>* pl, T (&u)[4][3]) {
#pragma unroll
      for (int c = 0; c < 4; c++) {
        const V4<T> v = pl[(row + cofs(c, 1)) * PX + lane + cofs(c, 0)];
        u[c][0] = v.x;
        u[c][1] = v.y;
        u[c][2] = v.z;
      }
    };
    auto modulus = [&](int kz) -> T {
      return (col_ok && kz >= 0 && kz < g.ez) ? __ldg(E + ex + (long long)g.ex * (ey + (long long)g.ey * kz)) : T(-1);
    };

    {
      T v[6];
      prefetch(z0 - 1, v);
      stage(P + ((z0 - 1) & 1) * PLANE, v);
      prefetch(z0, v);
      stage(P + (z0 & 1) * PLANE, v);
    }
    __syncthreads();
    T uo[4][3], fu[4][3];
    corners(P + ((z0 - 1) & 1) * PLANE, uo);
    __syncthreads();  // the first layer restages this buffer
#pragma unroll
    for (int c = 0; c < 4; c++) fu[c][0] = fu[c][1] = fu[c][2] = T(0);
    T Ee = modulus(z0 - 1);  // < 0: no element in this column at this layer

    for (int kz = z0 - 1; kz < z1; kz++) {
      T un[4][3];
      corners(P + ((kz + 1) & 1) * PLANE, un);
      T pf[6];
      const bool more = kz + 2 <= z1;  // plane kz + 2 is needed by the next layer
      if (more) prefetch(kz + 2, pf);
      const T Enext = modulus(kz + 1);
      const bool emits = kz >= z0 && owner;
      const auto pd = pre(emits ? main_off + nplane * kz : -1LL);
      T f[8][3];
      if (Ee >= T(0)) {
        T u[8][3];
#pragma unroll
        for (int c = 0; c < 4; c++)
#pragma unroll
          for (int r = 0; r < 3; r++) {
            u[c][r] = uo[c][r];
            u[c + 4][r] = un[c][r];
          }
        h8_element_forces(u, Ee, C, f);
      } else {
#pragma unroll
        for (int c = 0; c < 8; c++) f[c][0] = f[c][1] = f[c][2] = T(0);
      }
      // corner sums for plane kz: s_c = lower corner c of layer kz + upper corner c of layer kz - 1
      T a[3], b[3];
#pragma unroll
      for (int r = 0; r < 3; r++) {
        const T s0 = f[0][r] + fu[0][r], s1 = f[1][r] + fu[1][r];
        const T s2 = f[2][r] + fu[2][r], s3 = f[3][r] + fu[3][r];
        a[r] = s0 + __shfl_up_sync(0xffffffffu, s1, 1);  // node (ex, ey): elements ex and ex - 1
        b[r] = s3 + __shfl_up_sync(0xffffffffu, s2, 1);  // node (ex, ey + 1) from this row
      }
      X[(kz & 1) * THREADS + tid] = V4<T>{b[0], b[1], b[2], T(0)};
      if (more) stage(P + (kz & 1) * PLANE, pf);
      __syncthreads();
      if (emits) {
        const V4<T> w = X[(kz & 1) * THREADS + tid - 32];
        T y[3] = {a[0] + w.x, a[1] + w.y, a[2] + w.z};
        T us[3] = {uo[0][0], uo[0][1], uo[0][2]};
        emit(main_off + nplane * kz, y, us, pd);
      }
#pragma unroll
      for (int c = 0; c < 4; c++)
#pragma unroll
        for (int r = 0; r < 3; r++) {
          uo[c][r] = un[c][r];
          fu[c][r] = f[c + 4][r];
        }
      Ee = Enext;
    }
    __syncthreads();
  }
};

}  // namespace tp
