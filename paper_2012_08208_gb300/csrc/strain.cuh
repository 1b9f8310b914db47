// Element operator in generalised-strain form: K0 u_e = G^T C G u_e.
//
// G u_e are Walsh sums over the element corners of each displacement
// component, evaluated difference-first (every term is an edge difference
// u(corner) - u(corner - e_d)), so a rigid translation contributes exactly
// zero in any precision; the shear rows pair x- and y-edge differences term by
// term, so an infinitesimal rotation cancels exactly too.  C is the small
// block-diagonal matrix from the host (element_strain_C), and G^T is applied
// as an inverse Walsh butterfly.  Per element this is ~200 FP operations
// instead of the 576 FMAs of a dense 24 x 24 product (H8), and FP32 rounding
// stays relative to the strains rather than to the displacements.
#pragma once
#include "common.cuh"

namespace tp {

// Offset (0 or 1) of element corner c along `axis`; corner order (0,0),(1,0),
// (1,1),(0,1) at z = 0, then the same at z = 1.
__host__ __device__ constexpr int cofs(int c, int axis) {
  return axis == 0 ? (((c & 3) == 1 || (c & 3) == 2) ? 1 : 0)
                   : (axis == 1 ? (((c & 3) >= 2) ? 1 : 0) : (c >= 4 ? 1 : 0));
}

template <int DIM, typename T>
struct CMat {
  T k[DIM == 2 ? 25 : 324];
};

// ---------------------------------------------------------------------------
// Q4.  Corner order (0,0),(1,0),(1,1),(0,1).
// g = [a_x(10), a_y(01), a_x(01)+a_y(10), a_x(11), a_y(11)].

template <typename T>
__device__ __forceinline__ void q4_strain(const T (&ux)[4], const T (&uy)[4], T (&g)[5]) {
  const T dxb_x = ux[1] - ux[0], dxt_x = ux[2] - ux[3], dyl_x = ux[3] - ux[0], dyr_x = ux[2] - ux[1];
  const T dxb_y = uy[1] - uy[0], dxt_y = uy[2] - uy[3], dyl_y = uy[3] - uy[0], dyr_y = uy[2] - uy[1];
  g[0] = dxb_x + dxt_x;
  g[1] = dyl_y + dyr_y;
  g[2] = (dyl_x + dxb_y) + (dyr_x + dxt_y);
  g[3] = dxt_x - dxb_x;
  g[4] = dxt_y - dxb_y;
}

// sigma = E * C g (block structure: {0,1}, {2}, {3}, {4})
template <typename T>
__device__ __forceinline__ void q4_stress(const T (&g)[5], T E, const CMat<2, T>& C, T (&s)[5]) {
  s[0] = E * fma(C.k[0], g[0], C.k[1] * g[1]);
  s[1] = E * fma(C.k[5], g[0], C.k[6] * g[1]);
  s[2] = E * (C.k[12] * g[2]);
  s[3] = E * (C.k[18] * g[3]);
  s[4] = E * (C.k[24] * g[4]);
}

// Force at one corner (compile-time) from the element stresses: rows of G^T.
template <int CORNER, typename T>
__device__ __forceinline__ void q4_corner_force(const T (&s)[5], T& fx, T& fy) {
  constexpr int cx = (CORNER == 1 || CORNER == 2) ? 1 : 0;
  constexpr int cy = CORNER >= 2 ? 1 : 0;
  constexpr T sx = cx ? T(1) : T(-1), sy = cy ? T(1) : T(-1);
  fx = sx * s[0] + sy * s[2] + (sx * sy) * s[3];
  fy = sy * s[1] + sx * s[2] + (sx * sy) * s[4];
}

// ---------------------------------------------------------------------------
// H8.  Corner c has offsets (cofs(c,0), cofs(c,1), cofs(c,2)); u[c][comp].

__host__ __device__ constexpr int h8_corner(int x, int y, int z) {
  // inverse of cofs: (0,0)->0, (1,0)->1, (1,1)->2, (0,1)->3, +4 for z
  return (y == 0 ? (x == 0 ? 0 : 1) : (x == 0 ? 3 : 2)) + 4 * z;
}

// Walsh coefficient a(mode) of one component, mode bits (A,B,Cz), computed as a
// sum of edge differences along the first axis whose bit is set.
template <int A, int B, int Cz, typename T>
__device__ __forceinline__ T h8_walsh(const T (&u)[8][3], int comp) {
  constexpr int d = A ? 0 : (B ? 1 : 2);
  T acc = T(0);
  bool first = true;
#pragma unroll
  for (int j = 0; j < 4; j++) {
    // the two coordinates other than d
    int p = j & 1, q = (j >> 1) & 1;
    int x, y, z;
    if (d == 0) { x = 1; y = p; z = q; }
    else if (d == 1) { x = p; y = 1; z = q; }
    else { x = p; y = q; z = 1; }
    const int hi = h8_corner(x, y, z);
    const int lo = h8_corner(d == 0 ? 0 : x, d == 1 ? 0 : y, d == 2 ? 0 : z);
    int sgn = 1;
    if (d != 0 && A && x == 0) sgn = -sgn;
    if (d != 1 && B && y == 0) sgn = -sgn;
    if (d != 2 && Cz && z == 0) sgn = -sgn;
    const T diff = u[hi][comp] - u[lo][comp];
    if (first) { acc = sgn > 0 ? diff : -diff; first = false; }
    else acc = sgn > 0 ? acc + diff : acc - diff;
  }
  return acc;
}

// Shear row a_i(mode_i) + a_j(mode_j): the four edge differences of each term
// are paired one to one before summing (an infinitesimal rotation gives pairs
// that cancel exactly).
template <int Ai, int Bi, int Ci, int Aj, int Bj, int Cj, typename T>
__device__ __forceinline__ T h8_shear(const T (&u)[8][3], int ci, int cj) {
  constexpr int di = Ai ? 0 : (Bi ? 1 : 2);
  constexpr int dj = Aj ? 0 : (Bj ? 1 : 2);
  T acc = T(0);
#pragma unroll
  for (int j = 0; j < 4; j++) {
    int p = j & 1, q = (j >> 1) & 1;
    int xi, yi, zi, xj, yj, zj;
    if (di == 0) { xi = 1; yi = p; zi = q; } else if (di == 1) { xi = p; yi = 1; zi = q; } else { xi = p; yi = q; zi = 1; }
    if (dj == 0) { xj = 1; yj = p; zj = q; } else if (dj == 1) { xj = p; yj = 1; zj = q; } else { xj = p; yj = q; zj = 1; }
    const T a = u[h8_corner(xi, yi, zi)][ci] -
                u[h8_corner(di == 0 ? 0 : xi, di == 1 ? 0 : yi, di == 2 ? 0 : zi)][ci];
    const T b = u[h8_corner(xj, yj, zj)][cj] -
                u[h8_corner(dj == 0 ? 0 : xj, dj == 1 ? 0 : yj, dj == 2 ? 0 : zj)][cj];
    acc = j == 0 ? (a + b) : acc + (a + b);
  }
  return acc;
}

template <typename T>
__device__ __forceinline__ void h8_strain(const T (&u)[8][3], T (&g)[18]) {
  g[0] = h8_walsh<1, 0, 0>(u, 0);
  g[1] = h8_walsh<0, 1, 0>(u, 1);
  g[2] = h8_walsh<0, 0, 1>(u, 2);
  g[3] = h8_shear<0, 1, 0, 1, 0, 0>(u, 0, 1);
  g[4] = h8_walsh<1, 1, 1>(u, 2);
  g[5] = h8_shear<0, 0, 1, 1, 0, 0>(u, 0, 2);
  g[6] = h8_walsh<1, 1, 1>(u, 1);
  g[7] = h8_shear<0, 0, 1, 0, 1, 0>(u, 1, 2);
  g[8] = h8_walsh<1, 1, 1>(u, 0);
  g[9] = h8_walsh<1, 1, 0>(u, 1);
  g[10] = h8_walsh<1, 0, 1>(u, 2);
  g[11] = h8_walsh<1, 1, 0>(u, 0);
  g[12] = h8_walsh<0, 1, 1>(u, 2);
  g[13] = h8_walsh<1, 0, 1>(u, 0);
  g[14] = h8_walsh<0, 1, 1>(u, 1);
  g[15] = h8_walsh<0, 1, 1>(u, 0);
  g[16] = h8_walsh<1, 0, 1>(u, 1);
  g[17] = h8_walsh<1, 1, 0>(u, 2);
}

// sigma = C g restricted to the diagonal blocks {0..2}, {3,4}, {5,6}, {7,8},
// {9,10}, {11,12}, {13,14}, {15..17}.  Each block is its own instantiation, so
// every index is a compile-time constant for any value type (a runtime index
// would move g into local memory).
template <int START, int SIZE, typename T>
__device__ __forceinline__ void h8_stress_block(const T (&g)[18], const CMat<3, T>& C, T (&s)[18]) {
#pragma unroll
  for (int i = 0; i < SIZE; i++) {
    const int r = START + i;
    T acc = C.k[r * 18 + START] * g[START];
#pragma unroll
    for (int j = 1; j < SIZE; j++) acc = fma(C.k[r * 18 + START + j], g[START + j], acc);
    s[r] = acc;
  }
}
template <typename T>
__device__ __forceinline__ void h8_stress(const T (&g)[18], const CMat<3, T>& C, T (&s)[18]) {
  h8_stress_block<0, 3>(g, C, s);
  h8_stress_block<3, 2>(g, C, s);
  h8_stress_block<5, 2>(g, C, s);
  h8_stress_block<7, 2>(g, C, s);
  h8_stress_block<9, 2>(g, C, s);
  h8_stress_block<11, 2>(g, C, s);
  h8_stress_block<13, 2>(g, C, s);
  h8_stress_block<15, 3>(g, C, s);
}

// Inverse Walsh of one component: F[mode], mode = a + 2b + 4c, F[0] = 0;
// f(corner) = sum_mode F[mode] s_x^a s_y^b s_z^c.
template <typename T>
__device__ __forceinline__ void h8_inverse(const T (&F)[8], T (&f)[8]) {
  T Gz[2][2][2];  // [a][b][z]
#pragma unroll
  for (int a = 0; a < 2; a++)
#pragma unroll
    for (int b = 0; b < 2; b++) {
      const T f0 = F[a + 2 * b], f1 = F[a + 2 * b + 4];
      Gz[a][b][0] = f0 - f1;
      Gz[a][b][1] = f0 + f1;
    }
  T H[2][2][2];  // [a][y][z]
#pragma unroll
  for (int a = 0; a < 2; a++)
#pragma unroll
    for (int z = 0; z < 2; z++) {
      H[a][0][z] = Gz[a][0][z] - Gz[a][1][z];
      H[a][1][z] = Gz[a][0][z] + Gz[a][1][z];
    }
#pragma unroll
  for (int y = 0; y < 2; y++)
#pragma unroll
    for (int z = 0; z < 2; z++) {
      f[h8_corner(0, y, z)] = H[0][y][z] - H[1][y][z];
      f[h8_corner(1, y, z)] = H[0][y][z] + H[1][y][z];
    }
}

// Corner forces f[c][comp] = E * (G^T C G u)[c][comp].
template <typename T>
__device__ __forceinline__ void h8_element_forces(const T (&u)[8][3], T E, const CMat<3, T>& C,
                                                  T (&f)[8][3]) {
  T g[18];
  h8_strain(u, g);
#pragma unroll
  for (int i = 0; i < 18; i++) g[i] *= E;
  T s[18];
  h8_stress(g, C, s);
  // scatter stresses to per-component Walsh coefficients (mode = a + 2b + 4c)
  T Fx[8], Fy[8], Fz[8];
#pragma unroll
  for (int m = 0; m < 8; m++) Fx[m] = Fy[m] = Fz[m] = T(0);
  Fx[1] = s[0];                 // x(100)
  Fy[2] = s[1];                 // y(010)
  Fz[4] = s[2];                 // z(001)
  Fx[2] = s[3]; Fy[1] = s[3];   // x(010) + y(100)
  Fz[7] = s[4];                 // z(111)
  Fx[4] = s[5]; Fz[1] = s[5];   // x(001) + z(100)
  Fy[7] = s[6];                 // y(111)
  Fy[4] = s[7]; Fz[2] = s[7];   // y(001) + z(010)
  Fx[7] = s[8];                 // x(111)
  Fy[3] = s[9];                 // y(110)
  Fz[5] = s[10];                // z(101)
  Fx[3] = s[11];                // x(110)
  Fz[6] = s[12];                // z(011)
  Fx[5] = s[13];                // x(101)
  Fy[6] = s[14];                // y(011)
  Fx[6] = s[15];                // x(011)
  Fy[5] = s[16];                // y(101)
  Fz[3] = s[17];                // z(110)
  T fx[8], fy[8], fz[8];
  h8_inverse(Fx, fx);
  h8_inverse(Fy, fy);
  h8_inverse(Fz, fz);
#pragma unroll
  for (int c = 0; c < 8; c++) {
    f[c][0] = fx[c];
    f[c][1] = fy[c];
    f[c][2] = fz[c];
  }
}

// Element energy u^T K0 u = g^T C g (unit modulus).
template <typename T>
__device__ __forceinline__ T h8_energy(const T (&u)[8][3], const CMat<3, T>& C) {
  T g[18], s[18];
  h8_strain(u, g);
  h8_stress(g, C, s);
  T e = T(0);
#pragma unroll
  for (int i = 0; i < 18; i++) e = fma(g[i], s[i], e);
  return e;
}

template <typename T>
__device__ __forceinline__ T q4_energy(const T (&ux)[4], const T (&uy)[4], const CMat<2, T>& C) {
  T g[5], s[5];
  q4_strain(ux, uy, g);
  q4_stress(g, T(1), C, s);
  T e = T(0);
#pragma unroll
  for (int i = 0; i < 5; i++) e = fma(g[i], s[i], e);
  return e;
}

}  // namespace tp
