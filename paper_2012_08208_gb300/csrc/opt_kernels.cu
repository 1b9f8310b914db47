// Optimisation-side kernels of the GB300 SIMP library:
//   * the mesh-independency filter of Section 3.2.2 (Eq. "filter",
//     "filter_cond"; matrix form Eq. "filter_mat") as a shared-memory-staged
//     stencil over the structured grid (W_ab = max(0, rmin - |x_a - x_b|) is a
//     fixed set of taps; the dense distance matrix of Section 4.5 is never formed)
//   * the optimality-criteria update with a multi-point bisection on the
//     Lagrange multiplier (Eq. "update", Section 3.2.1), one cooperative launch.
#include <cmath>

#include "pcg_common.cuh"

namespace tp {

// ---------------------------------------------------------------------------
// Filter.

template <int DIM>
struct FTile {
  static constexpr int TX = 32;
  static constexpr int TY = DIM == 2 ? 8 : 4;
  static constexpr int TZ = DIM == 2 ? 1 : 2;
  static constexpr int TN = TX * TY * TZ;
};

struct FilterArgs {
  Grid g;
  int ntaps;
  int R;  // stencil radius (max |offset| per axis)
  int tiles_x, tiles_y, tiles_z;
  int mode;
  const double* rho;
  const double* dc;
  double* out;
  double wsum;  // sum of all weights in tap order: the row sum of an element whose taps all lie inside
  int off[3 * kMaxTaps];
  double w[kMaxTaps];
};

// mode 0 (sensitivity filter): out_a = sum_b W_ab rho_b dc_b / (rho_a sum_b W_ab)
// mode 1 (density filter):     out_a = sum_b W_ab rho_b / sum_b W_ab
// mode 2 (its chain rule):     out_a = sum_b W_ab dc_b / rowsum_b  (W symmetric;
//                              `rho` carries rowsum)
// mode 3 (row sums):           out_a = sum_b W_ab
// Elements outside the mesh carry no weight (rows truncated at the boundary).
template <int DIM>
__global__ void __launch_bounds__(256) filter_kernel(const __grid_constant__ FilterArgs a) {
  using F = FTile<DIM>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sG = reinterpret_cast<double*>(smem_raw);
  const int R = a.R;
  const int SX = F::TX + 2 * R, SY = F::TY + 2 * R, SZ = DIM == 3 ? F::TZ + 2 * R : 1;
  const int t = blockIdx.x;
  const int x0 = (t % a.tiles_x) * F::TX;
  const int y0 = ((t / a.tiles_x) % a.tiles_y) * F::TY;
  const int z0 = (t / (a.tiles_x * a.tiles_y)) * F::TZ;
  const Grid& g = a.g;
  const int total = SX * SY * SZ;
  for (int i = threadIdx.x; i < total; i += blockDim.x) {
    const int sx = i % SX, sy = (i / SX) % SY, sz = i / (SX * SY);
    const int gx = x0 - R + sx, gy = y0 - R + sy, gz = DIM == 3 ? z0 - R + sz : 0;
    double v = 0.0;
    if (gx >= 0 && gx < g.ex && gy >= 0 && gy < g.ey && gz >= 0 && gz < g.ez) {
      const long long e = gx + (long long)g.ex * (gy + (long long)g.ey * gz);
      v = a.mode == 0 ? a.rho[e] * a.dc[e] : (a.mode == 1 ? a.rho[e] : (a.mode == 2 ? a.dc[e] / a.rho[e] : 0.0));
    }
    sG[i] = v;
  }
  __syncthreads();
  for (int ln = threadIdx.x; ln < F::TN; ln += blockDim.x) {
    const int tx = ln % F::TX, ty = (ln / F::TX) % F::TY, tz = ln / (F::TX * F::TY);
    const int gx = x0 + tx, gy = y0 + ty, gz = DIM == 3 ? z0 + tz : 0;
    if (gx >= g.ex || gy >= g.ey || gz >= g.ez) continue;
    double num = 0.0, den = 0.0;
    const bool inside = gx >= R && gx + R < g.ex && gy >= R && gy + R < g.ey &&
                        (DIM == 2 || (gz >= R && gz + R < g.ez));
    if (inside) {  // every tap lies in the mesh: the row sum is the precomputed total (same order)
      for (int k = 0; k < a.ntaps; k++) {
        const int dx = a.off[3 * k], dy = a.off[3 * k + 1], dz = a.off[3 * k + 2];
        const int sidx = ((DIM == 3 ? tz + R + dz : 0) * SY + (ty + R + dy)) * SX + (tx + R + dx);
        num = fma(a.w[k], sG[sidx], num);
      }
      den = a.wsum;
    } else {
      for (int k = 0; k < a.ntaps; k++) {
        const int dx = a.off[3 * k], dy = a.off[3 * k + 1], dz = a.off[3 * k + 2];
        const int nx = gx + dx, ny = gy + dy, nz = gz + dz;
        if (nx < 0 || nx >= g.ex || ny < 0 || ny >= g.ey || nz < 0 || nz >= g.ez) continue;
        const int sidx = ((DIM == 3 ? tz + R + dz : 0) * SY + (ty + R + dy)) * SX + (tx + R + dx);
        num = fma(a.w[k], sG[sidx], num);
        den += a.w[k];
      }
    }
    const long long e = gx + (long long)g.ex * (gy + (long long)g.ey * gz);
    a.out[e] = a.mode == 0 ? num / (a.rho[e] * den) : (a.mode == 1 ? num / den : (a.mode == 2 ? num : den));
  }
}

cudaError_t launch_filter(cudaStream_t s, const FilterLaunch& Fl, int mode, const double* rho,
                          const double* dc, double* out) {
  FilterArgs a;
  a.g = Fl.g;
  a.ntaps = Fl.ntaps;
  int R = 0;
  for (int k = 0; k < Fl.ntaps; k++) {
    for (int d = 0; d < 3; d++) {
      a.off[3 * k + d] = Fl.off[3 * k + d];
      const int m = Fl.off[3 * k + d] < 0 ? -Fl.off[3 * k + d] : Fl.off[3 * k + d];
      if (m > R) R = m;
    }
    a.w[k] = Fl.w[k];
  }
  a.wsum = 0.0;
  for (int k = 0; k < Fl.ntaps; k++) a.wsum += Fl.w[k];
  a.R = R;
  a.mode = mode;
  a.rho = rho;
  a.dc = dc;
  a.out = out;
  size_t smem;
  if (Fl.g.dim == 2) {
    using F = FTile<2>;
    a.tiles_x = (Fl.g.ex + F::TX - 1) / F::TX;
    a.tiles_y = (Fl.g.ey + F::TY - 1) / F::TY;
    a.tiles_z = 1;
    smem = (size_t)(F::TX + 2 * R) * (F::TY + 2 * R) * sizeof(double);
  } else {
    using F = FTile<3>;
    a.tiles_x = (Fl.g.ex + F::TX - 1) / F::TX;
    a.tiles_y = (Fl.g.ey + F::TY - 1) / F::TY;
    a.tiles_z = (Fl.g.ez + F::TZ - 1) / F::TZ;
    smem = (size_t)(F::TX + 2 * R) * (F::TY + 2 * R) * (F::TZ + 2 * R) * sizeof(double);
  }
  const int ntiles = a.tiles_x * a.tiles_y * a.tiles_z;
  auto kern = Fl.g.dim == 2 ? filter_kernel<2> : filter_kernel<3>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  kern<<<ntiles, 256, smem, s>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// OC update (Eq. "update"): rho_new(lambda) per element, lambda from the
// volume constraint by a 16-way bisection.
//
// V(lambda) = sum_e rho_new_e(lambda) is non-increasing in lambda.  A pass
// evaluates V at 15 interior points of the bracket [l1, l2] in one sweep over
// the elements (B_e = rho_e sqrt(max(-dc~_e, 0)) precomputed, candidate
// B_e / sqrt(lambda_j)) and keeps the sub-interval where V - target changes
// sign: points with V - target > 0 move l1 up, the first point with
// V - target <= 0 becomes l2 (the paper's rule, Section 4.4 code).  A first
// pass widens the bracket: l2 = 1e9 * 10^j for the first j with V <= target.
// Passive elements are held at dmin inside the search.
//
// GB300 issues an FP64 operation at 1/64 of the FP32 rate, so the passes run
// in FP32 (double-float totals) until the bracket is 1e-5 wide relative to
// lambda (well above the FP32 evaluation error of V even when few elements are
// interior).  One FP64 pass then classifies every element at both ends of the
// bracket, widened by 4e-5: clamped high at both, clamped low at both, or
// interior at both.  If none changes state inside the bracket, V there is
// exactly C + A / sqrt(lambda) (C the clamped values, A the sum of B_e over the
// interior elements) and the root is lambda* = (A / (target - C))^2, checked
// against V at both ends in FP64.  If a few elements (at most kOcList) change
// state inside the bracket, their breakpoints (B_e / hi_e)^2 and
// (B_e / lo_e)^2 split it into pieces on each of which V has that form; the
// piece where V - target changes sign gives the exact root.  Otherwise FP64
// passes continue from the bracket (from scratch if V does not change sign
// across it) until l2 - l1 <= 1e-10 (l1 + l2), and the final update uses the
// midpoint.

constexpr int kOcK = 15;
constexpr int kOcList = 32;

// Exact root on [c1, c2] given the totals over the elements that keep their
// state (C: clamped values, A: sum of B_e of interior ones) and the m <=
// kOcList elements that change state, list[3 k .. 3 k + 2] = (B, lo, hi).
// One thread.  The elements and then the breakpoints are sorted, so the result
// does not depend on the order in which the list was filled.  Returns 0 if no
// piece brackets the root (the caller falls back to bisection).
__device__ double oc_piecewise_root(const double* list, int m, double c1, double c2, double C, double A,
                                    double target) {
  double e[kOcList][3];
  for (int k = 0; k < m; k++)
    for (int q = 0; q < 3; q++) e[k][q] = __ldcg(list + 3 * k + q);
  for (int k = 1; k < m; k++)  // insertion sort by (B, lo, hi)
    for (int j = k; j > 0; j--) {
      const bool gt = e[j - 1][0] > e[j][0] || (e[j - 1][0] == e[j][0] &&
                      (e[j - 1][1] > e[j][1] || (e[j - 1][1] == e[j][1] && e[j - 1][2] > e[j][2])));
      if (!gt) break;
      for (int q = 0; q < 3; q++) {
        const double t = e[j][q];
        e[j][q] = e[j - 1][q];
        e[j - 1][q] = t;
      }
    }
  // state at c1 and the breakpoints inside (c1, c2): kind 0 high -> interior,
  // kind 1 interior -> low (candidate B / sqrt(lambda) decreases with lambda)
  double tv[2 * kOcList];
  int tk[2 * kOcList], te[2 * kOcList], nt = 0;
  const double s1 = 1.0 / sqrt(c1);
  for (int k = 0; k < m; k++) {
    const double b = e[k][0], lo = e[k][1], hi = e[k][2], k1 = b * s1;
    if (k1 >= hi) C += hi;
    else if (k1 <= lo) C += lo;
    else A += b;
    const double la = (b / hi) * (b / hi), lb = (b / lo) * (b / lo);
    if (la > c1 && la < c2) { tv[nt] = la; tk[nt] = 0; te[nt++] = k; }
    if (lb > c1 && lb < c2) { tv[nt] = lb; tk[nt] = 1; te[nt++] = k; }
  }
  for (int k = 1; k < nt; k++)  // by value, ties by element then kind
    for (int j = k; j > 0; j--) {
      const bool gt = tv[j - 1] > tv[j] || (tv[j - 1] == tv[j] && (te[j - 1] > te[j] ||
                      (te[j - 1] == te[j] && tk[j - 1] > tk[j])));
      if (!gt) break;
      const double t = tv[j]; tv[j] = tv[j - 1]; tv[j - 1] = t;
      const int a1 = tk[j]; tk[j] = tk[j - 1]; tk[j - 1] = a1;
      const int a2 = te[j]; te[j] = te[j - 1]; te[j - 1] = a2;
    }
  double lo_end = c1;
  for (int i = 0; i <= nt; i++) {
    const double hi_end = i < nt ? tv[i] : c2;
    if (C + A / sqrt(hi_end) - target <= 0.0) {  // V crosses the target on [lo_end, hi_end]
      if (!(A > 0.0) || !(target > C)) return 0.0;
      const double rt = A / (target - C), lam = rt * rt;
      return (lam >= lo_end * (1.0 - 1e-12) && lam <= hi_end * (1.0 + 1e-12)) ? lam : 0.0;
    }
    if (i < nt) {
      const int k = te[i];
      if (tk[i] == 0) {
        C -= e[k][2];
        A += e[k][0];
      } else {
        A -= e[k][0];
        C += e[k][1];
      }
      lo_end = hi_end;
    }
  }
  return 0.0;
}

struct OcArgs {
  long long ne;
  const double* rho;
  const double* dcf;
  const int8_t* passive;
  double target, move, dmin;
  double* rho_new;
  double* B;
  double* part;
  GridBar* bar;
  OcStatus* st;
};

__device__ __forceinline__ double oc_clamp(double rho, double cand, double move, double dmin) {
  return fmax(dmin, fmax(rho - move, fmin(1.0, fmin(rho + move, cand))));
}

__global__ void __launch_bounds__(256) oc_kernel(const __grid_constant__ OcArgs a) {
  __shared__ double sRed[32 * kOcK];
  unsigned char* sm = reinterpret_cast<unsigned char*>(sRed);
  const int nb = gridDim.x;
  const long long stride = (long long)nb * blockDim.x;
  const long long first = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  unsigned gen = 0;
  bool ok = true;
  int passes = 0;
  // (B_e, rho_e) in FP32 during the search, in the memory of rho_new (written
  // last); B_e < 0 marks a passive element.  Every thread reads back only the
  // elements it wrote.
  float2* S2 = reinterpret_cast<float2*>(a.rho_new);
  double* list = a.part + (size_t)(2 * kOcK + 2) * nb + 1;
  unsigned* list_n = reinterpret_cast<unsigned*>(list - 1);
  if (blockIdx.x == 0 && threadIdx.x == 0) *list_n = 0u;  // read after at least one grid barrier
  for (long long e = first; e < a.ne; e += stride) {
    const double r = a.rho[e];
    const bool pas = a.passive != nullptr && a.passive[e] == 1;
    const double b = pas ? -1.0 : r * sqrt(fmax(-a.dcf[e], 0.0));
    a.B[e] = b;
    S2[e] = make_float2((float)b, (float)r);
  }

  // Search state.  Thread 0 takes every decision from the totals and
  // publishes it through shared memory; the 15 points of a pass (lambda_j,
  // 1 / sqrt(lambda_j) in FP64 and FP32) are formed once per CTA by 15 lanes.
  // Every CTA holds the same totals, so all take the same decisions.
  __shared__ double sh_l[2], sh_tot[kOcK], sh_lam[kOcK], sh_s[kOcK];
  __shared__ float sh_sf[kOcK];
  __shared__ int sh_state;
  auto set_points = [&](bool decades) {
    if (threadIdx.x < kOcK) {
      const int j = threadIdx.x;
      constexpr double p10[kOcK] = {1e0, 1e1, 1e2, 1e3, 1e4, 1e5, 1e6, 1e7, 1e8, 1e9, 1e10, 1e11, 1e12, 1e13, 1e14};
      const double l1 = sh_l[0], l2 = sh_l[1];
      const double lj = decades ? l2 * p10[j] : l1 + (l2 - l1) / (kOcK + 1) * (j + 1);
      sh_lam[j] = lj;
      sh_s[j] = 1.0 / sqrt(lj);
      sh_sf[j] = (float)sh_s[j];
    }
    __syncthreads();
  };
  // one pass: V at the points into sh_tot; partial sums alternate between
  // two slots so that the totals of pass k can be read while pass k+1 writes
  // its partials
  auto pass = [&](bool f32) -> bool {
    double* slot8 = a.part + (size_t)(passes & 1) * kOcK * nb;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (f32) {
      float2* slot = reinterpret_cast<float2*>(slot8);
      float sf[kOcK], acc[kOcK];
#pragma unroll
      for (int j = 0; j < kOcK; j++) {
        sf[j] = sh_sf[j];
        acc[j] = 0.f;
      }
      const float mv = (float)a.move, dm = (float)a.dmin;
      for (long long e = first; e < a.ne; e += stride) {
        const float2 v = S2[e];
        if (v.x < 0.f) {
#pragma unroll
          for (int j = 0; j < kOcK; j++) acc[j] += dm;
        } else {
          const float lo = fmaxf(dm, v.y - mv), hi = fminf(1.f, v.y + mv);
#pragma unroll
          for (int j = 0; j < kOcK; j++) acc[j] += fminf(hi, fmaxf(lo, v.x * sf[j]));
        }
      }
      block_partial_f<kOcK>(acc, slot, sm);
      if (!grid_sync(a.bar, gen)) return false;
      for (int i = warp; i < kOcK; i += nw) {  // double-float totals, fixed order
        dfl t{0.f, 0.f};
        for (int b = lane; b < nb; b += 32) {
          const float2 q = __ldcg(slot + (size_t)i * nb + b);
          t = dfl_add(t, dfl{q.x, q.y});
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
          t = dfl_add(t, dfl{__shfl_xor_sync(0xffffffffu, t.hi, o), __shfl_xor_sync(0xffffffffu, t.lo, o)});
        if (lane == 0) sh_tot[i] = (double)t.hi + (double)t.lo;
      }
    } else {
      double sd[kOcK], acc[kOcK];
#pragma unroll
      for (int j = 0; j < kOcK; j++) {
        sd[j] = sh_s[j];
        acc[j] = 0.0;
      }
      for (long long e = first; e < a.ne; e += stride) {
        const double r = a.rho[e], b = a.B[e];
#pragma unroll
        for (int j = 0; j < kOcK; j++) acc[j] += b < 0.0 ? a.dmin : oc_clamp(r, b * sd[j], a.move, a.dmin);
      }
      block_sum<kOcK>(acc, sRed);
      if (threadIdx.x == 0)
        for (int j = 0; j < kOcK; j++) slot8[(size_t)j * nb + blockIdx.x] = acc[j];
      if (!grid_sync(a.bar, gen)) return false;
      for (int i = warp; i < kOcK; i += nw) {
        double t = 0.0;
        for (int b = lane; b < nb; b += 32) t += __ldcg(slot8 + (size_t)i * nb + b);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) sh_tot[i] = t;
      }
    }
    __syncthreads();
    return true;
  };
  // widening pass(es) from l2 = 1e9; true when a bracket was found
  auto widen = [&](bool f32) -> bool {
    if (threadIdx.x == 0) {
      sh_l[0] = 0.0;
      sh_l[1] = 1e9;
    }
    __syncthreads();
    for (int round = 0; round < 20 && ok; round++) {
      set_points(true);
      ok = pass(f32);
      passes++;
      if (!ok) break;
      if (threadIdx.x == 0) {
        int jf = -1;
        for (int j = kOcK - 1; j >= 0; j--)
          if (sh_tot[j] - a.target <= 0.0) jf = j;
        if (jf >= 0) {
          if (jf > 0) sh_l[0] = sh_lam[jf - 1];
          sh_l[1] = sh_lam[jf];
          sh_state = 1;
        } else {
          sh_l[0] = sh_lam[kOcK - 1];
          sh_l[1] = sh_lam[kOcK - 1] * 10.0;
          sh_state = isfinite(sh_l[1]) ? 0 : -1;
        }
      }
      __syncthreads();
      const int st = sh_state;
      __syncthreads();
      if (st != 0) return st == 1;
    }
    return false;
  };
  // 16-way bisection until l2 - l1 <= rel (l1 + l2), or no progress
  auto bisect = [&](bool f32, double rel) {
    for (;;) {
      if (threadIdx.x == 0) sh_state = (sh_l[1] - sh_l[0]) > rel * (sh_l[0] + sh_l[1]) && passes < 200;
      __syncthreads();
      const int go = sh_state;
      __syncthreads();
      if (!go || !ok) break;
      set_points(false);
      ok = pass(f32);
      passes++;
      if (!ok) break;
      if (threadIdx.x == 0) {
        int jf = kOcK;
        for (int j = kOcK - 1; j >= 0; j--)
          if (sh_tot[j] - a.target <= 0.0) jf = j;
        const double nl1 = jf > 0 ? sh_lam[jf - 1] : sh_l[0];
        const double nl2 = jf < kOcK ? sh_lam[jf] : sh_l[1];
        sh_state = !(nl1 == sh_l[0] && nl2 == sh_l[1]);  // the bracket cannot shrink further in this precision
        sh_l[0] = nl1;
        sh_l[1] = nl2;
      }
      __syncthreads();
      const int moved = sh_state;
      __syncthreads();
      if (!moved) break;
    }
  };

  double lfinal = 0.0;
  bool found = widen(true), exact = false;
  int root = 0;
  if (found) {
    bisect(true, 1e-5);
    // certification of the FP32 bracket in FP64
    const double c1 = sh_l[0] * (1.0 - 4e-5), c2 = sh_l[1] * (1.0 + 4e-5);
    __shared__ double sh_s12[2];
    if (threadIdx.x == 0) {
      sh_s12[0] = c1 > 0.0 ? 1.0 / sqrt(c1) : 1e300;
      sh_s12[1] = 1.0 / sqrt(c2);
    }
    __syncthreads();
    const double s1 = sh_s12[0], s2 = sh_s12[1];
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};  // V(c1), V(c2), A, C, changing
    for (long long e = first; e < a.ne && ok; e += stride) {
      const double b = a.B[e];
      if (b < 0.0) {
        acc[0] += a.dmin;
        acc[1] += a.dmin;
        acc[3] += a.dmin;
        continue;
      }
      const double r = a.rho[e];
      const double lo = fmax(a.dmin, r - a.move), hi = fmin(1.0, r + a.move);
      const double k1 = b * s1, k2 = b * s2;  // k1 >= k2
      acc[0] += fmax(lo, fmin(hi, k1));
      acc[1] += fmax(lo, fmin(hi, k2));
      if (k2 >= hi) acc[3] += hi;
      else if (k1 <= lo) acc[3] += lo;
      else if (k2 > lo && k1 < hi) acc[2] += b;
      else {
        acc[4] += 1.0;
        const unsigned k = atomicAdd(list_n, 1u);
        if (k < (unsigned)kOcList) {
          list[3 * k] = b;
          list[3 * k + 1] = lo;
          list[3 * k + 2] = hi;
        }
      }
    }
    double* slot = a.part + (size_t)(passes & 1) * kOcK * nb;
    block_sum<5>(acc, sRed);
    if (threadIdx.x == 0)
      for (int j = 0; j < 5; j++) slot[(size_t)j * nb + blockIdx.x] = acc[j];
    if (ok) ok = grid_sync(a.bar, gen);
    passes++;
    double tot[5];
    grid_total<5>(slot, tot, sRed);
    const bool sign = tot[0] - a.target > 0.0 && tot[1] - a.target <= 0.0;
    if (ok && sign && tot[4] == 0.0 && tot[2] > 0.0 && a.target > tot[3]) {
      const double rt = tot[2] / (a.target - tot[3]);
      lfinal = rt * rt;
      exact = lfinal >= c1 && lfinal <= c2;
      root = exact ? 1 : 0;
    } else if (ok && sign && tot[4] <= (double)kOcList && c1 > 0.0) {
      __shared__ double s_root;
      if (threadIdx.x == 0) s_root = oc_piecewise_root(list, (int)tot[4], c1, c2, tot[3], tot[2], a.target);
      __syncthreads();
      lfinal = s_root;
      exact = lfinal > 0.0;
      root = exact ? 2 : 0;
    }
    if (!exact) {
      if (sign) {
        __syncthreads();
        if (threadIdx.x == 0) {
          sh_l[0] = c1;
          sh_l[1] = c2;
        }
        __syncthreads();
      } else {
        found = false;
      }
    }
  }
  if (ok && !exact) {
    if (!found) found = widen(false);
    if (found) bisect(false, 1e-10);
    lfinal = 0.5 * (sh_l[0] + sh_l[1]);
  }
  // final update
  __shared__ double sh_sfin;
  __syncthreads();
  if (threadIdx.x == 0) sh_sfin = 1.0 / sqrt(lfinal);
  __syncthreads();
  const double sfin = sh_sfin;
  double accv[2] = {0.0, 0.0};
  if (ok) {
    for (long long e = first; e < a.ne; e += stride) {
      const double r = a.rho[e], b = a.B[e];
      const double nv = b < 0.0 ? a.dmin : oc_clamp(r, b * sfin, a.move, a.dmin);
      a.rho_new[e] = nv;
      accv[0] += nv;
      accv[1] = fmax(accv[1], fabs(nv - r));
    }
  }
  double vol[1] = {accv[0]};
  block_sum<1>(vol, sRed);
  const double ch = block_max(accv[1], sRed);
  double* fin = a.part + (size_t)2 * kOcK * nb;
  if (threadIdx.x == 0) {
    fin[blockIdx.x] = vol[0];
    fin[(size_t)nb + blockIdx.x] = ch;
  }
  if (ok) ok = grid_sync(a.bar, gen);
  if (blockIdx.x == 0) {
    double v[1] = {0.0};
    double m = 0.0;
    if (ok) {
      for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        v[0] += __ldcg(fin + b);
        m = fmax(m, __ldcg(fin + nb + b));
      }
    }
    block_sum<1>(v, sRed);
    m = block_max(m, sRed);
    if (threadIdx.x == 0) {
      a.st->lambda = lfinal;
      a.st->volume = v[0];
      a.st->change = m;
      a.st->passes = passes;
      a.st->root = root;
      a.st->flags = (ok ? 0 : ERR_TIMEOUT) | (found || exact ? 0 : ERR_NAN);
    }
  }
}

cudaError_t launch_oc(cudaStream_t s, long long ne, const double* rho, const double* dcf,
                      const int8_t* passive, double volfrac, double move, double dmin,
                      double* rho_new, double* bscratch, double* part, GridBar* bar, OcStatus* st,
                      int nsm, int* grid_out, int max_grid) {
  OcArgs a;
  a.ne = ne;
  a.rho = rho;
  a.dcf = dcf;
  a.passive = passive;
  a.target = volfrac * (double)ne;
  a.move = move;
  a.dmin = dmin;
  a.rho_new = rho_new;
  a.B = bscratch;
  a.part = part;
  a.bar = bar;
  a.st = st;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, oc_kernel, 256, 0);
  if (e != cudaSuccess) return e;
  if (per_sm > 2) per_sm = 2;
  long long need = (ne + 255) / 256;
  int grid = per_sm * nsm;
  if (need < grid) grid = (int)need;
  if (max_grid > 0 && grid > max_grid) grid = max_grid;
  if (grid < 1) grid = 1;
  *grid_out = grid;
  void* args[] = {(void*)&a};
  return cudaLaunchCooperativeKernel((const void*)oc_kernel, dim3(grid), dim3(256), args, 0, s);
}

}  // namespace tp
