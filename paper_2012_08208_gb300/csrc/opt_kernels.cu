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
    for (int k = 0; k < a.ntaps; k++) {
      const int dx = a.off[3 * k], dy = a.off[3 * k + 1], dz = a.off[3 * k + 2];
      const int nx = gx + dx, ny = gy + dy, nz = gz + dz;
      if (nx < 0 || nx >= g.ex || ny < 0 || ny >= g.ey || nz < 0 || nz >= g.ez) continue;
      const int sidx = ((DIM == 3 ? tz + R + dz : 0) * SY + (ty + R + dy)) * SX + (tx + R + dx);
      num = fma(a.w[k], sG[sidx], num);
      den += a.w[k];
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
// OC update with a 16-way bisection.
//
// V(lambda) = sum_e rho_new_e(lambda) is non-increasing in lambda.  Each pass
// evaluates V at 15 interior points of the bracket [l1, l2] in one sweep over
// the elements (B_e = rho_e sqrt(max(-dc~_e, 0)) precomputed, candidate
// rho_e B_e / sqrt(lambda_j)), then keeps the sub-interval where
// V - target changes sign: points with V - target > 0 move l1 up, the first
// point with V - target <= 0 becomes l2 (the paper's rule, Section 4.4 code).
// The first pass widens the bracket: l2 = 1e9 * 10^j for the first j with
// V <= target.  Stop when l2 - l1 <= 1e-10 (l1 + l2); final rho_new uses the
// midpoint.  Passive elements are held at dmin inside the search.

constexpr int kOcK = 15;

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
  const int nb = gridDim.x;
  const long long stride = (long long)nb * blockDim.x;
  const long long first = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  unsigned gen = 0;
  bool ok = true;
  int passes = 0;
  double lam[kOcK], s[kOcK];

  // Partial sums alternate between two slots so that the totals of pass k can
  // be read while pass k+1 already writes its partials.
  auto sweep = [&](bool init, double (&tot)[kOcK]) -> bool {
    double* slot = a.part + (size_t)(passes & 1) * kOcK * nb;
    double acc[kOcK];
#pragma unroll
    for (int j = 0; j < kOcK; j++) acc[j] = 0.0;
    for (long long e = first; e < a.ne; e += stride) {
      const double r = a.rho[e];
      double b;
      if (init) {
        b = r * sqrt(fmax(-a.dcf[e], 0.0));
        a.B[e] = b;
      } else {
        b = a.B[e];
      }
      const bool pas = a.passive != nullptr && a.passive[e] == 1;
#pragma unroll
      for (int j = 0; j < kOcK; j++) acc[j] += pas ? a.dmin : oc_clamp(r, b * s[j], a.move, a.dmin);
    }
    block_sum<kOcK>(acc, sRed);
    if (threadIdx.x == 0)
      for (int j = 0; j < kOcK; j++) slot[(size_t)j * nb + blockIdx.x] = acc[j];
    if (!grid_sync(a.bar, gen)) return false;
    grid_total<kOcK>(slot, tot, sRed);
    return true;
  };

  // widening pass: lambda_j = 1e9 * 10^j
  double l1 = 0.0, l2 = 1e9;
  bool found = false;
  for (int round = 0; round < 20 && ok && !found; round++) {
#pragma unroll
    for (int j = 0; j < kOcK; j++) {
      lam[j] = l2 * pow(10.0, (double)j);
      s[j] = 1.0 / sqrt(lam[j]);
    }
    double tot[kOcK];
    ok = sweep(round == 0, tot);
    passes++;
    if (!ok) break;
    int jf = -1;
#pragma unroll
    for (int j = kOcK - 1; j >= 0; j--)
      if (tot[j] - a.target <= 0.0) jf = j;
    if (jf >= 0) {
      found = true;
      if (jf > 0) l1 = lam[jf - 1];
      l2 = lam[jf];
    } else {
      l1 = lam[kOcK - 1];
      l2 = lam[kOcK - 1] * 10.0;
      if (!isfinite(l2)) break;
    }
  }
  // multi-point bisection
  while (ok && found && (l2 - l1) > 1e-10 * (l1 + l2) && passes < 200) {
    const double h = (l2 - l1) / (kOcK + 1);
#pragma unroll
    for (int j = 0; j < kOcK; j++) {
      lam[j] = l1 + h * (j + 1);
      s[j] = 1.0 / sqrt(lam[j]);
    }
    double tot[kOcK];
    ok = sweep(false, tot);
    passes++;
    if (!ok) break;
    int jf = kOcK;
#pragma unroll
    for (int j = kOcK - 1; j >= 0; j--)
      if (tot[j] - a.target <= 0.0) jf = j;
    const double nl1 = jf > 0 ? lam[jf - 1] : l1;
    const double nl2 = jf < kOcK ? lam[jf] : l2;
    if (nl1 == l1 && nl2 == l2) break;  // bracket cannot shrink further in FP64
    l1 = nl1;
    l2 = nl2;
  }
  // final update at the midpoint
  const double lmid = 0.5 * (l1 + l2);
  double accv[2] = {0.0, 0.0};
  if (ok) {
    for (long long e = first; e < a.ne; e += stride) {
      const double r = a.rho[e];
      double nv;
      if (a.passive != nullptr && a.passive[e] == 1) {
        nv = a.dmin;
      } else {
        const double cand = r * sqrt(fmax(-a.dcf[e], 0.0) / lmid);
        nv = oc_clamp(r, cand, a.move, a.dmin);
      }
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
      a.st->lambda = lmid;
      a.st->volume = v[0];
      a.st->change = m;
      a.st->passes = passes;
      a.st->flags = (ok ? 0 : ERR_TIMEOUT) | (found ? 0 : ERR_NAN);
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
