// Batched SIMP iteration for many independent 2D problems of uneven size
// (Q4, one load case each), all solved in one persistent launch.
//
// Every instance is the problem of Section 4 (SIMP, Section 3.2 sensitivities,
// Section 3.2.2 filter, Eq. "update" OC with bisection) on its own grid.  The
// instances are independent, so the batch is a work list: each instance gets a
// contiguous range of CTAs proportional to its number of node tiles, and every
// CTA serves one instance.  All instances advance their CG iterations in
// lock-step between grid barriers; an instance that has converged skips its
// work.  The FP64 true-residual updates run inside the same launch, so a whole
// SIMP iteration (moduli, diagonal, CG, sensitivities, filter, OC) is a fixed
// sequence of kernels that is captured once in a CUDA graph and replayed.
// The tile height and CTAs per SM are chosen by tp_batch_autotune.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/topo.h"
#include "pcg_common.cuh"

namespace tp {

struct BInst {
  Grid g;               // instance grid (dim 2)
  long long noff, eoff; // offsets into the concatenated node / element arrays
  int tiles_x, ntiles;  // node tiles of the instance
  int cta0, ncta;       // CTAs serving the instance
  double tol2ff;        // tol^2 ||f||^2 (free DOFs)
  double volfrac, move, dmin, penal, dE, Emin;
  int tap0, ntaps;      // filter taps in the shared tap table
};

struct BOut {
  int iters, updates, state, oc_flags;
  double rr_true, ff, compliance;
  double lambda, volume, change;
};

// ---------------------------------------------------------------------------
// helpers

__device__ __forceinline__ int find_inst(const BInst* in, int n, long long idx, bool nodes) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const long long off = nodes ? in[mid].noff : in[mid].eoff;
    if (off <= idx) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Sum of one value over the CTAs [c0, c0 + nc) of an instance (per-CTA FP64
// slots, fixed order); result broadcast to the CTA.
__device__ __forceinline__ double inst_total(const double* slot, int c0, int nc, double* sbuf) {
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int c = threadIdx.x; c < nc; c += 32) s += __ldcg(slot + c0 + c);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) *sbuf = s;
  }
  __syncthreads();
  const double v = *sbuf;
  __syncthreads();
  return v;
}

// Per-CTA partial (one value): FP64 block sum written to slot[blockIdx.x].
__device__ __forceinline__ void cta_partial1(double v, double* slot, double* sred) {
  double a[1] = {v};
  block_sum<1>(a, sred);
  if (threadIdx.x == 0) slot[blockIdx.x] = a[0];
}

// ---------------------------------------------------------------------------
// moduli and Jacobi diagonal for all instances

__global__ void batch_young_kernel(const BInst* in, int n, long long ne_tot, const double* rho, float* E32,
                                   double* E64) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne_tot;
       e += (long long)gridDim.x * blockDim.x) {
    const BInst& I = in[find_inst(in, n, e, false)];
    const double r = rho[e];
    const double rp = I.penal == 3.0 ? r * r * r : pow(r, I.penal);
    const double E = I.Emin + rp * I.dE;
    E64[e] = E;
    E32[e] = (float)E;
  }
}

struct BDiagArgs {
  const BInst* in;
  int n;
  long long nn_tot;
  const double* E64;
  const uint8_t* mask;
  float* inv32;
  double kd[8];
};

__global__ void batch_diag_kernel(const __grid_constant__ BDiagArgs a) {
  for (long long gn = blockIdx.x * (long long)blockDim.x + threadIdx.x; gn < a.nn_tot;
       gn += (long long)gridDim.x * blockDim.x) {
    const BInst& I = a.in[find_inst(a.in, a.n, gn, true)];
    const long long n = gn - I.noff;
    const int x = (int)(n % I.g.nx), y = (int)(n / I.g.nx);
    double d[2] = {0.0, 0.0};
#pragma unroll
    for (int cn = 0; cn < 4; cn++) {
      const int ex = x - cofs(cn, 0), ey = y - cofs(cn, 1);
      if (ex < 0 || ey < 0 || ex >= I.g.ex || ey >= I.g.ey) continue;
      const double E = a.E64[I.eoff + ex + (long long)I.g.ex * ey];
      d[0] += E * a.kd[2 * cn];
      d[1] += E * a.kd[2 * cn + 1];
    }
    const uint8_t mk = a.mask[gn];
#pragma unroll
    for (int r = 0; r < 2; r++) {
      const double v = ((mk >> r) & 1) ? 1.0 : 1.0 / d[r];
      a.inv32[2 * I.noff + r * I.g.nn + n] = (float)v;
    }
  }
}

// ---------------------------------------------------------------------------
// The batched persistent CG (FP32 operator and vectors, FP64 reductions via
// FP64 block sums, FP64 true-residual updates inside the launch).

struct BCgArgs {
  const BInst* in;
  const int* cta_inst;
  int ninst;
  const float* E32;
  const double* E64;
  const uint8_t* mask;
  const float* inv32;
  const double* f;
  double* x64;
  float* xl;
  float* r;
  float* z;
  float* p0;
  float* p1;
  float* q;
  double* part;      // [slot][gridDim.x]
  unsigned* flags;   // [4]: need (2 parity slots), active (2 parity slots)
  GridBar* bar;
  BOut* out;
  double drop2;
  int max_it;
  CMat<2, float> Cf;
  CMat<2, double> Cd;
};

constexpr int BSLOT_PQ = 0, BSLOT_RZ = 1, BSLOT_RR = 2, BSLOT_RT = 3, BSLOT_RZT = 4, BSLOT_C = 5;

template <int TY>
__global__ void __launch_bounds__(256) batch_cg_kernel(const __grid_constant__ BCgArgs a) {
  using OpF = Q4Tile<float, TY>;
  using OpD = Q4Tile<double, TY>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double sred[32];
  __shared__ double sbuf;
  __shared__ float scoef[2];
  __shared__ int sflag[2];
  const int nb = gridDim.x;
  const BInst I = a.in[a.cta_inst[blockIdx.x]];
  const int k = blockIdx.x - I.cta0;
  const Grid g = I.g;
  TileMapG tm;
  tm.tiles_x = I.tiles_x;
  tm.tiles_y = (g.ny + TY - 1) / TY;
  tm.tiles_z = 1;
  tm.ntiles = I.ntiles;
  tm.zlen = 1;
  const long long nn = g.nn;
  const long long vo = 2 * I.noff;
  const float* E32 = a.E32 + I.eoff;
  const double* E64 = a.E64 + I.eoff;
  const uint8_t* mask = a.mask + I.noff;
  const float* inv = a.inv32 + vo;
  const double* f = a.f + vo;
  double* x64 = a.x64 + vo;
  float* xl = a.xl + vo;
  float* r = a.r + vo;
  float* z = a.z + vo;
  float* q = a.q + vo;
  float* P[2] = {a.p0 + vo, a.p1 + vo};
  const bool t0 = threadIdx.x == 0;
  unsigned gen = 0;
  bool ok = true;

  // Scalar state of this CTA's instance, owned by thread 0 (FP64 work on one
  // thread only); the values the other threads need are shared through smem.
  __shared__ int s_state;
  if (t0) s_state = 0;
  int state = 0, stall = 0, it = 0, updates = 0, pbuf = 0;
  double rz = 0.0, rr_ref = 0.0, beta = 0.0, rr_true = 0.0;
  auto share = [&](double al) {
    if (t0) {
      s_state = state;
      scoef[0] = (float)beta;
      scoef[1] = (float)al;
    }
    __syncthreads();
  };

  auto merge = [&]() {
    for (int t = k; t < I.ntiles; t += I.ncta)
      OpF::for_each_own(g, tm, t, [&](long long node) {
#pragma unroll
        for (int c = 0; c < 2; c++) {
          const long long i = c * nn + node;
          x64[i] += (double)xl[i];
          xl[i] = 0.f;
        }
      });
  };
  // r = f - K64 x64, z = D^-1 r; per-CTA partials of ||r||^2 (FP64) and r.z
  auto residual = [&]() {
    double srr = 0.0, srz = 0.0;
    for (int t = k; t < I.ntiles; t += I.ncta)
      OpD::template apply<1>(
          g, tm, t, E64, a.Cd, smem_raw, 1,
          [&](long long node, int v, bool) -> double {
            return ((mask[node] >> v) & 1) ? 0.0 : __ldcg(x64 + v * nn + node);
          },
          [&](long long node, int, const double(&yv)[2], const double(&)[2]) {
            const uint8_t mk = mask[node];
#pragma unroll
            for (int c = 0; c < 2; c++) {
              const long long i = c * nn + node;
              const double r64 = ((mk >> c) & 1) ? 0.0 : f[i] - yv[c];
              const float rt = (float)r64;
              const float zt = rt * inv[i];
              r[i] = rt;
              z[i] = zt;
              srr += r64 * r64;
              srz += (double)rt * (double)zt;
            }
          });
    cta_partial1(srr, a.part + (size_t)BSLOT_RT * nb, sred);
    cta_partial1(srz, a.part + (size_t)BSLOT_RZT * nb, sred);
  };
  // after a residual phase and its barrier: totals and the instance's update (thread 0)
  // `own` = the update was requested by this instance; only then does a true
  // residual that failed to halve count towards stagnation (updates requested
  // by other instances can come after only a few iterations).
  auto after_residual = [&](bool init, bool own) {
    const double rr = inst_total(a.part + (size_t)BSLOT_RT * nb, I.cta0, I.ncta, &sbuf);
    const double rzt = inst_total(a.part + (size_t)BSLOT_RZT * nb, I.cta0, I.ncta, &sbuf);
    if (t0) {
      rr_true = rr;
      if (init) {
        rr_ref = rr;
        rz = rzt;
        beta = 0.0;
        state = rr <= I.tol2ff ? 1 : 0;
      } else if (state == 0) {
        if (own) stall = rr > 0.25 * rr_ref ? stall + 1 : 0;
        rr_ref = rr;
        beta = rz != 0.0 ? rzt / rz : 0.0;
        rz = rzt;
        if (rr <= I.tol2ff) state = 1;
        else if (stall >= 6) state = 3;
      }
    }
    share(0.0);
  };
  // global flag counters (parity slot by iteration): written before a barrier,
  // read after it; CTA 0 clears the other parity slot
  auto flag_add = [&](int which, int par, bool v) {
    if (t0 && v) atomicAdd(&a.flags[2 * which + par], 1u);
  };
  auto flag_read = [&](int which, int par) -> bool {
    if (t0) {
      sflag[0] = *(volatile unsigned*)&a.flags[2 * which + par] != 0;
      if (blockIdx.x == 0) a.flags[2 * which + (par ^ 1)] = 0u;
    }
    __syncthreads();
    const bool v = sflag[0] != 0;
    __syncthreads();
    return v;
  };

  residual();
  ok = grid_sync(a.bar, gen);
  if (ok) after_residual(true, false);
  bool fresh = true;
  flag_add(1, 0, s_state == 0);
  if (ok) ok = grid_sync(a.bar, gen);
  bool go = ok && flag_read(1, 0);

  while (go && it < a.max_it) {
    const bool act = s_state == 0;
    // ---- phase A
    const float b = scoef[0];
    const float* Pold = P[pbuf];
    float* Pnew = P[pbuf ^ 1];
    float spq = 0.f;
    if (act) {
      for (int t = k; t < I.ntiles; t += I.ncta)
        OpF::template apply<1>(
            g, tm, t, E32, a.Cf, smem_raw, 1,
            [&](long long node, int v, bool) -> float {
              const long long i = v * nn + node;
              float val = __ldcg(z + i);
              if (b != 0.f) val = fmaf(b, __ldcg(Pold + i), val);
              return val;
            },
            [&](long long node, int, const float(&yv)[2], const float(&us)[2]) {
              const uint8_t mk = mask[node];
#pragma unroll
              for (int c = 0; c < 2; c++) {
                const long long i = c * nn + node;
                const float qv = ((mk >> c) & 1) ? 0.f : yv[c];
                q[i] = qv;
                Pnew[i] = us[c];
                spq = fmaf(us[c], qv, spq);
              }
            });
    }
    cta_partial1((double)spq, a.part + (size_t)BSLOT_PQ * nb, sred);
    if (!(ok = grid_sync(a.bar, gen))) break;
    {
      const double pq = inst_total(a.part + (size_t)BSLOT_PQ * nb, I.cta0, I.ncta, &sbuf);
      double alpha = 0.0;
      if (t0 && state == 0) {
        if (!(pq > 0.0) || !isfinite(pq)) state = 2;
        else alpha = rz / pq;
      }
      share(alpha);
    }
    // ---- phase B
    const float al = scoef[1];
    float srz = 0.f, srr = 0.f;
    if (s_state == 0) {
      for (int t = k; t < I.ntiles; t += I.ncta)
        OpF::for_each_own(g, tm, t, [&](long long node) {
          float rv[2], pv[2], qv[2], xv[2], iv[2];
#pragma unroll
          for (int c = 0; c < 2; c++) {
            const long long i = c * nn + node;
            rv[c] = r[i];
            pv[c] = Pnew[i];
            qv[c] = q[i];
            xv[c] = xl[i];
            iv[c] = inv[i];
          }
#pragma unroll
          for (int c = 0; c < 2; c++) {
            const long long i = c * nn + node;
            const float rn = fmaf(-al, qv[c], rv[c]);
            const float zn = rn * iv[c];
            xl[i] = fmaf(al, pv[c], xv[c]);
            r[i] = rn;
            z[i] = zn;
            srz = fmaf(rn, zn, srz);
            srr = fmaf(rn, rn, srr);
          }
        });
    }
    cta_partial1((double)srz, a.part + (size_t)BSLOT_RZ * nb, sred);
    cta_partial1((double)srr, a.part + (size_t)BSLOT_RR * nb, sred);
    if (!(ok = grid_sync(a.bar, gen))) break;
    const double rzn = inst_total(a.part + (size_t)BSLOT_RZ * nb, I.cta0, I.ncta, &sbuf);
    const double rr = inst_total(a.part + (size_t)BSLOT_RR * nb, I.cta0, I.ncta, &sbuf);
    it++;
    pbuf ^= 1;
    fresh = false;
    bool need = false;
    if (t0) need = state == 0 && (rr <= I.tol2ff || rr <= a.drop2 * rr_ref);
    const bool own_need = need;
    flag_add(0, it & 1, need);
    if (!(ok = grid_sync(a.bar, gen))) break;
    const bool any_need = flag_read(0, it & 1);
    if (any_need) {
      merge();
      if (!(ok = grid_sync(a.bar, gen))) break;
      residual();
      if (!(ok = grid_sync(a.bar, gen))) break;
      after_residual(false, own_need);
      updates++;
      fresh = true;
    } else {
      if (t0 && state == 0) {
        beta = rz != 0.0 ? rzn / rz : 0.0;
        rz = rzn;
      }
      share(0.0);
    }
    flag_add(1, it & 1, s_state == 0);
    if (!(ok = grid_sync(a.bar, gen))) break;
    go = flag_read(1, it & 1);
  }
  if (ok && !fresh) {
    merge();
    ok = grid_sync(a.bar, gen);
    if (ok) residual();
    if (ok) ok = grid_sync(a.bar, gen);
    if (ok) {
      const int st_keep = t0 ? state : 0;
      after_residual(false, false);
      if (t0 && st_keep == 0 && state == 3) state = 0;  // one final evaluation is not stagnation
      updates++;
    }
  }
  // compliance c = f . x64 over the instance
  double sc = 0.0;
  if (ok)
    for (int t = k; t < I.ntiles; t += I.ncta)
      OpF::for_each_own(g, tm, t, [&](long long node) {
        sc = fma(f[node], x64[node], sc);
        sc = fma(f[nn + node], x64[nn + node], sc);
      });
  cta_partial1(sc, a.part + (size_t)BSLOT_C * nb, sred);
  if (ok) ok = grid_sync(a.bar, gen);
  const double comp = inst_total(a.part + (size_t)BSLOT_C * nb, I.cta0, I.ncta, &sbuf);
  if (k == 0 && t0) {
    BOut& o = a.out[a.cta_inst[blockIdx.x]];
    o.iters = it;
    o.updates = updates;
    o.state = ok ? state : -1;
    o.rr_true = rr_true;
    o.compliance = comp;
  }
}

// ---------------------------------------------------------------------------
// sensitivities and filter for all instances (FP64)

struct BSensArgs {
  const BInst* in;
  int n;
  long long ne_tot;
  const double* x64;
  const double* rho;
  double* dc;
  CMat<2, double> C;
};

__global__ void batch_sens_kernel(const __grid_constant__ BSensArgs a) {
  for (long long ge = blockIdx.x * (long long)blockDim.x + threadIdx.x; ge < a.ne_tot;
       ge += (long long)gridDim.x * blockDim.x) {
    const BInst& I = a.in[find_inst(a.in, a.n, ge, false)];
    const long long e = ge - I.eoff;
    const int ex = (int)(e % I.g.ex), ey = (int)(e / I.g.ex);
    const double* x = a.x64 + 2 * I.noff;
    double ux[4], uy[4];
#pragma unroll
    for (int m = 0; m < 4; m++) {
      const long long node = (ex + cofs(m, 0)) + (long long)I.g.nx * (ey + cofs(m, 1));
      ux[m] = x[node];
      uy[m] = x[I.g.nn + node];
    }
    const double ce = q4_energy(ux, uy, a.C);
    const double rr = a.rho[ge];
    const double rp1 = I.penal == 3.0 ? rr * rr : pow(rr, I.penal - 1.0);
    a.dc[ge] = -I.penal * rp1 * I.dE * ce;
  }
}

struct BFiltArgs {
  const BInst* in;
  int n;
  long long ne_tot;
  const int* taps;      // (dx, dy) pairs
  const double* w;
  const double* rho;
  const double* dc;
  double* dcf;
};

__global__ void batch_filter_kernel(const __grid_constant__ BFiltArgs a) {
  for (long long ge = blockIdx.x * (long long)blockDim.x + threadIdx.x; ge < a.ne_tot;
       ge += (long long)gridDim.x * blockDim.x) {
    const BInst& I = a.in[find_inst(a.in, a.n, ge, false)];
    const long long e = ge - I.eoff;
    const int ex = (int)(e % I.g.ex), ey = (int)(e / I.g.ex);
    double num = 0.0, den = 0.0;
    for (int t = I.tap0; t < I.tap0 + I.ntaps; t++) {
      const int nx = ex + a.taps[2 * t], ny = ey + a.taps[2 * t + 1];
      if (nx < 0 || ny < 0 || nx >= I.g.ex || ny >= I.g.ey) continue;
      const long long nb = I.eoff + nx + (long long)I.g.ex * ny;
      num = fma(a.w[t], a.rho[nb] * a.dc[nb], num);
      den += a.w[t];
    }
    a.dcf[ge] = num / (a.rho[ge] * den);
  }
}

// ---------------------------------------------------------------------------
// batched OC: per-instance 16-way bisection (same readings as oc_kernel), CTAs
// of an instance evaluate contiguous element chunks; one grid barrier per pass.

struct BOcArgs {
  const BInst* in;
  const int* cta_inst;
  const double* rho;
  const double* dcf;
  double* rho_new;
  double* part;     // [16][gridDim.x]
  unsigned* flags;  // [2] parity counters: instances not done
  GridBar* bar;
  BOut* out;
};

__global__ void __launch_bounds__(256) batch_oc_kernel(const __grid_constant__ BOcArgs a) {
  constexpr int K = 15;
  __shared__ double sred[32 * K];
  __shared__ double stot[K];
  __shared__ double slam[K], ss[K];
  __shared__ int sflag;
  const int nb = gridDim.x;
  const BInst I = a.in[a.cta_inst[blockIdx.x]];
  const int k = blockIdx.x - I.cta0;
  const long long ne = I.g.ne;
  const long long chunk = (ne + I.ncta - 1) / I.ncta;
  const long long e0 = I.eoff + k * chunk, e1 = I.eoff + min(ne, (k + 1) * chunk);
  const double target = I.volfrac * (double)ne;
  unsigned gen = 0;
  bool ok = true;
  double l1 = 0.0, l2 = 1e9;
  int phase = 0;  // 0 widening, 1 bisection, 2 done
  int passes = 0;
  auto eval = [&](double (&tot)[K]) -> bool {
    double acc[K];
#pragma unroll
    for (int j = 0; j < K; j++) acc[j] = 0.0;
    if (phase < 2) {
      double s[K];
#pragma unroll
      for (int j = 0; j < K; j++) s[j] = ss[j];
      for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const double rr = a.rho[e];
        const double bb = rr * sqrt(fmax(-a.dcf[e], 0.0));
#pragma unroll
        for (int j = 0; j < K; j++)
          acc[j] += fmax(I.dmin, fmax(rr - I.move, fmin(1.0, fmin(rr + I.move, bb * s[j]))));
      }
    }
    block_sum<K>(acc, sred);
    if (threadIdx.x == 0)
      for (int j = 0; j < K; j++) a.part[(size_t)j * nb + blockIdx.x] = acc[j];
    if (!grid_sync(a.bar, gen)) return false;
    for (int j = 0; j < K; j++) tot[j] = inst_total(a.part + (size_t)j * nb, I.cta0, I.ncta, &stot[j]);
    return true;
  };
  bool go = true;
  while (go && ok && passes < 200) {
    if (threadIdx.x < K) {
      const int j = threadIdx.x;
      const double lj = phase == 0 ? l2 * pow(10.0, (double)j) : l1 + (l2 - l1) / (K + 1) * (j + 1);
      slam[j] = lj;
      ss[j] = 1.0 / sqrt(lj);
    }
    __syncthreads();
    double lam[K];
#pragma unroll
    for (int j = 0; j < K; j++) lam[j] = slam[j];
    double tot[K];
    ok = eval(tot);
    if (!ok) break;
    passes++;
    if (phase == 0) {
      int jf = -1;
      for (int j = K - 1; j >= 0; j--)
        if (tot[j] - target <= 0.0) jf = j;
      if (jf >= 0) {
        if (jf > 0) l1 = lam[jf - 1];
        l2 = lam[jf];
        phase = 1;
      } else {
        l1 = lam[K - 1];
        l2 = lam[K - 1] * 10.0;
        if (!isfinite(l2)) phase = 2;
      }
    } else if (phase == 1) {
      int jf = K;
      for (int j = K - 1; j >= 0; j--)
        if (tot[j] - target <= 0.0) jf = j;
      const double nl1 = jf > 0 ? lam[jf - 1] : l1;
      const double nl2 = jf < K ? lam[jf] : l2;
      if (nl1 == l1 && nl2 == l2) phase = 2;
      l1 = nl1;
      l2 = nl2;
    }
    if (phase == 1 && (l2 - l1) <= 1e-10 * (l1 + l2)) phase = 2;
    // continue while any instance still searches
    if (threadIdx.x == 0 && phase < 2) atomicAdd(&a.flags[passes & 1], 1u);
    ok = grid_sync(a.bar, gen);
    if (!ok) break;
    if (threadIdx.x == 0) {
      sflag = *(volatile unsigned*)&a.flags[passes & 1] != 0;
      if (blockIdx.x == 0) a.flags[(passes & 1) ^ 1] = 0u;
    }
    __syncthreads();
    go = sflag != 0;
    __syncthreads();
  }
  const double lmid = 0.5 * (l1 + l2);
  double v[2] = {0.0, 0.0};
  double ch = 0.0;
  for (long long e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const double rr = a.rho[e];
    const double cand = rr * sqrt(fmax(-a.dcf[e], 0.0) / lmid);
    const double nv = fmax(I.dmin, fmax(rr - I.move, fmin(1.0, fmin(rr + I.move, cand))));
    a.rho_new[e] = nv;
    v[0] += nv;
    ch = fmax(ch, fabs(nv - rr));
  }
  block_sum<2>(v, sred);
  const double cm = block_max(ch, sred);
  if (threadIdx.x == 0) {
    a.part[blockIdx.x] = v[0];
    a.part[(size_t)nb + blockIdx.x] = cm;
  }
  if (ok) ok = grid_sync(a.bar, gen);
  const double vol = inst_total(a.part, I.cta0, I.ncta, &stot[0]);
  if (threadIdx.x < 32) {
    double m = 0.0;
    for (int c = threadIdx.x; c < I.ncta; c += 32) m = fmax(m, __ldcg(a.part + nb + I.cta0 + c));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) stot[1] = m;
  }
  __syncthreads();
  if (k == 0 && threadIdx.x == 0) {
    BOut& o = a.out[a.cta_inst[blockIdx.x]];
    o.lambda = lmid;
    o.volume = vol;
    o.change = stot[1];
    o.oc_flags = (ok ? 0 : ERR_TIMEOUT) | (phase == 2 ? 0 : ERR_NAN);
  }
}

}  // namespace tp

// ===========================================================================
// Host side

using namespace tp;

struct tp_batch {
  int n = 0;
  cudaStream_t stream = nullptr;
  int dev = 0, nsm = 0;
  std::vector<tp_params> prm;
  std::vector<BInst> inst;
  std::vector<int> taps;
  std::vector<double> wts;
  std::vector<double> ff;
  long long nn_tot = 0, ne_tot = 0;
  std::vector<double> K0, C;
  int tile_rows = 8, ctas_per_sm = 2;
  // device
  BInst* d_inst = nullptr;
  int* d_cta = nullptr;
  int* d_taps = nullptr;
  double* d_w = nullptr;
  double *rho = nullptr, *rho_new = nullptr, *E64 = nullptr, *f = nullptr, *x64 = nullptr, *dc = nullptr,
         *dcf = nullptr, *part = nullptr;
  float *E32 = nullptr, *inv32 = nullptr, *xl = nullptr, *r = nullptr, *z = nullptr, *p0 = nullptr, *p1 = nullptr,
        *q = nullptr;
  uint8_t* mask = nullptr;
  unsigned* flags = nullptr;
  GridBar* bar = nullptr;
  BOut* out = nullptr;
  int grid = 0;
  size_t npart = 0;
  std::vector<uint8_t> have_fixed, have_loads;
  // graph
  cudaGraphExec_t gexec = nullptr;
  bool graph_ok = false;
  tp_solve_opts gopts{};
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::string err;
  long long launches = 0;
};

namespace {

tp_status bfail(tp_batch* b, tp_status s, const std::string& m) {
  if (b) b->err = m;
  return s;
}

#define BCK(call, what)                                                                  \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      cudaGetLastError();                                                                \
      return bfail(b, e_ == cudaErrorMemoryAllocation ? TP_ERR_OOM : TP_ERR_CUDA,        \
                   std::string(what) + ": " + cudaGetErrorString(e_));                   \
    }                                                                                    \
  } while (0)

int bgrid(long long n) {
  long long g = (n + 255) / 256;
  return (int)std::max(1LL, std::min(g, 152LL * 16));
}

template <int TY>
cudaError_t launch_batch_cg_ty(tp_batch* b, cudaStream_t s, const BCgArgs& a, size_t smem) {
  auto kern = batch_cg_kernel<TY>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)&a};
  return cudaLaunchCooperativeKernel((const void*)kern, dim3(b->grid), dim3(256), args, smem, s);
}

template <int TY>
int max_ctas_per_sm_ty(size_t smem) {
  int per = 0;
  cudaFuncSetAttribute(batch_cg_kernel<TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_cg_kernel<TY>, 256, smem);
  return per;
}

size_t cg_smem(int ty) { return (size_t)(34 * (ty + 2) * 2 + 33 * (ty + 1)) * sizeof(double); }

// Assign CTAs to instances in proportion to their tiles (at least one each).
tp_status plan(tp_batch* b) {
  const int ty = b->tile_rows;
  int per = ty == 4 ? max_ctas_per_sm_ty<4>(cg_smem(4)) : ty == 8 ? max_ctas_per_sm_ty<8>(cg_smem(8))
                                                                  : max_ctas_per_sm_ty<16>(cg_smem(16));
  per = std::min(per, b->ctas_per_sm);
  int per_oc = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_oc, batch_oc_kernel, 256, 0);
  per = std::min(per, per_oc);
  if (per < 1) return bfail(b, TP_ERR_CUDA, "no co-resident CTA fits");
  long long total_tiles = 0;
  for (auto& I : b->inst) {
    I.tiles_x = (I.g.nx + 31) / 32;
    I.ntiles = I.tiles_x * ((I.g.ny + ty - 1) / ty);
    total_tiles += I.ntiles;
  }
  int grid = std::min<long long>((long long)per * b->nsm, std::max<long long>(total_tiles, b->n));
  if (grid < b->n) return bfail(b, TP_ERR_ARG, "more instances than co-resident CTAs");
  // proportional allocation with at least one CTA and at most ntiles CTAs per instance
  std::vector<int> c(b->n, 1);
  int used = b->n;
  std::vector<double> want(b->n);
  for (int i = 0; i < b->n; i++) want[i] = (double)b->inst[i].ntiles / total_tiles * grid;
  while (used < grid) {
    int best = -1;
    double bs = -1e300;
    for (int i = 0; i < b->n; i++) {
      if (c[i] >= b->inst[i].ntiles) continue;
      const double sc = want[i] - c[i];
      if (sc > bs) {
        bs = sc;
        best = i;
      }
    }
    if (best < 0) break;
    c[best]++;
    used++;
  }
  b->grid = used;
  std::vector<int> cta_inst(used);
  int c0 = 0;
  for (int i = 0; i < b->n; i++) {
    b->inst[i].cta0 = c0;
    b->inst[i].ncta = c[i];
    for (int j = 0; j < c[i]; j++) cta_inst[c0 + j] = i;
    c0 += c[i];
  }
  if (b->d_cta) cudaFree(b->d_cta);
  BCK(cudaMalloc((void**)&b->d_cta, sizeof(int) * used), "alloc");
  BCK(cudaMemcpy(b->d_cta, cta_inst.data(), sizeof(int) * used, cudaMemcpyHostToDevice), "copy");
  BCK(cudaMemcpy(b->d_inst, b->inst.data(), sizeof(BInst) * b->n, cudaMemcpyHostToDevice), "copy");
  if (b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  b->graph_ok = false;
  return TP_OK;
}

// Enqueue one SIMP iteration for all instances on stream s.
tp_status enqueue_step(tp_batch* b, cudaStream_t s, const tp_solve_opts& o) {
  const long long ne = b->ne_tot, nn = b->nn_tot;
  batch_young_kernel<<<bgrid(ne), 256, 0, s>>>(b->d_inst, b->n, ne, b->rho, b->E32, b->E64);
  BDiagArgs da;
  da.in = b->d_inst;
  da.n = b->n;
  da.nn_tot = nn;
  da.E64 = b->E64;
  da.mask = b->mask;
  da.inv32 = b->inv32;
  for (int i = 0; i < 8; i++) da.kd[i] = b->K0[i * 8 + i];
  batch_diag_kernel<<<bgrid(nn), 256, 0, s>>>(da);
  BCK(cudaGetLastError(), "batch moduli");
  BCK(cudaMemsetAsync(b->xl, 0, sizeof(float) * 2 * nn, s), "memset");
  BCK(cudaMemsetAsync(b->bar, 0, sizeof(GridBar), s), "memset");
  BCK(cudaMemsetAsync(b->flags, 0, sizeof(unsigned) * 4, s), "memset");
  BCgArgs a;
  a.in = b->d_inst;
  a.cta_inst = b->d_cta;
  a.ninst = b->n;
  a.E32 = b->E32;
  a.E64 = b->E64;
  a.mask = b->mask;
  a.inv32 = b->inv32;
  a.f = b->f;
  a.x64 = b->x64;
  a.xl = b->xl;
  a.r = b->r;
  a.z = b->z;
  a.p0 = b->p0;
  a.p1 = b->p1;
  a.q = b->q;
  a.part = b->part;
  a.flags = b->flags;
  a.bar = b->bar;
  a.out = b->out;
  const double drop = o.update_drop > 0.0 ? o.update_drop : 0.1;
  a.drop2 = drop * drop;
  a.max_it = o.max_it;
  fill_c<2, float>(a.Cf, b->C.data());
  fill_c<2, double>(a.Cd, b->C.data());
  const int ty = b->tile_rows;
  const size_t smem = cg_smem(ty);
  cudaError_t e = ty == 4 ? launch_batch_cg_ty<4>(b, s, a, smem)
                          : ty == 8 ? launch_batch_cg_ty<8>(b, s, a, smem) : launch_batch_cg_ty<16>(b, s, a, smem);
  BCK(e, "batch cg kernel");
  BSensArgs sa;
  sa.in = b->d_inst;
  sa.n = b->n;
  sa.ne_tot = ne;
  sa.x64 = b->x64;
  sa.rho = b->rho;
  sa.dc = b->dc;
  fill_c<2, double>(sa.C, b->C.data());
  batch_sens_kernel<<<bgrid(ne), 256, 0, s>>>(sa);
  BFiltArgs fa;
  fa.in = b->d_inst;
  fa.n = b->n;
  fa.ne_tot = ne;
  fa.taps = b->d_taps;
  fa.w = b->d_w;
  fa.rho = b->rho;
  fa.dc = b->dc;
  fa.dcf = b->dcf;
  batch_filter_kernel<<<bgrid(ne), 256, 0, s>>>(fa);
  BCK(cudaGetLastError(), "batch sens/filter");
  BCK(cudaMemsetAsync(b->bar, 0, sizeof(GridBar), s), "memset");
  BCK(cudaMemsetAsync(b->flags, 0, sizeof(unsigned) * 4, s), "memset");
  BOcArgs oa;
  oa.in = b->d_inst;
  oa.cta_inst = b->d_cta;
  oa.rho = b->rho;
  oa.dcf = b->dcf;
  oa.rho_new = b->rho_new;
  oa.part = b->part;
  oa.flags = b->flags;
  oa.bar = b->bar;
  oa.out = b->out;
  void* oargs[] = {(void*)&oa};
  BCK(cudaLaunchCooperativeKernel((const void*)batch_oc_kernel, dim3(b->grid), dim3(256), oargs, 0, s),
      "batch oc kernel");
  BCK(cudaMemcpyAsync(b->rho, b->rho_new, sizeof(double) * ne, cudaMemcpyDeviceToDevice, s), "copy");
  b->launches += 6;
  return TP_OK;
}

}  // namespace

extern "C" {

tp_status tp_batch_create(int n, const tp_params* params, void* cuda_stream, tp_batch** out) {
  if (!params || !out || n < 1) return TP_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < n; i++) {
    const tp_params& q = params[i];
    if (q.dim != 2 || q.n_cases != 1 || q.nelx < 1 || q.nely < 1) return TP_ERR_ARG;
    if (!(q.volfrac > 0.0 && q.volfrac <= 1.0) || !(q.rmin > 0.0) || !(q.penal >= 1.0)) return TP_ERR_ARG;
    if (!(q.nu >= 0.0 && q.nu < 0.5) || !(q.Emin > 0.0 && q.Emin < q.E0)) return TP_ERR_ARG;
    if (!(q.dmin > 0.0 && q.dmin < 1.0) || !(q.move > 0.0)) return TP_ERR_ARG;
    if (q.nu != params[0].nu) return TP_ERR_ARG;  // one element matrix for the batch
  }
  tp_batch* b = new tp_batch();
  b->n = n;
  b->stream = (cudaStream_t)cuda_stream;
  b->prm.assign(params, params + n);
  b->inst.resize(n);
  b->ff.assign(n, 0.0);
  b->have_fixed.assign(n, 0);
  b->have_loads.assign(n, 0);
  b->K0.resize(64);
  element_k0(2, params[0].nu, b->K0.data());
  b->C.resize(25);
  double recon = 0.0;
  element_strain_C(2, b->K0.data(), b->C.data(), &recon);
  long long nn = 0, ne = 0;
  for (int i = 0; i < n; i++) {
    const tp_params& q = params[i];
    BInst& I = b->inst[i];
    memset(&I, 0, sizeof(I));
    I.g.dim = 2;
    I.g.ex = q.nelx;
    I.g.ey = q.nely;
    I.g.ez = 1;
    I.g.nx = q.nelx + 1;
    I.g.ny = q.nely + 1;
    I.g.nz = 1;
    I.g.nn = (long long)I.g.nx * I.g.ny;
    I.g.ne = (long long)I.g.ex * I.g.ey;
    I.noff = nn;
    I.eoff = ne;
    nn += I.g.nn;
    ne += I.g.ne;
    I.volfrac = q.volfrac;
    I.move = q.move;
    I.dmin = q.dmin;
    I.penal = q.penal;
    I.dE = q.E0 - q.Emin;
    I.Emin = q.Emin;
    int off[3 * kMaxTaps];
    double w[kMaxTaps];
    const int nt = filter_taps(2, q.rmin, kMaxTaps, off, w);
    if (nt < 1) {
      delete b;
      return TP_ERR_ARG;
    }
    I.tap0 = (int)b->wts.size();
    I.ntaps = nt;
    for (int t = 0; t < nt; t++) {
      b->taps.push_back(off[3 * t]);
      b->taps.push_back(off[3 * t + 1]);
      b->wts.push_back(w[t]);
    }
  }
  b->nn_tot = nn;
  b->ne_tot = ne;
  cudaError_t e = cudaGetDevice(&b->dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, b->dev);
  auto A = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes > 0 ? bytes : 16);
  };
  A((void**)&b->d_inst, sizeof(BInst) * n);
  A((void**)&b->d_taps, sizeof(int) * b->taps.size());
  A((void**)&b->d_w, sizeof(double) * b->wts.size());
  A((void**)&b->rho, 8 * ne);
  A((void**)&b->rho_new, 8 * ne);
  A((void**)&b->E64, 8 * ne);
  A((void**)&b->E32, 4 * ne);
  A((void**)&b->dc, 8 * ne);
  A((void**)&b->dcf, 8 * ne);
  A((void**)&b->f, 8 * 2 * nn);
  A((void**)&b->x64, 8 * 2 * nn);
  A((void**)&b->inv32, 4 * 2 * nn);
  for (float** p : {&b->xl, &b->r, &b->z, &b->p0, &b->p1, &b->q}) A((void**)p, 4 * 2 * nn);
  A((void**)&b->mask, nn);
  A((void**)&b->flags, sizeof(unsigned) * 4);
  A((void**)&b->bar, sizeof(GridBar));
  A((void**)&b->out, sizeof(BOut) * n);
  b->npart = (size_t)16 * 152 * 16 + 64;
  A((void**)&b->part, 8 * b->npart);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_taps, b->taps.data(), sizeof(int) * b->taps.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_w, b->wts.data(), sizeof(double) * b->wts.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b->mask, 0, nn);
  if (e == cudaSuccess) e = cudaMemset(b->x64, 0, 8 * 2 * nn);
  if (e == cudaSuccess) e = cudaMemset(b->f, 0, 8 * 2 * nn);
  if (e == cudaSuccess) e = cudaEventCreate(&b->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&b->ev1);
  if (e == cudaSuccess) {
    // uniform initial density volfrac
    std::vector<double> rho(ne);
    for (int i = 0; i < n; i++)
      for (long long k = 0; k < b->inst[i].g.ne; k++) rho[b->inst[i].eoff + k] = params[i].volfrac;
    e = cudaMemcpy(b->rho, rho.data(), 8 * ne, cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    tp_batch_destroy(b);
    return e == cudaErrorMemoryAllocation ? TP_ERR_OOM : TP_ERR_CUDA;
  }
  if (plan(b) != TP_OK) {
    tp_batch_destroy(b);
    return TP_ERR_CUDA;
  }
  *out = b;
  return TP_OK;
}

void tp_batch_destroy(tp_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  void* ptrs[] = {b->d_inst, b->d_cta, b->d_taps, b->d_w, b->rho, b->rho_new, b->E64, b->E32, b->dc, b->dcf,
                  b->f, b->x64, b->inv32, b->xl, b->r, b->z, b->p0, b->p1, b->q, b->mask, b->flags, b->bar,
                  b->out, b->part};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  delete b;
}

const char* tp_batch_last_error(const tp_batch* b) { return b ? b->err.c_str() : "null batch"; }

tp_status tp_batch_set_fixed(tp_batch* b, int i, const uint8_t* fixed) {
  if (!b || !fixed || i < 0 || i >= b->n) return bfail(b, TP_ERR_ARG, "bad argument");
  const BInst& I = b->inst[i];
  std::vector<uint8_t> m(I.g.nn, 0);
  long long nf = 0;
  for (long long d = 0; d < 2 * I.g.nn; d++)
    if (fixed[d]) {
      m[d / 2] |= (uint8_t)(1u << (d % 2));
      nf++;
    }
  if (nf == 0) return bfail(b, TP_ERR_ARG, "no fixed DOF: the stiffness would be singular");
  BCK(cudaMemcpy(b->mask + I.noff, m.data(), I.g.nn, cudaMemcpyHostToDevice), "copy mask");
  b->have_fixed[i] = 1;
  b->have_loads[i] = 0;
  return TP_OK;
}

tp_status tp_batch_set_loads(tp_batch* b, int i, const double* fv) {
  if (!b || !fv || i < 0 || i >= b->n) return bfail(b, TP_ERR_ARG, "bad argument");
  if (!b->have_fixed[i]) return bfail(b, TP_ERR_STATE, "set the fixed DOFs of the instance first");
  const BInst& I = b->inst[i];
  std::vector<uint8_t> m(I.g.nn);
  BCK(cudaMemcpy(m.data(), b->mask + I.noff, I.g.nn, cudaMemcpyDeviceToHost), "copy mask");
  std::vector<double> planar(2 * I.g.nn);
  double s = 0.0;
  for (long long nd = 0; nd < I.g.nn; nd++)
    for (int c = 0; c < 2; c++) {
      double v = fv[2 * nd + c];
      if (!std::isfinite(v)) return bfail(b, TP_ERR_ARG, "loads contain NaN or Inf");
      if ((m[nd] >> c) & 1) v = 0.0;
      planar[c * I.g.nn + nd] = v;
      s += v * v;
    }
  if (!(s > 0.0)) return bfail(b, TP_ERR_ARG, "the instance has no load on free DOFs");
  b->ff[i] = s;
  BCK(cudaMemcpy(b->f + 2 * I.noff, planar.data(), 8 * 2 * I.g.nn, cudaMemcpyHostToDevice), "copy loads");
  b->have_loads[i] = 1;
  b->graph_ok = false;
  return TP_OK;
}

tp_status tp_batch_set_density(tp_batch* b, int i, const double* rho) {
  if (!b || !rho || i < 0 || i >= b->n) return bfail(b, TP_ERR_ARG, "bad argument");
  const BInst& I = b->inst[i];
  for (long long e = 0; e < I.g.ne; e++)
    if (!(rho[e] > 0.0 && rho[e] <= 1.0)) return bfail(b, TP_ERR_ARG, "densities must lie in (0, 1]");
  BCK(cudaMemcpy(b->rho + I.eoff, rho, 8 * I.g.ne, cudaMemcpyHostToDevice), "copy density");
  return TP_OK;
}

tp_status tp_batch_set_tiles(tp_batch* b, int tile_rows, int ctas_per_sm) {
  if (!b) return TP_ERR_ARG;
  if (tile_rows != 4 && tile_rows != 8 && tile_rows != 16) return bfail(b, TP_ERR_ARG, "tile_rows must be 4, 8 or 16");
  if (ctas_per_sm < 1 || ctas_per_sm > 8) return bfail(b, TP_ERR_ARG, "ctas_per_sm must lie in 1..8");
  b->tile_rows = tile_rows;
  b->ctas_per_sm = ctas_per_sm;
  return plan(b);
}

tp_status tp_batch_step(tp_batch* b, const tp_solve_opts* opts, tp_batch_info* info, double* compliance) {
  if (!b || !opts) return bfail(b, TP_ERR_ARG, "null argument");
  for (int i = 0; i < b->n; i++)
    if (!b->have_loads[i]) return bfail(b, TP_ERR_STATE, "every instance needs fixed DOFs and loads");
  if (!(opts->tol > 0.0) || opts->max_it < 1 || opts->precision != TP_PREC_MIXED)
    return bfail(b, TP_ERR_ARG, "batch solves use TP_PREC_MIXED with tol > 0 and max_it >= 1");
  for (int i = 0; i < b->n; i++) b->inst[i].tol2ff = opts->tol * opts->tol * b->ff[i];
  const bool same = b->graph_ok && memcmp(&b->gopts, opts, sizeof(*opts)) == 0;
  if (!same) {
    BCK(cudaMemcpy(b->d_inst, b->inst.data(), sizeof(BInst) * b->n, cudaMemcpyHostToDevice), "copy");
    if (b->gexec) {
      cudaGraphExecDestroy(b->gexec);
      b->gexec = nullptr;
    }
    b->graph_ok = false;
    // capture the step into a CUDA graph (replayed on later steps)
    cudaStream_t cs;
    BCK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "stream");
    cudaGraph_t gr = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    tp_status st = TP_OK;
    if (e == cudaSuccess) st = enqueue_step(b, cs, *opts);
    cudaError_t e2 = cudaStreamEndCapture(cs, &gr);
    if (e == cudaSuccess && st == TP_OK && e2 == cudaSuccess && gr) {
      if (cudaGraphInstantiate(&b->gexec, gr, 0) == cudaSuccess) b->graph_ok = true;
    }
    if (gr) cudaGraphDestroy(gr);
    cudaStreamDestroy(cs);
    cudaGetLastError();
    b->gopts = *opts;
  }
  BCK(cudaEventRecord(b->ev0, b->stream), "event");
  if (b->graph_ok) {
    BCK(cudaGraphLaunch(b->gexec, b->stream), "graph launch");
    b->launches += 6;
  } else {
    tp_status st = enqueue_step(b, b->stream, *opts);
    if (st != TP_OK) return st;
  }
  BCK(cudaEventRecord(b->ev1, b->stream), "event");
  std::vector<BOut> o(b->n);
  BCK(cudaMemcpyAsync(o.data(), b->out, sizeof(BOut) * b->n, cudaMemcpyDeviceToHost, b->stream), "copy");
  BCK(cudaStreamSynchronize(b->stream), "sync");
  float ms = 0.f;
  cudaEventElapsedTime(&ms, b->ev0, b->ev1);
  int maxit = 0, upd = 0, conv = 1, timeout = 0, brk = 0;
  double mrr = 0.0;
  for (int i = 0; i < b->n; i++) {
    maxit = std::max(maxit, o[i].iters);
    upd = std::max(upd, o[i].updates);
    conv &= o[i].state == 1;
    timeout |= o[i].state < 0 || (o[i].oc_flags & ERR_TIMEOUT);
    brk |= o[i].state == 2;
    mrr = std::max(mrr, std::sqrt(o[i].rr_true / b->ff[i]));
    if (compliance) compliance[i] = o[i].compliance;
  }
  if (info) {
    memset(info, 0, sizeof(*info));
    info->max_iters = maxit;
    info->updates = upd;
    info->converged = conv;
    info->max_rel_res = mrr;
    info->ms = ms;
    info->graph = b->graph_ok ? 1 : 0;
    info->tile_rows = b->tile_rows;
    info->ctas = b->grid;
  }
  if (timeout) return bfail(b, TP_ERR_TIMEOUT, "a device-side wait timed out in a batch kernel");
  if (brk) return bfail(b, TP_ERR_BREAKDOWN, "CG breakdown in an instance");
  if (!conv) return bfail(b, TP_ERR_NOT_CONVERGED, "an instance did not reach the tolerance");
  return TP_OK;
}

tp_status tp_batch_get(tp_batch* b, int i, int what, double* dst, double* scalars) {
  if (!b || i < 0 || i >= b->n || (!dst && !scalars)) return bfail(b, TP_ERR_ARG, "bad argument");
  const BInst& I = b->inst[i];
  BCK(cudaStreamSynchronize(b->stream), "sync");
  if (dst) {
    if (what == TP_RHO) {
      BCK(cudaMemcpy(dst, b->rho + I.eoff, 8 * I.g.ne, cudaMemcpyDeviceToHost), "copy");
    } else if (what == TP_DC) {
      BCK(cudaMemcpy(dst, b->dc + I.eoff, 8 * I.g.ne, cudaMemcpyDeviceToHost), "copy");
    } else if (what == TP_DCF) {
      BCK(cudaMemcpy(dst, b->dcf + I.eoff, 8 * I.g.ne, cudaMemcpyDeviceToHost), "copy");
    } else if (what == TP_U) {
      std::vector<double> pl(2 * I.g.nn);
      BCK(cudaMemcpy(pl.data(), b->x64 + 2 * I.noff, 8 * 2 * I.g.nn, cudaMemcpyDeviceToHost), "copy");
      for (long long nd = 0; nd < I.g.nn; nd++)
        for (int c = 0; c < 2; c++) dst[2 * nd + c] = pl[c * I.g.nn + nd];
    } else {
      return bfail(b, TP_ERR_ARG, "unknown quantity");
    }
  }
  if (scalars) {
    BOut o;
    BCK(cudaMemcpy(&o, b->out + i, sizeof(o), cudaMemcpyDeviceToHost), "copy");
    scalars[0] = o.compliance;
    scalars[1] = o.lambda;
    scalars[2] = o.volume;
    scalars[3] = o.change;
    scalars[4] = o.iters;
    scalars[5] = std::sqrt(o.rr_true / b->ff[i]);
  }
  return TP_OK;
}

long long tp_batch_launch_count(const tp_batch* b) { return b ? b->launches : 0; }

}  // extern "C"

// Autotuner: sweeps the tile height (4, 8, 16 node rows) and CTAs per SM (1, 2,
// 4) on this batch, timing a short CG on the current densities, and keeps the
// fastest.  Results are cached in a small JSON file keyed by the size class
// (instance count, total nodes rounded to 2 significant digits, SM count).
namespace {

std::string size_class(const tp_batch* b) {
  double v = (double)b->nn_tot;
  int e = 0;
  while (v >= 100.0) {
    v /= 10.0;
    e++;
  }
  char buf[128];
  snprintf(buf, sizeof(buf), "q4 n=%d nodes=%de%d sm=%d", b->n, (int)v, e, b->nsm);
  return buf;
}

bool cache_lookup(const char* path, const std::string& key, int* ty, int* cps) {
  if (!path) return false;
  FILE* fp = fopen(path, "r");
  if (!fp) return false;
  std::string txt;
  char buf[4096];
  size_t n;
  while ((n = fread(buf, 1, sizeof(buf), fp)) > 0) txt.append(buf, n);
  fclose(fp);
  const size_t k = txt.find("\"" + key + "\"");
  if (k == std::string::npos) return false;
  const size_t a = txt.find("\"tile_rows\":", k), c = txt.find("\"ctas_per_sm\":", k);
  if (a == std::string::npos || c == std::string::npos) return false;
  *ty = atoi(txt.c_str() + a + 12);
  *cps = atoi(txt.c_str() + c + 14);
  return (*ty == 4 || *ty == 8 || *ty == 16) && *cps >= 1 && *cps <= 8;
}

void cache_store(const char* path, const std::string& key, int ty, int cps, double us) {
  if (!path) return;
  std::string txt;
  if (FILE* fp = fopen(path, "r")) {
    char buf[4096];
    size_t n;
    while ((n = fread(buf, 1, sizeof(buf), fp)) > 0) txt.append(buf, n);
    fclose(fp);
  }
  // keep the other entries (one per line), replace this key
  std::vector<std::string> lines;
  size_t pos = 0;
  while (pos < txt.size()) {
    size_t e = txt.find('\n', pos);
    if (e == std::string::npos) e = txt.size();
    std::string ln = txt.substr(pos, e - pos);
    if (ln.find("\"tile_rows\"") != std::string::npos && ln.find("\"" + key + "\"") == std::string::npos) {
      while (!ln.empty() && (ln.back() == ',' || ln.back() == ' ')) ln.pop_back();
      lines.push_back(ln);
    }
    pos = e + 1;
  }
  char buf[512];
  snprintf(buf, sizeof(buf), "  \"%s\": {\"tile_rows\": %d, \"ctas_per_sm\": %d, \"us_per_iter\": %.3f}", key.c_str(),
           ty, cps, us);
  lines.push_back(buf);
  FILE* fp = fopen(path, "w");
  if (!fp) return;
  fprintf(fp, "{\n");
  for (size_t i = 0; i < lines.size(); i++) fprintf(fp, "%s%s\n", lines[i].c_str(), i + 1 < lines.size() ? "," : "");
  fprintf(fp, "}\n");
  fclose(fp);
}

// Time `iters` CG iterations (no FP64 update triggers) on the current state.
tp_status time_cg(tp_batch* b, int iters, double* us_per_iter) {
  tp_solve_opts o{};
  o.tol = 1e-300;
  o.max_it = iters;
  o.precision = TP_PREC_MIXED;
  o.warm_start = TP_WARM_PREVIOUS;
  o.update_drop = 1e-300;
  const long long nn = b->nn_tot;
  double* save = nullptr;
  BCK(cudaMalloc((void**)&save, 8 * 2 * nn), "alloc");
  cudaError_t e = cudaMemcpyAsync(save, b->x64, 8 * 2 * nn, cudaMemcpyDeviceToDevice, b->stream);
  for (int i = 0; i < b->n && e == cudaSuccess; i++) b->inst[i].tol2ff = 1e-300;
  if (e == cudaSuccess) e = cudaMemcpy(b->d_inst, b->inst.data(), sizeof(BInst) * b->n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaEventRecord(b->ev0, b->stream);
  BCgArgs a;
  memset(&a, 0, sizeof(a));
  a.in = b->d_inst;
  a.cta_inst = b->d_cta;
  a.ninst = b->n;
  a.E32 = b->E32;
  a.E64 = b->E64;
  a.mask = b->mask;
  a.inv32 = b->inv32;
  a.f = b->f;
  a.x64 = b->x64;
  a.xl = b->xl;
  a.r = b->r;
  a.z = b->z;
  a.p0 = b->p0;
  a.p1 = b->p1;
  a.q = b->q;
  a.part = b->part;
  a.flags = b->flags;
  a.bar = b->bar;
  a.out = b->out;
  a.drop2 = 0.0;
  a.max_it = o.max_it;
  fill_c<2, float>(a.Cf, b->C.data());
  fill_c<2, double>(a.Cd, b->C.data());
  if (e == cudaSuccess) e = cudaMemsetAsync(b->xl, 0, sizeof(float) * 2 * nn, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->bar, 0, sizeof(GridBar), b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->flags, 0, sizeof(unsigned) * 4, b->stream);
  const int ty = b->tile_rows;
  const size_t smem = cg_smem(ty);
  if (e == cudaSuccess)
    e = ty == 4 ? launch_batch_cg_ty<4>(b, b->stream, a, smem)
                : ty == 8 ? launch_batch_cg_ty<8>(b, b->stream, a, smem) : launch_batch_cg_ty<16>(b, b->stream, a, smem);
  if (e == cudaSuccess) e = cudaEventRecord(b->ev1, b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->x64, save, 8 * 2 * nn, cudaMemcpyDeviceToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  cudaFree(save);
  BCK(e, "autotune timing");
  float ms = 0.f;
  cudaEventElapsedTime(&ms, b->ev0, b->ev1);
  *us_per_iter = 1000.0 * ms / iters;
  b->graph_ok = false;
  return TP_OK;
}

}  // namespace

extern "C" tp_status tp_batch_autotune(tp_batch* b, const char* cache_path, int* tile_rows, int* ctas_per_sm) {
  if (!b) return TP_ERR_ARG;
  for (int i = 0; i < b->n; i++)
    if (!b->have_loads[i]) return bfail(b, TP_ERR_STATE, "every instance needs fixed DOFs and loads");
  const std::string key = size_class(b);
  int ty = 0, cps = 0;
  if (!cache_lookup(cache_path, key, &ty, &cps)) {
    // moduli / diagonal of the current densities for the timing runs
    tp_solve_opts o{1e-6, 1, TP_PREC_MIXED, TP_WARM_PREVIOUS, 0.1};
    (void)o;
    const long long ne = b->ne_tot, nn = b->nn_tot;
    batch_young_kernel<<<bgrid(ne), 256, 0, b->stream>>>(b->d_inst, b->n, ne, b->rho, b->E32, b->E64);
    BDiagArgs da;
    da.in = b->d_inst;
    da.n = b->n;
    da.nn_tot = nn;
    da.E64 = b->E64;
    da.mask = b->mask;
    da.inv32 = b->inv32;
    for (int i = 0; i < 8; i++) da.kd[i] = b->K0[i * 8 + i];
    batch_diag_kernel<<<bgrid(nn), 256, 0, b->stream>>>(da);
    BCK(cudaGetLastError(), "autotune moduli");
    double best = 1e300;
    for (int t : {4, 8, 16})
      for (int c : {1, 2, 4}) {
        if (tp_batch_set_tiles(b, t, c) != TP_OK) continue;
        double us = 0.0;
        if (time_cg(b, 30, &us) != TP_OK) continue;  // warm-up
        if (time_cg(b, 100, &us) != TP_OK) continue;
        if (us < best) {
          best = us;
          ty = t;
          cps = c;
        }
      }
    if (ty == 0) return bfail(b, TP_ERR_CUDA, "autotune found no runnable configuration");
    cache_store(cache_path, key, ty, cps, best);
  }
  tp_status s = tp_batch_set_tiles(b, ty, cps);
  if (s != TP_OK) return s;
  if (tile_rows) *tile_rows = ty;
  if (ctas_per_sm) *ctas_per_sm = cps;
  return TP_OK;
}

