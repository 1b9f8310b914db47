// Persistent Jacobi-preconditioned CG kernel (one cooperative launch per solve).
#pragma once
#include "tile.cuh"

namespace tp {

// ---------------------------------------------------------------------------
// Persistent Jacobi-PCG over all load cases.
//
// Per iteration two grid barriers:
//   phase A  p = z + beta p_old (formed while loading the halo tile), q = K p,
//            partial p.q                                         -> barrier
//   phase B  x_l += alpha p, r -= alpha q, z = D^-1 r, partial r.z and r.r
//                                                                   -> barrier
// Reliable update (FP64): when a case's recurrence residual has dropped by
// `drop` since the last update, or has reached the tolerance, x64 += x_l and
// r = f - K64 x64 is recomputed in FP64 (its norm is the true residual that
// decides convergence); the search direction is kept.

template <int DIM, typename T>
struct PcgArgs {
  Grid g;
  TileMap<DIM> tm;
  int nc, nv;
  const T* E;
  const double* E64;
  const uint8_t* mask;
  const T* invd;
  const double* f;
  double* x64;
  T* xl;
  T* r;
  T* z;
  T* p0;
  T* p1;
  T* q;
  double* part;
  GridBar* bar;
  PcgStatus* st;
  double tol2ff[kMaxCases];
  double drop2;
  int max_it;
  KMat<DIM, T> kT;
  KMat<DIM, double> kD;
};

// partial-sum slots in `part` (each slot holds gridDim.x doubles)
constexpr int SLOT_RES = 0;   // 16: rr_true[8], rz[8]
constexpr int SLOT_A = 16;    // 8: pq[8]
constexpr int SLOT_B = 24;    // 16: rz[8], rr[8]
constexpr int kPartSlots = 40;
constexpr int kStallUpdates = 6;  // updates without progress before a case stops

template <int DIM, typename T, int NCM>
__global__ void __launch_bounds__(kThreads) pcg_kernel(const __grid_constant__ PcgArgs<DIM, T> a) {
  using G = TileGeom<DIM>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sRed = reinterpret_cast<double*>(smem_raw);  // 32 * 16 doubles
  T* sCoef = reinterpret_cast<T*>(smem_raw + 32 * 16 * sizeof(double));  // beta[8] | alpha[8]
  int* sAct = reinterpret_cast<int*>(smem_raw + 32 * 16 * sizeof(double) + 16 * sizeof(double));
  unsigned char* sTile = smem_raw + 32 * 16 * sizeof(double) + 32 * sizeof(double);
  const int nc = a.nc, nv = a.nv;
  const long long nvals = a.g.nn * nv;
  const int nb = gridDim.x;
  unsigned gen = 0;
  bool ok = true;

  // Per-case scalars; every thread holds identical copies (computed from the
  // same deterministic grid totals), indexed with compile-time indices only.
  int state[NCM];
  double rz[NCM], rr_ref[NCM], beta[NCM], alpha[NCM], rr_true[NCM];
  int stall[NCM];
#pragma unroll
  for (int c = 0; c < NCM; c++) {
    state[c] = c < nc ? 0 : 1;
    rz[c] = rr_ref[c] = beta[c] = alpha[c] = rr_true[c] = 0.0;
    stall[c] = 0;
  }
  auto publish = [&]() {  // block-uniform coefficients to shared memory
    __syncthreads();
    if (threadIdx.x < NCM) {
      sCoef[threadIdx.x] = (T)pick(beta, threadIdx.x);
      sCoef[NCM + threadIdx.x] = (T)pick(alpha, threadIdx.x);
      sAct[threadIdx.x] = pick(state, threadIdx.x) == 0;
    }
    __syncthreads();
  };

  // r = f - K64 x64 (FP64), z = D^-1 r; totals: rr_true, rz.
  auto residual_phase = [&](double (&rrt)[NCM], double (&rzo)[NCM]) -> bool {
    double acc[2 * NCM];
#pragma unroll
    for (int i = 0; i < 2 * NCM; i++) acc[i] = 0.0;
    double* sX = reinterpret_cast<double*>(sTile);
    double* sE = sX + G::HN * nv;
    for (int t = blockIdx.x; t < a.tm.ntiles; t += nb) {
      int x0, y0, z0;
      tile_origin<DIM>(a.tm, t, x0, y0, z0);
      load_E<DIM, double>(a.g, x0, y0, z0, a.E64, sE);
      load_halo<DIM, double>(a.g, x0, y0, z0, nv, sX, [&](long long node, int v, bool) -> double {
        const int comp = v % DIM;
        return ((a.mask[node] >> comp) & 1) ? 0.0 : __ldcg(a.x64 + node * nv + v);
      });
      __syncthreads();
      for (int ln = threadIdx.x; ln < G::TN; ln += blockDim.x) {
        int tx, ty, tz;
        long long node;
        if (!own_node<DIM>(a.g, ln, x0, y0, z0, tx, ty, tz, node)) continue;
        const uint8_t mk = a.mask[node];
        for (int cs = 0; cs < nc; cs++) {
          double kx[DIM];
          node_apply<DIM, double>(sX, sE, nv, cs, tx, ty, tz, a.kD, kx);
          double srr = 0.0, srz = 0.0;
#pragma unroll
          for (int r = 0; r < DIM; r++) {
            const long long idx = node * nv + cs * DIM + r;
            const double r64 = ((mk >> r) & 1) ? 0.0 : __ldg(a.f + idx) - kx[r];
            const T rt = (T)r64;
            const T zt = rt * __ldg(a.invd + node * DIM + r);
            a.r[idx] = rt;
            a.z[idx] = zt;
            srr += r64 * r64;
            srz += (double)rt * (double)zt;
          }
          addto<2 * NCM>(acc, cs, srr);
          addto<2 * NCM>(acc, NCM + cs, srz);
        }
      }
      __syncthreads();
    }
    block_sum<2 * NCM>(acc, sRed);
    if (threadIdx.x == 0)
      for (int i = 0; i < 2 * NCM; i++) a.part[(size_t)(SLOT_RES + i) * nb + blockIdx.x] = acc[i];
    if (!grid_sync(a.bar, gen)) return false;
    double tot[2 * NCM];
    grid_total<2 * NCM>(a.part + (size_t)SLOT_RES * nb, tot, sRed);
#pragma unroll
    for (int c = 0; c < NCM; c++) {
      rrt[c] = tot[c];
      rzo[c] = tot[NCM + c];
    }
    return true;
  };

  // x64 += x_l, x_l = 0
  auto merge_phase = [&]() -> bool {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nvals;
         i += (long long)nb * blockDim.x) {
      const T v = a.xl[i];
      a.x64[i] = __ldcg(a.x64 + i) + (double)v;
      a.xl[i] = T(0);
    }
    return grid_sync(a.bar, gen);
  };

  int it = 0, updates = 0, flags = 0;
  bool fresh = true;  // x_l merged and r is the true residual
  ok = residual_phase(rr_true, rz);
  if (ok) {
#pragma unroll
    for (int c = 0; c < NCM; c++) {
      rr_ref[c] = rr_true[c];
      if (c < nc && rr_true[c] <= a.tol2ff[c]) state[c] = 1;
    }
  }

  while (ok && it < a.max_it) {
    bool any = false;
#pragma unroll
    for (int c = 0; c < NCM; c++) any |= state[c] == 0;
    if (!any) break;
    publish();

    // ---- phase A: p = z + beta p_old, q = K p, partial p.q
    const T* Pold = (it & 1) ? a.p1 : a.p0;
    T* Pnew = (it & 1) ? a.p0 : a.p1;
    double accA[NCM];
#pragma unroll
    for (int i = 0; i < NCM; i++) accA[i] = 0.0;
    {
      T* sP = reinterpret_cast<T*>(sTile);
      T* sE = sP + G::HN * nv;
      for (int t = blockIdx.x; t < a.tm.ntiles; t += nb) {
        int x0, y0, z0;
        tile_origin<DIM>(a.tm, t, x0, y0, z0);
        load_E<DIM, T>(a.g, x0, y0, z0, a.E, sE);
        load_halo<DIM, T>(a.g, x0, y0, z0, nv, sP, [&](long long node, int v, bool own) -> T {
          const long long idx = node * nv + v;
          const T b = sCoef[v / DIM];
          T val = __ldcg(a.z + idx);
          if (b != T(0)) val = fma(b, __ldcg(Pold + idx), val);
          if (own) Pnew[idx] = val;
          return val;
        });
        __syncthreads();
        for (int ln = threadIdx.x; ln < G::TN; ln += blockDim.x) {
          int tx, ty, tz;
          long long node;
          if (!own_node<DIM>(a.g, ln, x0, y0, z0, tx, ty, tz, node)) continue;
          const uint8_t mk = a.mask[node];
          const int hself = (((DIM == 3 ? tz + 1 : 0) * G::HY + ty + 1) * G::HX + tx + 1) * nv;
          for (int cs = 0; cs < nc; cs++) {
            if (!sAct[cs]) continue;
            T kq[DIM];
            node_apply<DIM, T>(sP, sE, nv, cs, tx, ty, tz, a.kT, kq);
            double spq = 0.0;
#pragma unroll
            for (int r = 0; r < DIM; r++) {
              const T qv = ((mk >> r) & 1) ? T(0) : kq[r];
              a.q[node * nv + cs * DIM + r] = qv;
              spq += (double)sP[hself + cs * DIM + r] * (double)qv;
            }
            addto<NCM>(accA, cs, spq);
          }
        }
        __syncthreads();
      }
    }
    block_sum<NCM>(accA, sRed);
    if (threadIdx.x == 0)
      for (int i = 0; i < NCM; i++) a.part[(size_t)(SLOT_A + i) * nb + blockIdx.x] = accA[i];
    if (!(ok = grid_sync(a.bar, gen))) break;
    {
      double pq[NCM];
      grid_total<NCM>(a.part + (size_t)SLOT_A * nb, pq, sRed);
#pragma unroll
      for (int c = 0; c < NCM; c++) {
        alpha[c] = 0.0;
        if (state[c] != 0) continue;
        if (!(pq[c] > 0.0) || !isfinite(pq[c]) || !isfinite(rz[c])) {
          state[c] = 2;
          flags |= ERR_BREAKDOWN;
          continue;
        }
        alpha[c] = rz[c] / pq[c];
      }
    }
    publish();

    // ---- phase B: x_l += alpha p, r -= alpha q, z = D^-1 r, partial r.z, r.r
    double accB[2 * NCM];
#pragma unroll
    for (int i = 0; i < 2 * NCM; i++) accB[i] = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nvals;
         i += (long long)nb * blockDim.x) {
      const long long node = i / nv;
      const int v = (int)(i - node * nv);
      const int cs = v / DIM, comp = v - cs * DIM;
      const T al = sCoef[NCM + cs];
      T rv = __ldcg(a.r + i);
      T zv;
      if (al != T(0)) {
        const T pv = __ldcg(Pnew + i), qv = __ldcg(a.q + i);
        a.xl[i] = fma(al, pv, a.xl[i]);
        rv = fma(-al, qv, rv);
        a.r[i] = rv;
        zv = rv * __ldg(a.invd + node * DIM + comp);
        a.z[i] = zv;
      } else {
        zv = __ldcg(a.z + i);
      }
      addto<2 * NCM>(accB, cs, (double)rv * (double)zv);
      addto<2 * NCM>(accB, NCM + cs, (double)rv * (double)rv);
    }
    block_sum<2 * NCM>(accB, sRed);
    if (threadIdx.x == 0)
      for (int i = 0; i < 2 * NCM; i++) a.part[(size_t)(SLOT_B + i) * nb + blockIdx.x] = accB[i];
    if (!(ok = grid_sync(a.bar, gen))) break;
    double rzn[NCM], rr[NCM];
    {
      double tot[2 * NCM];
      grid_total<2 * NCM>(a.part + (size_t)SLOT_B * nb, tot, sRed);
#pragma unroll
      for (int c = 0; c < NCM; c++) {
        rzn[c] = tot[c];
        rr[c] = tot[NCM + c];
      }
    }
    it++;
    fresh = false;

    bool need = false;
#pragma unroll
    for (int c = 0; c < NCM; c++)
      if (state[c] == 0 && (rr[c] <= a.tol2ff[c] || rr[c] <= a.drop2 * rr_ref[c])) need = true;
    if (need) {
      if (!(ok = merge_phase())) break;
      if (!(ok = residual_phase(rr_true, rzn))) break;
      updates++;
      fresh = true;
#pragma unroll
      for (int c = 0; c < NCM; c++) {
        if (state[c] != 0) continue;
        // stagnation: the true residual no longer halves between updates
        stall[c] = rr_true[c] > 0.25 * rr_ref[c] ? stall[c] + 1 : 0;
        rr_ref[c] = rr_true[c];
        if (rr_true[c] <= a.tol2ff[c]) state[c] = 1;
        else if (stall[c] >= kStallUpdates) state[c] = 3;
      }
    }
#pragma unroll
    for (int c = 0; c < NCM; c++) {
      beta[c] = (state[c] == 0 && rz[c] != 0.0) ? rzn[c] / rz[c] : 0.0;
      rz[c] = rzn[c];
    }
  }
  if (ok && !fresh) {
    ok = merge_phase();
    if (ok) {
      double dummy[NCM];
      ok = residual_phase(rr_true, dummy);
      updates++;
    }
    if (ok) {
#pragma unroll
      for (int c = 0; c < NCM; c++)
        if (state[c] == 0 && rr_true[c] <= a.tol2ff[c]) state[c] = 1;
    }
  }
  if (!ok) flags |= ERR_TIMEOUT;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.st->iters = it;
    a.st->updates = updates;
    a.st->flags = flags;
    for (int c = 0; c < NCM; c++) {
      a.st->state[c] = state[c];
      a.st->rr_true[c] = rr_true[c];
    }
    for (int c = NCM; c < kMaxCases; c++) {
      a.st->state[c] = 1;
      a.st->rr_true[c] = 0.0;
    }
  }
}

template <int DIM, typename T, int NCM>
static cudaError_t pcg_impl(cudaStream_t s, const PcgLaunch& L, int nsm, int* grid_out) {
  using G = TileGeom<DIM>;
  PcgArgs<DIM, T> a;
  a.g = L.g;
  a.tm = tile_map<DIM>(L.g);
  a.nc = L.nc;
  a.nv = L.nc * DIM;
  a.E = (const T*)L.E;
  a.E64 = L.E64;
  a.mask = L.mask;
  a.invd = (const T*)L.invdiag;
  a.f = L.f;
  a.x64 = L.x64;
  a.xl = (T*)L.xl;
  a.r = (T*)L.r;
  a.z = (T*)L.z;
  a.p0 = (T*)L.p0;
  a.p1 = (T*)L.p1;
  a.q = (T*)L.q;
  a.part = L.part;
  a.bar = L.bar;
  a.st = L.st;
  for (int c = 0; c < kMaxCases; c++) a.tol2ff[c] = L.tol2ff[c];
  a.drop2 = L.drop2;
  a.max_it = L.max_it;
  fill_k<DIM, T>(a.kT, L.K0);
  fill_k<DIM, double>(a.kD, L.K0);
  const size_t tile_bytes = (size_t)(G::HN * a.nv + G::EN) * sizeof(double);
  const size_t smem = 32 * 16 * sizeof(double) + 32 * sizeof(double) + tile_bytes;
  auto kern = pcg_kernel<DIM, T, NCM>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int grid = per_sm * nsm;
  if (grid > a.tm.ntiles) grid = a.tm.ntiles;
  if (grid < 1) grid = 1;
  *grid_out = grid;
  void* args[] = {(void*)&a};
  return cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(kThreads), args, smem, s);
}

template <int DIM, typename T>
static cudaError_t pcg_nc(cudaStream_t s, const PcgLaunch& L, int nsm, int* grid_out) {
  if (L.nc == 1) return pcg_impl<DIM, T, 1>(s, L, nsm, grid_out);
  if (L.nc <= 4) return pcg_impl<DIM, T, 4>(s, L, nsm, grid_out);
  return pcg_impl<DIM, T, 8>(s, L, nsm, grid_out);
}

}  // namespace tp
