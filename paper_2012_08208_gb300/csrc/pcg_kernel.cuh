// One segment of the persistent Jacobi-preconditioned CG (cooperative launch).
//
// All load cases advance in lock-step.  Per iteration two grid barriers:
//   phase A  p = z + beta p_old (formed while the tile operator loads its
//            input), q = K p, partial p.q                        -> barrier
//   phase B  x_l += alpha p, r -= alpha q, z = D^-1 r, partial r.z, r.r
//                                                                 -> barrier
// The segment returns when a case's recurrence residual has dropped by
// `drop` since the last FP64 update or has reached the tolerance (an update is
// due), or at max_it.  The host then runs the FP64 true-residual update
// (fem_kernels.cu), which replaces r by f - K64 x64 and sets the next beta;
// the search direction is kept (reliable update).
#pragma once
#include "pcg_common.cuh"

namespace tp {

constexpr int SLOT_A = 0;   // NCM partials: p.q
constexpr int SLOT_B = 8;   // 2 NCM partials: r.z, r.r

template <int DIM, typename T>
struct SegArgs {
  Grid g;
  TileMapG tm;
  int nc, nv;
  const T* E;
  const uint8_t* mask;
  const T* invd;
  T* xl;
  T* r;
  T* z;
  T* p0;
  T* p1;
  T* q;
  double* part;
  GridBar* bar;
  CgState* cs;
  double tol2ff[kMaxCases];
  double drop2;
  int max_it;
  CMat<DIM, T> C;
};

constexpr size_t kSegHeader = 32 * 16 * sizeof(double) + 32 * sizeof(double);

// CTA partial / grid total in the precision policy of the CG type: double-float
// accumulation for FP32 data, FP64 for FP64 data.  Slots hold 8 bytes per value.
template <int NV, typename T>
__device__ __forceinline__ void cta_partial(T (&v)[NV], double* slot, unsigned char* sm) {
  if constexpr (std::is_same<T, float>::value) block_partial_f<NV>(v, reinterpret_cast<float2*>(slot), sm);
  else block_partial_d<NV>(v, slot, sm);
}
template <int NV>
__device__ __forceinline__ void cta_total_any(const double* slot, double (&out)[NV], unsigned char* sm, bool f32) {
  if (f32) grid_total_f<NV>(reinterpret_cast<const float2*>(slot), out, sm);
  else grid_total_d<NV>(slot, out, sm);
}

template <int DIM, typename T, int NCM>
__global__ void __launch_bounds__(TileOp<DIM, T>::THREADS)
    cg_segment_kernel(const __grid_constant__ SegArgs<DIM, T> a) {
  using Op = TileOp<DIM, T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sCoef = reinterpret_cast<T*>(smem_raw + 32 * 16 * sizeof(double));  // beta[8] | alpha[8]
  int* sAct = reinterpret_cast<int*>(smem_raw + 32 * 16 * sizeof(double) + 16 * sizeof(double));
  unsigned char* sTile = smem_raw + kSegHeader;
  const int nc = a.nc, nv = a.nv, nb = gridDim.x;

  int it = a.cs->it, pbuf = a.cs->pbuf;
  int state[NCM];
  double rz[NCM], rr_ref[NCM], beta[NCM], alpha[NCM];
#pragma unroll
  for (int c = 0; c < NCM; c++) {
    state[c] = c < nc ? a.cs->state[c] : 1;
    rz[c] = a.cs->rz[c];
    rr_ref[c] = a.cs->rr_ref[c];
    beta[c] = a.cs->beta[c];
    alpha[c] = 0.0;
  }
  unsigned gen = 0;
  bool ok = true, need = false;
  int flags = 0;
  auto publish = [&]() {
    __syncthreads();
    if (threadIdx.x < NCM) {
      sCoef[threadIdx.x] = (T)pick(beta, threadIdx.x);
      sCoef[kMaxCases + threadIdx.x] = (T)pick(alpha, threadIdx.x);
      sAct[threadIdx.x] = pick(state, threadIdx.x) == 0;
    }
    __syncthreads();
  };

  while (it < a.max_it) {
    bool any = false;
#pragma unroll
    for (int c = 0; c < NCM; c++) any |= state[c] == 0;
    if (!any) break;
    publish();

    // ---- phase A
    const T* Pold = pbuf ? a.p1 : a.p0;
    T* Pnew = pbuf ? a.p0 : a.p1;
    // per-thread partial sums in the CG precision; FP64 from the block level on
    T accAt[NCM];
#pragma unroll
    for (int i = 0; i < NCM; i++) accAt[i] = T(0);
    for (int t = blockIdx.x; t < a.tm.ntiles; t += nb) {
      for (int cs = 0; cs < nc; cs++) {
        if (!sAct[cs]) continue;
        const T b = sCoef[cs];
        T spq = T(0);
        Op::apply(
            a.g, a.tm, t, a.E, a.C, sTile,
            [&](long long node, int comp, bool own) -> T {
              const long long idx = node * nv + cs * DIM + comp;
              T v = __ldcg(a.z + idx);
              if (b != T(0)) v = fma(b, __ldcg(Pold + idx), v);
              if (own) Pnew[idx] = v;
              return v;
            },
            [&](long long node, const T(&yv)[DIM], const T(&us)[DIM]) {
              const uint8_t mk = a.mask[node];
#pragma unroll
              for (int r = 0; r < DIM; r++) {
                const T qv = ((mk >> r) & 1) ? T(0) : yv[r];
                a.q[node * nv + cs * DIM + r] = qv;
                spq = fma(us[r], qv, spq);
              }
            });
#pragma unroll
        for (int c2 = 0; c2 < NCM; c2++)
          if (c2 == cs) accAt[c2] += spq;
      }
    }
    cta_partial<NCM>(accAt, a.part + (size_t)SLOT_A * nb, smem_raw);
    if (!(ok = grid_sync(a.bar, gen))) break;
    {
      double pq[NCM];
      cta_total_any<NCM>(a.part + (size_t)SLOT_A * nb, pq, smem_raw, std::is_same<T, float>::value);
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

    // ---- phase B (one node per thread, all cases and components of the node)
    T accBt[2 * NCM];
#pragma unroll
    for (int i = 0; i < 2 * NCM; i++) accBt[i] = T(0);
    const long long nn = a.g.nn;
    for (long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x; node < nn;
         node += (long long)nb * blockDim.x) {
      T inv[DIM];
#pragma unroll
      for (int r = 0; r < DIM; r++) inv[r] = __ldg(a.invd + node * DIM + r);
#pragma unroll
      for (int cs = 0; cs < NCM; cs++) {
        if (cs >= nc) break;
        const T al = sCoef[kMaxCases + cs];
#pragma unroll
        for (int r = 0; r < DIM; r++) {
          const long long i = node * nv + cs * DIM + r;
          T rv = __ldcg(a.r + i);
          T zv;
          if (al != T(0)) {
            const T pv = __ldcg(Pnew + i), qv = __ldcg(a.q + i);
            a.xl[i] = fma(al, pv, a.xl[i]);
            rv = fma(-al, qv, rv);
            a.r[i] = rv;
            zv = rv * inv[r];
            a.z[i] = zv;
          } else {
            zv = __ldcg(a.z + i);
          }
          accBt[cs] = fma(rv, zv, accBt[cs]);
          accBt[NCM + cs] = fma(rv, rv, accBt[NCM + cs]);
        }
      }
    }
    cta_partial<2 * NCM>(accBt, a.part + (size_t)SLOT_B * nb, smem_raw);
    if (!(ok = grid_sync(a.bar, gen))) break;
    double rzn[NCM], rr[NCM];
    {
      double tot[2 * NCM];
      cta_total_any<2 * NCM>(a.part + (size_t)SLOT_B * nb, tot, smem_raw, std::is_same<T, float>::value);
#pragma unroll
      for (int c = 0; c < NCM; c++) {
        rzn[c] = tot[c];
        rr[c] = tot[NCM + c];
      }
    }
    it++;
    pbuf ^= 1;
#pragma unroll
    for (int c = 0; c < NCM; c++)
      if (state[c] == 0 && (rr[c] <= a.tol2ff[c] || rr[c] <= a.drop2 * rr_ref[c])) need = true;
    if (need) break;  // rz keeps the value the finalize step divides by
#pragma unroll
    for (int c = 0; c < NCM; c++) {
      beta[c] = (state[c] == 0 && rz[c] != 0.0) ? rzn[c] / rz[c] : 0.0;
      rz[c] = rzn[c];
    }
  }
  if (!ok) flags |= ERR_TIMEOUT;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.cs->it = it;
    a.cs->pbuf = pbuf;
    a.cs->need = need ? 1 : 0;
    a.cs->flags |= flags;
#pragma unroll
    for (int c = 0; c < NCM; c++) {
      if (c < nc) a.cs->state[c] = state[c];
      a.cs->rz[c] = rz[c];
      a.cs->beta[c] = beta[c];
    }
  }
}

template <int DIM, typename T, int NCM>
static cudaError_t segment_impl(cudaStream_t s, const Solver& S, int nsm, int* grid_out) {
  using Op = TileOp<DIM, T>;
  SegArgs<DIM, T> a;
  a.g = S.g;
  a.tm = Op::map(S.g, S.zlen);
  a.nc = S.nc;
  a.nv = S.nc * DIM;
  a.E = (const T*)S.E;
  a.mask = S.mask;
  a.invd = (const T*)S.invdiag;
  a.xl = (T*)S.xl;
  a.r = (T*)S.r;
  a.z = (T*)S.z;
  a.p0 = (T*)S.p0;
  a.p1 = (T*)S.p1;
  a.q = (T*)S.q;
  a.part = S.part;
  a.bar = S.bar;
  a.cs = S.cs;
  for (int c = 0; c < kMaxCases; c++) a.tol2ff[c] = S.tol2ff[c];
  a.drop2 = S.drop2;
  a.max_it = S.max_it;
  fill_c<DIM, T>(a.C, S.C);
  const size_t smem = kSegHeader + Op::smem_bytes();
  auto kern = cg_segment_kernel<DIM, T, NCM>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Op::THREADS, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int grid = per_sm * nsm;
  if (grid > a.tm.ntiles) grid = a.tm.ntiles;
  if (grid < 1) grid = 1;
  *grid_out = grid;
  void* args[] = {(void*)&a};
  return cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(Op::THREADS), args, smem, s);
}

template <int DIM, typename T>
static cudaError_t segment_nc(cudaStream_t s, const Solver& S, int nsm, int* grid_out) {
  if (S.nc == 1) return segment_impl<DIM, T, 1>(s, S, nsm, grid_out);
  if (S.nc <= 4) return segment_impl<DIM, T, 4>(s, S, nsm, grid_out);
  return segment_impl<DIM, T, 8>(s, S, nsm, grid_out);
}

}  // namespace tp
