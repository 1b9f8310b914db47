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
  long long* trace;  // optional: per-iteration timestamps of CTA 0 (kTraceIters x 4)
  CMat<DIM, T> C;
};

constexpr int kTraceIters = 32;
constexpr int kTracePts = 8;
__device__ __forceinline__ long long globaltimer() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Shared-memory layout of the segment kernel: reduction scratch, then the
// per-case control block (owned by thread 0; FP64 scalar work stays off the
// other threads), then the tile operator's buffers.
struct SegCtl {
  double rz[kMaxCases], rr_ref[kMaxCases], beta[kMaxCases], alpha[kMaxCases];
  double tot[2 * kMaxCases];
  float coef_f[2 * kMaxCases];   // beta | alpha in FP32
  double coef_d[2 * kMaxCases];  // beta | alpha in FP64
  int state[kMaxCases];
  int act[kMaxCases];
  int it, pbuf, need, go, flags;
};
constexpr size_t kRedBytes = 32 * 16 * sizeof(double);
constexpr size_t kSegHeader = kRedBytes + ((sizeof(SegCtl) + 255) / 256) * 256;

// CTA partial / grid total in the precision policy of the CG type: double-float
// accumulation for FP32 data, FP64 for FP64 data.  Slots hold 8 bytes per value.
// The total lands in ctl->tot (read by thread 0 after a barrier).
template <int NV, typename T>
__device__ __forceinline__ void cta_partial(T (&v)[NV], double* slot, unsigned char* sm) {
  if constexpr (std::is_same<T, float>::value) block_partial_f<NV>(v, reinterpret_cast<float2*>(slot), sm);
  else block_partial_d<NV>(v, slot, sm);
}
template <int NV, typename T>
__device__ __forceinline__ void cta_total(const double* slot, SegCtl* ctl) {
  // one warp per value; each lane loads its share of the per-CTA partials in
  // batches of 8 independent loads, then accumulates in a fixed order
  constexpr int kB = 8;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nb = gridDim.x;
  for (int i = warp; i < NV; i += nw) {
    if constexpr (std::is_same<T, float>::value) {
      const float2* part = reinterpret_cast<const float2*>(slot) + (size_t)i * nb;
      dfl s{0.f, 0.f};
      for (int b0 = 0; b0 < nb; b0 += 32 * kB) {
        float2 buf[kB];
#pragma unroll
        for (int j = 0; j < kB; j++) {
          const int b = b0 + j * 32 + lane;
          buf[j] = b < nb ? __ldcg(part + b) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int j = 0; j < kB; j++) s = dfl_add(s, dfl{buf[j].x, buf[j].y});
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const dfl t{__shfl_xor_sync(0xffffffffu, s.hi, o), __shfl_xor_sync(0xffffffffu, s.lo, o)};
        s = dfl_add(s, t);
      }
      if (lane == 0) ctl->tot[i] = (double)s.hi + (double)s.lo;
    } else {
      const double* part = slot + (size_t)i * nb;
      double s = 0.0;
      for (int b0 = 0; b0 < nb; b0 += 32 * kB) {
        double buf[kB];
#pragma unroll
        for (int j = 0; j < kB; j++) {
          const int b = b0 + j * 32 + lane;
          buf[j] = b < nb ? __ldcg(part + b) : 0.0;
        }
#pragma unroll
        for (int j = 0; j < kB; j++) s += buf[j];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) ctl->tot[i] = s;
    }
  }
  __syncthreads();
}

template <int DIM, typename T, int NCM>
__global__ void __launch_bounds__(TileOp<DIM, T>::THREADS)
    cg_segment_kernel(const __grid_constant__ SegArgs<DIM, T> a) {
  using Op = TileOp<DIM, T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SegCtl* ctl = reinterpret_cast<SegCtl*>(smem_raw + kRedBytes);
  unsigned char* sTile = smem_raw + kSegHeader;
  const int nc = a.nc, nv = a.nv, nb = gridDim.x;
  const long long nn = a.g.nn;
  const bool t0 = threadIdx.x == 0;
  constexpr bool F32 = std::is_same<T, float>::value;
  auto coef = [&](int i) -> T {
    if constexpr (F32) return ctl->coef_f[i];
    else return ctl->coef_d[i];
  };
  // publishes beta / alpha / activity of case c for the next phase
  auto publish_case = [&](int c) {
    ctl->coef_f[c] = (float)ctl->beta[c];
    ctl->coef_f[kMaxCases + c] = (float)ctl->alpha[c];
    ctl->coef_d[c] = ctl->beta[c];
    ctl->coef_d[kMaxCases + c] = ctl->alpha[c];
    ctl->act[c] = ctl->state[c] == 0;
  };
  auto publish = [&]() {
    for (int c = 0; c < kMaxCases; c++) publish_case(c);
  };
  if (t0) {
    ctl->it = a.cs->it;
    ctl->pbuf = a.cs->pbuf;
    ctl->need = 0;
    ctl->flags = 0;
    for (int c = 0; c < kMaxCases; c++) {
      ctl->state[c] = c < nc ? a.cs->state[c] : 1;
      ctl->rz[c] = a.cs->rz[c];
      ctl->rr_ref[c] = a.cs->rr_ref[c];
      ctl->beta[c] = a.cs->beta[c];
      ctl->alpha[c] = 0.0;
    }
    bool any = false;
    for (int c = 0; c < nc; c++) any |= ctl->state[c] == 0;
    ctl->go = any && ctl->it < a.max_it;
    publish();
  }
  __syncthreads();
  unsigned gen = 0;
  bool ok = true;

  while (ctl->go) {
    if (a.trace && blockIdx.x == 0 && t0) a.trace[kTracePts * (ctl->it % kTraceIters) + 0] = globaltimer();
    // ---- phase A: p = z + beta p_old, q = K p, partial p.q
    const int pbuf = ctl->pbuf;
    const T* Pold = pbuf ? a.p1 : a.p0;
    T* Pnew = pbuf ? a.p0 : a.p1;
    T accAt[NCM];
#pragma unroll
    for (int i = 0; i < NCM; i++) accAt[i] = T(0);
    // The loader only loads (a store between loads would keep the compiler from
    // batching them); p of the tile's own nodes is written at emit time.
    for (int t = blockIdx.x; t < a.tm.ntiles; t += nb) {
      Op::template apply<NCM>(
          a.g, a.tm, t, a.E, a.C, sTile, nc,
          [&](long long node, int v, bool) -> T {
            const long long idx = (long long)v * nn + node;
            const T b = coef(v / DIM);
            T val = __ldcg(a.z + idx);
            if (b != T(0)) val = fma(b, __ldcg(Pold + idx), val);
            return val;
          },
          [&](long long node, int cs, const T(&yv)[DIM], const T(&us)[DIM]) {
            const uint8_t mk = a.mask[node];
            T spq = T(0);
#pragma unroll
            for (int r = 0; r < DIM; r++) {
              const T qv = ((mk >> r) & 1) ? T(0) : yv[r];
              const long long idx = (long long)(cs * DIM + r) * nn + node;
              a.q[idx] = qv;
              Pnew[idx] = us[r];
              spq = fma(us[r], qv, spq);
            }
#pragma unroll
            for (int c2 = 0; c2 < NCM; c2++)
              if (c2 == cs) accAt[c2] += spq;
          });
    }
    if (a.trace && blockIdx.x == 0 && t0) a.trace[kTracePts * (ctl->it % kTraceIters) + 1] = globaltimer();
    cta_partial<NCM>(accAt, a.part + (size_t)SLOT_A * nb, smem_raw);
    if (a.trace && blockIdx.x == 0 && t0) a.trace[kTracePts * (ctl->it % kTraceIters) + 2] = globaltimer();
    if (!(ok = grid_sync(a.bar, gen))) break;
    if (a.trace && blockIdx.x == 0 && t0) a.trace[kTracePts * (ctl->it % kTraceIters) + 3] = globaltimer();
    cta_total<NCM, T>(a.part + (size_t)SLOT_A * nb, ctl);
    if (threadIdx.x < kMaxCases) {  // one lane per case
      const int c = threadIdx.x;
      double al = 0.0;
      bool brk = false;
      if (c < NCM && ctl->state[c] == 0) {
        const double pq = ctl->tot[c];
        if (!(pq > 0.0) || !isfinite(pq) || !isfinite(ctl->rz[c])) {
          ctl->state[c] = 2;
          brk = true;
        } else {
          al = ctl->rz[c] / pq;
        }
      }
      ctl->alpha[c] = al;
      publish_case(c);
      if (__any_sync(0xffu, brk) && c == 0) ctl->flags |= ERR_BREAKDOWN;
    }
    __syncthreads();

    if (a.trace && blockIdx.x == 0 && t0) a.trace[kTracePts * (ctl->it % kTraceIters) + 4] = globaltimer();

    // ---- phase B.  Nodes are visited with the thread mapping of phase A's
    // output, so every value read here (r, x_l, q, p of the node) was last
    // written by this same thread (or by an earlier kernel): L1-cached loads
    // are coherent, and each cache line is fetched from L2 once.
    T accBt[2 * NCM];
#pragma unroll
    for (int i = 0; i < 2 * NCM; i++) accBt[i] = T(0);
    for (int t = blockIdx.x; t < a.tm.ntiles; t += nb) {
      Op::for_each_own(a.g, a.tm, t, [&](long long node) {
        if constexpr (DIM == 3) {
          // Each thread walks its node column plane by plane, and the stores of
          // one plane keep the next plane's loads from being issued early: ask
          // L2 for the column four planes ahead (no registers held).
          const long long ahead = node + 4LL * a.g.nx * a.g.ny;
          if (ahead < nn) {
#pragma unroll
            for (int v = 0; v < NCM * DIM; v++) {
              if (v < nv) {
                const long long i = (long long)v * nn + ahead;
                prefetch_l2(a.r + i);
                prefetch_l2(Pnew + i);
                prefetch_l2(a.q + i);
                prefetch_l2(a.xl + i);
              }
            }
#pragma unroll
            for (int r = 0; r < DIM; r++) prefetch_l2(a.invd + (long long)r * nn + ahead);
          }
        }
        // all loads of the node first, then arithmetic, then stores
        constexpr int NVM = NCM * DIM;
        T rv[NVM], pv[NVM], qv[NVM], xv[NVM], inv[DIM];
#pragma unroll
        for (int r = 0; r < DIM; r++) inv[r] = __ldg(a.invd + (long long)r * nn + node);
#pragma unroll
        for (int v = 0; v < NVM; v++) {
          if (v < nv) {
            const long long i = (long long)v * nn + node;
            rv[v] = a.r[i];
            pv[v] = Pnew[i];
            qv[v] = a.q[i];
            xv[v] = a.xl[i];
          }
        }
#pragma unroll
        for (int v = 0; v < NVM; v++) {
          if (v >= nv) break;
          const int cs = v / DIM, r = v - cs * DIM;
          const T al = coef(kMaxCases + cs);
          const T rn = fma(-al, qv[v], rv[v]);
          const T zn = rn * inv[r];
          xv[v] = fma(al, pv[v], xv[v]);
          rv[v] = rn;
          pv[v] = zn;  // reuse as z
          accBt[cs] = fma(rn, zn, accBt[cs]);
          accBt[NCM + cs] = fma(rn, rn, accBt[NCM + cs]);
        }
#pragma unroll
        for (int v = 0; v < NVM; v++) {
          if (v < nv) {
            const long long i = (long long)v * nn + node;
            a.xl[i] = xv[v];
            a.r[i] = rv[v];
            a.z[i] = pv[v];
          }
        }
      });
    }
    if (a.trace && blockIdx.x == 0 && t0) a.trace[kTracePts * (ctl->it % kTraceIters) + 5] = globaltimer();
    cta_partial<2 * NCM>(accBt, a.part + (size_t)SLOT_B * nb, smem_raw);
    if (!(ok = grid_sync(a.bar, gen))) break;
    if (a.trace && blockIdx.x == 0 && t0) a.trace[kTracePts * (ctl->it % kTraceIters) + 6] = globaltimer();
    cta_total<2 * NCM, T>(a.part + (size_t)SLOT_B * nb, ctl);
    if (a.trace && blockIdx.x == 0 && t0) a.trace[kTracePts * (ctl->it % kTraceIters) + 7] = globaltimer();
    if (threadIdx.x < kMaxCases) {  // one lane per case
      const int c = threadIdx.x;
      const bool on = c < NCM && c < nc && ctl->state[c] == 0;
      const double rr = on ? ctl->tot[NCM + c] : 0.0;
      const bool due = on && (rr <= a.tol2ff[c] || rr <= a.drop2 * ctl->rr_ref[c]);
      const bool need = __any_sync(0xffu, due);
      if (!need && c < NCM && c < nc) {  // otherwise rz keeps the value the update step divides by
        const double rzn = ctl->tot[c];
        ctl->beta[c] = (on && ctl->rz[c] != 0.0) ? rzn / ctl->rz[c] : 0.0;
        ctl->rz[c] = rzn;
      }
      const bool any = __any_sync(0xffu, c < nc && ctl->state[c] == 0);
      const int it = ctl->it + 1;
      publish_case(c);
      __syncwarp(0xffu);
      if (c == 0) {
        ctl->it = it;
        ctl->pbuf ^= 1;
        ctl->need = need;
        ctl->go = !need && any && it < a.max_it;
      }
    }
    __syncthreads();
  }
  if (blockIdx.x == 0 && t0) {
    a.cs->it = ctl->it;
    a.cs->pbuf = ctl->pbuf;
    a.cs->need = ctl->need;
    // a CTA that gave up at a barrier leaves the launch early; its error bit in
    // the barrier word reaches the host even if CTA 0's own waits all ended
    const bool timed_out = !ok || (ld_volatile_i32(&a.bar->err) & ERR_TIMEOUT);
    a.cs->flags |= ctl->flags | (timed_out ? ERR_TIMEOUT : 0);
    for (int c = 0; c < NCM && c < kMaxCases; c++) {
      if (c < nc) a.cs->state[c] = ctl->state[c];
      a.cs->rz[c] = ctl->rz[c];
      a.cs->beta[c] = ctl->beta[c];
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
  a.trace = S.trace;
  fill_c<DIM, T>(a.C, S.C);
  const size_t smem = kSegHeader + Op::smem_bytes(S.nc);
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
