// Persistent multigrid-preconditioned CG segment (cooperative launch): the
// FP32 inner iteration of TP_PRECOND_MG -- CG on the correction d of one
// segment, K d = r, preconditioned by one V-cycle -- in a single kernel.
// Every step of the V-cycle is a phase of the grid separated by a bounded grid
// barrier, instead of a kernel launch of its own.
//
// Per iteration (pbuf selects p_old / p_new):
//   M  p_new = z + beta p_old (formed while the tile operator loads it),
//      q = K p_new, partial p.q                                   -> barrier
//      alpha = r.z / p.q (every CTA, from the same totals)
//   U  d += alpha p, r -= alpha q, x0 = omega D^-1 r (first smoothing step
//      of the finest level)                                       -> barrier
//   V  z = V(r): per level Chebyshev steps, residual, restriction, dense
//      coarsest solve, prolongation, steps (each                  -> barrier);
//      the last finest-level step also forms partial r.z, r.r
//      beta, stopping rule (every CTA, identically)
// The segment starts with z = V(r) and beta = 0.  It stops as the
// graph-captured path does (tolerance with margin 1/2 on the recurrence
// residual, 1e-5 of the starting residual, stagnation, breakdown, iteration
// limit); CTA 0 then writes the iteration count and the reason to the control
// block.  Before the launch: r (finest b) = (float) r64, the finest x0, d = 0
// and the control block (mg_seg_init); the barrier word zeroed.
#include <type_traits>

#include "mg.h"
#include "mg_ops.cuh"
#include "pcg_common.cuh"

namespace tp {
namespace {

constexpr int kMgMaxLevels = 12;

struct MgLevelArgs {
  Grid g;
  int f;
  const float* S;
  const uint8_t* mask;
  const float* invd;
  float* x[2];
  float* b;
  float* t;
};

template <int DIM>
struct MgSegArgs {
  int nl, nc, nu, nu0, cn;  // nu0: the degree on the finest level
  MgLevelArgs lv[kMgMaxLevels];
  TileMapG tm;
  const float* E;     // finest-level moduli
  const float* cinv;  // coarsest dense inverse
  float* d;
  float* p[2];
  float* q;
  MgCtl* ctl;
  double* part;
  GridBar* bar;
  long long* trace;  // optional: barrier timestamps of CTA 0 in the segment's third iteration
  float omega;
  float ca[8], cc[8], cw[8];
  CMat<DIM, float> C;
};

// Per-CTA control, in shared memory (written by thread 0 or one lane per case).
struct MgSegCtl {
  double tot[2 * kMaxCases];
  double rz[kMaxCases], rr_start[kMaxCases], ff[kMaxCases], alpha[kMaxCases], beta[kMaxCases], pq[kMaxCases],
      rr[kMaxCases];
  float af[kMaxCases], bf[kMaxCases];
  double best, tol2;
  int it, best_it, it_limit, stop, reason;
};
constexpr int kSlotPQ = 0;             // kMaxCases partials per CTA: p.q
constexpr int kSlotRZ = kMaxCases;     // 2 kMaxCases partials per CTA: r.z | r.r
constexpr size_t kRedBytesMg = 32 * 2 * kMaxCases * sizeof(float);
constexpr size_t kMgHeader = kRedBytesMg + ((sizeof(MgSegCtl) + 255) / 256) * 256;

// Totals of NV per-CTA double-float partials slot[i * nb + cta] (float2: hi,
// lo) into tot[0, NV): one warp per value, accumulated in double-float in a
// fixed order, so every CTA obtains the identical totals.  FP32 operations
// only: on GB300 an FP64 add costs 64 FP32 issue slots.
template <int NV>
__device__ __forceinline__ void slot_totals(const double* slot8, double* tot) {
  const float2* slot = reinterpret_cast<const float2*>(slot8);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nb = gridDim.x;
  for (int i = warp; i < NV; i += nw) {
    dfl s{0.f, 0.f};
    for (int b0 = 0; b0 < nb; b0 += 32 * 8) {
      float2 buf[8];
#pragma unroll
      for (int j = 0; j < 8; j++) {
        const int b = b0 + j * 32 + lane;
        buf[j] = b < nb ? __ldcg(slot + (size_t)i * nb + b) : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int j = 0; j < 8; j++) s = dfl_add(s, dfl{buf[j].x, buf[j].y});
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const dfl t{__shfl_xor_sync(0xffffffffu, s.hi, o), __shfl_xor_sync(0xffffffffu, s.lo, o)};
      s = dfl_add(s, t);
    }
    if (lane == 0) tot[i] = (double)s.hi + (double)s.lo;
  }
  __syncthreads();
}

template <int DIM, int NCM>
__global__ void __launch_bounds__(256, 2) mg_seg_kernel(const __grid_constant__ MgSegArgs<DIM> a) {
  using Op = TileOp<DIM, float>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MgSegCtl* sc = reinterpret_cast<MgSegCtl*>(smem_raw + kRedBytesMg);
  unsigned char* sTile = smem_raw + kMgHeader;
  const int nb = gridDim.x, nc = a.nc, L = a.nl;
  const long long n0 = a.lv[0].g.nn * DIM;  // finest DOFs per case
  const long long gtid = blockIdx.x * (long long)blockDim.x + threadIdx.x, gthreads = (long long)nb * blockDim.x;
  const long long gwarp = gtid >> 5, gwarps = gthreads >> 5;
  const int lane = threadIdx.x & 31;
  unsigned gen = 0;
  bool ok = true;
  // After a barrier timeout every later barrier returns at once (the error
  // word is set), so the phases below finish quickly and the loop ends.
  int tpos = 0;
  auto sync = [&]() {
    ok = grid_sync(a.bar, gen) && ok;
    if (a.trace && blockIdx.x == 0 && threadIdx.x == 0 && sc->it == 2 && tpos < 64) {
      long long t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      a.trace[tpos++] = t;
    }
  };

  if (threadIdx.x == 0) {
    for (int c = 0; c < kMaxCases; c++) {
      sc->ff[c] = a.ctl->ff[c];
      sc->rz[c] = sc->rr_start[c] = sc->alpha[c] = sc->beta[c] = sc->pq[c] = sc->rr[c] = 0.0;
      sc->af[c] = sc->bf[c] = 0.f;
    }
    sc->tol2 = a.ctl->tol2;
    sc->it_limit = a.ctl->it_limit;
    sc->best = 0.0;
    sc->it = sc->best_it = sc->stop = sc->reason = 0;
  }
  __syncthreads();

  // ---- finest-level Chebyshev step / residual on the tile operator; with
  // dots, also the partial r.z, r.r (r = b, z = y) into slot RZ.
  //   2D: one unit = one tile with all cases; the operator values go to
  //   shared memory, then an epilogue over the tile's own nodes issues all of
  //   a node's loads (b, w, scale, every case) before any store.
  //   3D: the streaming tile operator; each emit loads before it stores.
  auto fine_sweep = [&](const float* u, const float* w, float* y, int mode, float ca, float cc, float om, bool dots) {
    const MgLevelArgs& l = a.lv[0];
    const float* bv = l.b;
    float acc[2 * NCM];
#pragma unroll
    for (int i = 0; i < 2 * NCM; i++) acc[i] = 0.f;
    for (int t = blockIdx.x; t < a.tm.ntiles; t += nb) {
      if constexpr (DIM == 2) {
        constexpr int TX = Op::TX, TY = Op::TY, TXY = TX * TY;
        float* sK = reinterpret_cast<float*>(sTile + Op::smem_bytes(nc));  // [v][TY][TX]
        const int x0 = (t % a.tm.tiles_x) * TX, y0 = (t / a.tm.tiles_x) * TY;
        Op::template apply<NCM>(
            l.g, a.tm, t, a.E, a.C, sTile, nc,
            [&](long long node, int v, bool) -> float {
              const int c = v >> 1, comp = v & 1;
              return ((l.mask[node] >> comp) & 1) ? 0.f : __ldcg(u + c * n0 + node * 2 + comp);
            },
            [&](long long node, int c, const float(&kv)[DIM], const float(&)[DIM]) {
              const int gx = (int)(node % l.g.nx), gy = (int)(node / l.g.nx);
              const int ln = (gx - x0) + TX * (gy - y0);
              sK[(2 * c) * TXY + ln] = kv[0];
              sK[(2 * c + 1) * TXY + ln] = kv[1];
            });
        // apply ends with a barrier: sK and the staged inputs are complete
#pragma unroll
        for (int k = 0; k < Op::NPT; k++) {
          const int ln = threadIdx.x + k * Op::THREADS;
          const int tx = ln % TX, ty = ln / TX, gx = x0 + tx, gy = y0 + ty;
          if (gx >= l.g.nx || gy >= l.g.ny) continue;
          const int node = gx + l.g.nx * gy;
          const uint8_t mk = l.mask[node];
          const float s0 = l.invd[2 * node] * om, s1 = l.invd[2 * node + 1] * om;
          float bb[2 * NCM], ww[2 * NCM];
#pragma unroll
          for (int c = 0; c < NCM; c++) {
            if (c < nc) {
              const long long i = c * n0 + 2LL * node;
              const float2 b2 = __ldcg(reinterpret_cast<const float2*>(bv + i));
              bb[2 * c] = b2.x;
              bb[2 * c + 1] = b2.y;
              if (w) {
                const float2 w2 = __ldcg(reinterpret_cast<const float2*>(w + i));
                ww[2 * c] = w2.x;
                ww[2 * c + 1] = w2.y;
              }
            }
          }
#pragma unroll
          for (int c = 0; c < NCM; c++) {
            if (c < nc) {
              float o[2];
#pragma unroll
              for (int r = 0; r < 2; r++) {
                const float res = bb[2 * c + r] - sK[(2 * c + r) * TXY + ln];
                float out = res;
                if (mode == 1) {
                  out = fmaf(ca, Op::staged(sTile, 2 * c + r, tx, ty), (r ? s1 : s0) * res);
                  if (w) out = fmaf(cc, ww[2 * c + r], out);
                }
                o[r] = ((mk >> r) & 1) ? 0.f : out;
                acc[c] = fmaf(bb[2 * c + r], o[r], acc[c]);
                acc[NCM + c] = fmaf(bb[2 * c + r], bb[2 * c + r], acc[NCM + c]);
              }
              *reinterpret_cast<float2*>(y + c * n0 + 2LL * node) = make_float2(o[0], o[1]);
            }
          }
        }
        __syncthreads();  // the next tile's apply overwrites the staged inputs and sK
      } else {
        Op::template apply<NCM>(
            l.g, a.tm, t, a.E, a.C, sTile, nc,
            [&](long long node, int v, bool) -> float {
              const int c = v / DIM, comp = v - c * DIM;
              return ((l.mask[node] >> comp) & 1) ? 0.f : __ldcg(u + c * n0 + node * DIM + comp);
            },
            [&](long long node, int c, const float(&kv)[DIM], const float(&us)[DIM]) {
              const uint8_t mk = l.mask[node];
              const long long off = (long long)c * n0 + node * DIM;
              float bb[DIM], ww[DIM], sd[DIM];
#pragma unroll
              for (int r = 0; r < DIM; r++) {
                bb[r] = __ldcg(bv + off + r);
                ww[r] = w ? __ldcg(w + off + r) : 0.f;
                sd[r] = l.invd[node * DIM + r];
              }
              float srz = 0.f, srr = 0.f;
#pragma unroll
              for (int r = 0; r < DIM; r++) {
                const float res = bb[r] - kv[r];
                float out = res;
                if (mode == 1) out = fmaf(cc, ww[r], fmaf(ca, us[r], om * sd[r] * res));
                out = ((mk >> r) & 1) ? 0.f : out;
                y[off + r] = out;
                srz = fmaf(bb[r], out, srz);
                srr = fmaf(bb[r], bb[r], srr);
              }
#pragma unroll
              for (int c2 = 0; c2 < NCM; c2++)
                if (c2 == c) {
                  acc[c2] += srz;
                  acc[NCM + c2] += srr;
                }
            });
      }
    }
    if (dots) block_partial_f<2 * NCM>(acc, reinterpret_cast<float2*>(a.part + (size_t)kSlotRZ * nb), smem_raw);
  };
  // ---- coarse-level step / residual (grid-stride over case x node)
  auto coarse_sweep = [&](int li, const float* u, const float* w, float* y, int mode, float ca, float cc, float om) {
    const MgLevelArgs& l = a.lv[li];
    const int nn = (int)l.g.nn;
    for (int it = (int)gtid; it < nc * nn; it += (int)gthreads) {  // one pass over case x node
      const int c = it / nn, nd = it - c * nn;
      mgops::stencil_node<DIM, true>(l.g, l.S, l.mask, l.invd, u, w, l.b, y, mode, ca, cc, om, nd, (long long)c * nn * DIM);
    }
  };
  auto sweep = [&](int li, const float* u, const float* w, float* y, int mode, float ca, float cc, float om,
                   bool dots) {
    if (li == 0) fine_sweep(u, w, y, mode, ca, cc, om, dots);
    else coarse_sweep(li, u, w, y, mode, ca, cc, om);
  };
  auto restrict_to = [&](int li) {  // level li -> li + 1
    const MgLevelArgs& l = a.lv[li];
    const MgLevelArgs& c = a.lv[li + 1];
    float* x0 = li + 1 == L - 1 ? nullptr : c.x[0];  // the dense solve needs no first step
    const int nnc = (int)c.g.nn;
    const long long ndf = l.g.nn * DIM, ndc = (long long)nnc * DIM;
    if (c.f == 2) {
      for (int it = (int)gtid; it < nc * nnc; it += (int)gthreads) {
        const int cs = it / nnc, nd = it - cs * nnc;
        mgops::restrict2_node<DIM, true>(l.g, c.g, l.mask, c.mask, l.t, c.b, x0, c.invd, a.omega, nd, cs * ndf, cs * ndc);
      }
    } else {
      for (int it = (int)gwarp; it < nc * nnc; it += (int)gwarps) {
        const int cs = it / nnc, nd = it - cs * nnc;
        mgops::restrict_warp<DIM, true>(l.g, c.g, c.f, l.mask, c.mask, l.t, c.b, x0, c.invd, a.omega, nd, cs * ndf,
                                  cs * ndc, lane);
      }
    }
  };
  auto prolong_from = [&](int li, const float* xc, float* xf) {  // level li + 1 -> li
    const MgLevelArgs& l = a.lv[li];
    const MgLevelArgs& c = a.lv[li + 1];
    const int nn = (int)l.g.nn;
    const long long ndf = (long long)nn * DIM, ndc = c.g.nn * DIM;
    for (int it = (int)gtid; it < nc * nn; it += (int)gthreads) {
      const int cs = it / nn, nd = it - cs * nn;
      mgops::prolong_node<DIM, true>(l.g, c.g, c.f, l.mask, xc, xf, nd, cs * ndf, cs * ndc);
    }
  };
  // ---- z = V(r); the last finest step forms the partials r.z, r.r and the
  // caller's barrier follows it.  Returns the finest result buffer.
  auto vcycle = [&]() -> const float* {
    int curs[kMgMaxLevels];
    for (int li = 0; li < L - 1; li++) {
      const MgLevelArgs& l = a.lv[li];
      int cu = 0;
      const int nuL = li == 0 ? a.nu0 : a.nu;
      for (int k = 2; k <= nuL; k++) {
        sweep(li, l.x[cu], k == 2 ? nullptr : l.x[cu ^ 1], l.x[cu ^ 1], 1, a.ca[k], a.cc[k], a.cw[k], false);
        sync();
        cu ^= 1;
      }
      sweep(li, l.x[cu], nullptr, l.t, 2, 0.f, 0.f, 0.f, false);
      sync();
      restrict_to(li);
      sync();
      curs[li] = cu;
    }
    {
      const MgLevelArgs& l = a.lv[L - 1];
      for (int i = (int)gwarp; i < a.cn; i += (int)gwarps) mgops::dense_row<true>(a.cn, nc, a.cinv, l.b, l.x[0], i, lane);
      sync();
    }
    const float* xc = a.lv[L - 1].x[0];
    for (int li = L - 2; li >= 0; li--) {
      const MgLevelArgs& l = a.lv[li];
      int cu = curs[li];
      prolong_from(li, xc, l.x[cu]);
      sync();
      const int nuL = li == 0 ? a.nu0 : a.nu;
      for (int k = 1; k <= nuL; k++) {
        const bool last = li == 0 && k == nuL;
        if (k == 1) sweep(li, l.x[cu], nullptr, l.x[cu ^ 1], 1, 1.f, 0.f, a.omega, last);
        else sweep(li, l.x[cu], l.x[cu ^ 1], l.x[cu ^ 1], 1, a.ca[k], a.cc[k], a.cw[k], last);
        sync();
        cu ^= 1;
      }
      xc = l.x[cu];
    }
    return xc;
  };

  // ---- segment start: z = V(r), rz, rr, beta = 0
  const float* z = vcycle();
  slot_totals<2 * NCM>(a.part + (size_t)kSlotRZ * nb, sc->tot);
  if (threadIdx.x < kMaxCases) {
    const int c = threadIdx.x;
    sc->rz[c] = c < nc ? sc->tot[c] : 0.0;
    sc->rr[c] = c < nc ? sc->tot[NCM + c] : 0.0;
    sc->rr_start[c] = sc->rr[c];
    sc->beta[c] = 0.0;
    sc->bf[c] = 0.f;
  }
  __syncthreads();
  int pbuf = 0;
  const MgLevelArgs& l0 = a.lv[0];
  while (ok) {
    // ---- M: p_new = z + beta p_old, q = K p_new, partial p.q
    const float* Pold = a.p[pbuf];
    float* Pnew = a.p[pbuf ^ 1];
    {
      float acc[NCM];
#pragma unroll
      for (int i = 0; i < NCM; i++) acc[i] = 0.f;
      for (int t = blockIdx.x; t < a.tm.ntiles; t += nb) {
        Op::template apply<NCM>(
            l0.g, a.tm, t, a.E, a.C, sTile, nc,
            [&](long long node, int v, bool) -> float {
              const int c = v / DIM, comp = v - c * DIM;
              if ((l0.mask[node] >> comp) & 1) return 0.f;
              const long long i = c * n0 + node * DIM + comp;
              const float bc = sc->bf[c];
              float val = __ldcg(z + i);
              if (bc != 0.f) val = fmaf(bc, __ldcg(Pold + i), val);
              return val;
            },
            [&](long long node, int c, const float(&kv)[DIM], const float(&us)[DIM]) {
              const uint8_t mk = l0.mask[node];
              float spq = 0.f;
#pragma unroll
              for (int r = 0; r < DIM; r++) {
                const long long i = c * n0 + node * DIM + r;
                const float qv = ((mk >> r) & 1) ? 0.f : kv[r];
                a.q[i] = qv;
                Pnew[i] = us[r];
                spq = fmaf(us[r], qv, spq);
              }
#pragma unroll
              for (int c2 = 0; c2 < NCM; c2++)
                if (c2 == c) acc[c2] += spq;
            });
      }
      block_partial_f<NCM>(acc, reinterpret_cast<float2*>(a.part + (size_t)kSlotPQ * nb), smem_raw);
    }
    sync();
    slot_totals<NCM>(a.part + (size_t)kSlotPQ * nb, sc->tot);
    if (threadIdx.x < kMaxCases) {
      const int c = threadIdx.x;
      double al = 0.0;
      if (c < nc) {
        const double pq = sc->tot[c];
        sc->pq[c] = pq;
        al = (pq > 0.0 && isfinite(pq)) ? sc->rz[c] / pq : 0.0;
      }
      sc->alpha[c] = al;
      sc->af[c] = (float)al;
    }
    __syncthreads();
    // ---- U: d += alpha p, r -= alpha q, x0 = omega D^-1 r
    for (int i = (int)gtid; i < nc * (int)n0; i += (int)gthreads) {  // one pass over case x DOF
      const int c = i / (int)n0, j = i - c * (int)n0;
      const float al = sc->af[c];
      const float pv = __ldcg(Pnew + i), dv = __ldcg(a.d + i), qv = __ldcg(a.q + i), bv = __ldcg(l0.b + i);
      const float sd = l0.invd[j];
      a.d[i] = fmaf(al, pv, dv);
      const float rv = fmaf(-al, qv, bv);
      l0.b[i] = rv;
      l0.x[0][i] = a.omega * sd * rv;
    }
    sync();
    // ---- V: z = V(r), partial r.z, r.r
    z = vcycle();
    slot_totals<2 * NCM>(a.part + (size_t)kSlotRZ * nb, sc->tot);
    if (threadIdx.x == 0) {
      const int it = sc->it + 1;
      sc->it = it;
      bool brk = false, done = true, inner = true;
      double worst = 0.0;
      for (int c = 0; c < nc; c++) {
        const double rzn = sc->tot[c], rec = sc->tot[NCM + c];
        sc->beta[c] = sc->rz[c] != 0.0 ? rzn / sc->rz[c] : 0.0;
        sc->bf[c] = (float)sc->beta[c];
        sc->rz[c] = rzn;
        sc->rr[c] = rec;
        brk |= !isfinite(rec) || !(sc->pq[c] > 0.0);
        done &= rec <= 0.25 * sc->tol2 * sc->ff[c];
        inner &= rec <= 1e-10 * sc->rr_start[c];
        worst = fmax(worst, rec / sc->ff[c]);
      }
      if (sc->best == 0.0 || worst < 0.25 * sc->best) {
        sc->best = worst;
        sc->best_it = it;
      }
      const bool stall = it - sc->best_it >= 50, limit = it >= sc->it_limit;
      sc->reason = (done ? MG_STOP_DONE : 0) | (inner ? MG_STOP_INNER : 0) | (stall ? MG_STOP_STALL : 0) |
                   (brk ? MG_STOP_BREAK : 0) | (limit ? MG_STOP_LIMIT : 0);
      sc->stop = sc->reason != 0;
    }
    __syncthreads();
    if (sc->stop) break;
    pbuf ^= 1;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    MgCtl* g = a.ctl;
    g->it = sc->it;
    g->reason = sc->reason | (ok ? 0 : MG_STOP_BREAK);
    g->stop = 1;
    g->timeout = ok ? 0 : 1;
    for (int c = 0; c < kMaxCases; c++) {
      g->sc[c] = sc->alpha[c];
      g->sc[8 + c] = sc->beta[c];
      g->sc[16 + c] = sc->rz[c];
      g->sc[24 + c] = sc->pq[c];
      g->sc[32 + c] = sc->rr[c];
    }
  }
}

template <int DIM>
cudaError_t launch_impl(cudaStream_t s, const MgHierarchy& M, const double* C, const float* E32, int zlen,
                        double* part, GridBar* bar, long long* trace, int nsm, int* grid_out) {
  using Op = TileOp<DIM, float>;
  if ((int)M.lv.size() > kMgMaxLevels || M.lv.size() < 2) return cudaErrorInvalidValue;
  // the grid-stride loops index case x value with 32-bit integers
  if ((long long)M.nc * M.lv[0].g.nn * DIM >= (1LL << 31)) return cudaErrorInvalidValue;
  MgSegArgs<DIM> a;
  memset(&a, 0, sizeof(a));
  a.nl = (int)M.lv.size();
  a.nc = M.nc;
  a.nu = M.nu;
  a.nu0 = M.nu0;
  a.cn = M.cn;
  for (int i = 0; i < a.nl; i++) {
    const MgLevel& l = M.lv[i];
    MgLevelArgs& d = a.lv[i];
    d.g = l.g;
    d.f = l.f;
    d.S = l.S;
    d.mask = l.mask;
    d.invd = l.invd;
    d.x[0] = l.x[0];
    d.x[1] = l.x[1];
    d.b = l.b;
    d.t = l.t;
  }
  a.tm = Op::map(M.lv[0].g, zlen);
  a.E = E32;
  a.cinv = M.cinv;
  a.d = M.d32;
  a.p[0] = M.p32;
  a.p[1] = M.p32b;
  a.q = M.q32;
  a.ctl = M.ctl;
  a.part = part;
  a.bar = bar;
  a.trace = trace;
  a.omega = M.omega;
  for (int k = 0; k < 8; k++) {
    a.ca[k] = M.ca[k];
    a.cc[k] = M.cc[k];
    a.cw[k] = M.cw[k];
  }
  fill_c<DIM, float>(a.C, C);
  // tile operator buffers, then (2D) the operator values of the tile's own nodes
  size_t smem = kMgHeader + Op::smem_bytes(M.nc);
  if constexpr (DIM == 2) smem += (size_t)Op::TX * Op::TY * 2 * M.nc * sizeof(float);
  auto kern = M.nc == 1 ? mg_seg_kernel<DIM, 1> : (M.nc <= 4 ? mg_seg_kernel<DIM, 4> : mg_seg_kernel<DIM, 8>);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int grid = std::min(per_sm, 2) * nsm;
  *grid_out = grid;
  e = cudaMemsetAsync(bar, 0, sizeof(GridBar), s);
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)&a};
  return cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(256), args, smem, s);
}

}  // namespace

cudaError_t launch_mg_segment(cudaStream_t s, const MgHierarchy& M, const double* C, const float* E32, int zlen,
                              double* part, GridBar* bar, long long* trace, int nsm, int* grid_out) {
  return M.lv[0].g.dim == 2 ? launch_impl<2>(s, M, C, E32, zlen, part, bar, trace, nsm, grid_out)
                            : launch_impl<3>(s, M, C, E32, zlen, part, bar, trace, nsm, grid_out);
}

}  // namespace tp
