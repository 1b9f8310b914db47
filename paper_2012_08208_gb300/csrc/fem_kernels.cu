// Matrix-free finite-element kernels of the GB300 SIMP library:
//   * modified-SIMP moduli E_e = Emin + rho_e^p (E0 - Emin)
//   * Jacobi diagonal of K(rho)
//   * the boundary-conditioned operator y = K(rho) u (tile operators of tileop.cuh)
//   * the FP64 true-residual update of the CG (x64 += x_l; r = f - K64 x64)
//   * compliance and element sensitivities
// The discrete system is that of Section 3.1 (Eq. "fe_form") with the SIMP
// penalisation of Eq. "simp_fn"; the element energy u_e^T K0 u_e enters the
// sensitivity of Section 3.2.
#include "pcg_common.cuh"
#include "df32.cuh"
#include "mg_dots.cuh"

namespace tp {

static int grid_for(long long n, int threads = 256) {
  long long b = (n + threads - 1) / threads;
  if (b > 152 * 16) b = 152 * 16;
  if (b < 1) b = 1;
  return (int)b;
}

// ---------------------------------------------------------------------------
// Moduli, diagonal, layout conversion.

__global__ void young_kernel(const double* __restrict__ rho, float* E32, double* E64, long long ne,
                             double E0, double Emin, double penal) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne;
       e += (long long)gridDim.x * blockDim.x) {
    const double r = rho[e];
    const double rp = penal == 3.0 ? r * r * r : pow(r, penal);
    const double E = Emin + rp * (E0 - Emin);
    E64[e] = E;
    E32[e] = (float)E;
  }
}

template <int DIM>
struct DiagArgs {
  Grid g;
  const double* E64;
  const uint8_t* mask;
  float* inv32;
  double* inv64;
  double kd[DIM * (DIM == 2 ? 4 : 8)];  // diagonal of K0
};

template <int DIM>
__global__ void diag_kernel(const __grid_constant__ DiagArgs<DIM> a) {
  constexpr int NCORN = DIM == 2 ? 4 : 8;
  const Grid& g = a.g;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < g.nn;
       n += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(n % g.nx), y = (int)((n / g.nx) % g.ny), z = (int)(n / ((long long)g.nx * g.ny));
    double d[DIM];
#pragma unroll
    for (int r = 0; r < DIM; r++) d[r] = 0.0;
#pragma unroll
    for (int cn = 0; cn < NCORN; cn++) {
      const int ex = x - cofs(cn, 0), ey = y - cofs(cn, 1), ez = DIM == 3 ? z - cofs(cn, 2) : 0;
      if (ex < 0 || ey < 0 || ez < 0 || ex >= g.ex || ey >= g.ey || ez >= g.ez) continue;
      const double E = a.E64[ex + (long long)g.ex * (ey + (long long)g.ey * ez)];
#pragma unroll
      for (int r = 0; r < DIM; r++) d[r] += E * a.kd[DIM * cn + r];
    }
    const uint8_t mk = a.mask[n];
#pragma unroll
    for (int r = 0; r < DIM; r++) {
      const double v = ((mk >> r) & 1) ? 1.0 : 1.0 / d[r];
      a.inv64[r * g.nn + n] = v;
      a.inv32[r * g.nn + n] = (float)v;
    }
  }
}

// ABI layout [case][node * dim + comp]  <->  internal planar layout
// [(case * dim + comp) * n_nodes + node].
__global__ void to_internal_kernel(const double* __restrict__ src, double* dst, long long nn, int dim,
                                   int nc, const uint8_t* mask, int zero_fixed) {
  const long long total = nn * dim * nc;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long v = i / nn, node = i - v * nn;
    const int c = (int)(v / dim), comp = (int)(v - (long long)c * dim);
    double val = src[(long long)c * nn * dim + node * dim + comp];
    if (zero_fixed && ((mask[node] >> comp) & 1)) val = 0.0;
    dst[i] = val;
  }
}

__global__ void to_abi_kernel(const double* __restrict__ src, double* dst, long long nn, int dim, int nc) {
  const long long total = nn * dim * nc;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i / (nn * dim));
    const long long rem = i - (long long)c * nn * dim;
    const long long node = rem / dim;
    const int comp = (int)(rem - node * dim);
    dst[i] = src[((long long)c * dim + comp) * nn + node];
  }
}

// ---------------------------------------------------------------------------
// Standalone boundary-conditioned operator: y = K u on free DOFs with the fixed
// entries of u read as 0, y = u on fixed DOFs.  One CTA per tile; blockIdx.y
// selects the vector (stride n_dof).

template <int DIM, typename T>
struct MvArgs {
  Grid g;
  TileMapG tm;
  const T* E;
  const uint8_t* mask;
  const T* u;
  T* y;
  long long stride;
  const int* stop;  // optional: return at once when set
  // PCG dot product p.q formed in the epilogue (3D FP32): dots >= 0 adds u.y
  // (u read as 0 on fixed DOFs) and completes it as pcg_dots_complete(what = dots)
  int dots;
  double* part;
  MgCtl* ctl;
  CMat<DIM, T> C;
};

template <int DIM, typename T, int MINB = 1>
__global__ void __launch_bounds__(TileOp<DIM, T>::THREADS, MINB)
    matvec_kernel(const __grid_constant__ MvArgs<DIM, T> a) {
  if (halted(a.stop)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const T* u = a.u + blockIdx.y * a.stride;
  T* y = a.y + blockIdx.y * a.stride;
  auto load = [&](long long node, int comp, bool) -> T {
    return ((a.mask[node] >> comp) & 1) ? T(0) : u[node * DIM + comp];
  };
  if constexpr (DIM == 3) {
    T d0 = T(0);  // this thread's share of the fused p.q
    // the fixed bits of the output node are loaded before the layer's arithmetic
    TileOp<3, T>::apply1_pre(
        a.g, a.tm, blockIdx.x, a.E, a.C, smem_raw, load,
        [&](long long node) -> uint8_t { return node >= 0 ? a.mask[node] : (uint8_t)0; },
        [&](long long node, const T(&yv)[3], const T(&us)[3], uint8_t mk) {
#pragma unroll
          for (int r = 0; r < 3; r++) {
            const T v = ((mk >> r) & 1) ? u[node * 3 + r] : yv[r];
            y[node * 3 + r] = v;
            if (a.dots >= 0) d0 = fma(us[r], v, d0);
          }
        });
    if (a.dots >= 0) {
      double acc[2] = {(double)d0, 0.0};
      pcg_dots_complete(acc, a.part, a.ctl, a.dots);
    }
  } else {
    TileOp<DIM, T>::template apply<1>(
        a.g, a.tm, blockIdx.x, a.E, a.C, smem_raw, 1, [&](long long node, int comp, bool own) {
          return load(node, comp, own);
        },
        [&](long long node, int, const T(&yv)[DIM], const T(&)[DIM]) {
          const uint8_t mk = a.mask[node];
#pragma unroll
          for (int r = 0; r < DIM; r++) y[node * DIM + r] = ((mk >> r) & 1) ? u[node * DIM + r] : yv[r];
        });
  }
}

// z-chunk length of a streaming 3D tile kernel: the balanced depth with the
// fewest rounds x (depth + 3) when `resident` CTAs run at once (a tile streams
// depth + 1 element layers after a two-plane prologue).
static int zlen_for(const Grid& g, int resident) {
  const int tx = (g.nx + 30) / 31, ty = (g.ny + 6) / 7;
  int best = 16;
  long long best_cost = -1;
  for (int zl = 1; zl <= g.nz; zl++) {
    const int chunks = (g.nz + zl - 1) / zl;
    const int zb = (g.nz + chunks - 1) / chunks;
    if (zb != zl) continue;
    const long long ntiles = (long long)tx * ty * chunks;
    const long long rounds = (ntiles + resident - 1) / resident;
    const long long cost = rounds * (zl + 3);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = zl;
    }
  }
  return best;
}

// CTAs of `kern` (THREADS threads, `smem` bytes) resident on the whole device.
template <class K>
static int resident_ctas(K kern, int threads, size_t smem) {
  int dev = 0, nsm = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return 0;
  }
  return per_sm * nsm;
}

template <int DIM, typename T>
static cudaError_t matvec_impl(cudaStream_t s, const Grid& g, const double* C, const void* E,
                               const uint8_t* mask, const void* u, void* y, int ncopies, int zlen, const int* stop,
                               int dots = -1, double* part = nullptr, MgCtl* ctl = nullptr) {
  using Op = TileOp<DIM, T>;
  MvArgs<DIM, T> a;
  a.g = g;
  a.tm = Op::map(g, zlen);
  a.E = (const T*)E;
  a.mask = mask;
  a.u = (const T*)u;
  a.y = (T*)y;
  a.stride = g.nn * DIM;
  a.stop = stop;
  a.dots = DIM == 3 && sizeof(T) == 4 ? dots : -1;
  a.part = part;
  a.ctl = ctl;
  fill_c<DIM, T>(a.C, C);
  const size_t smem = Op::smem_bytes();
  // H8 FP32: 3 resident CTAs per SM (80 registers); measured fastest
  auto kern = DIM == 3 ? (sizeof(T) == 4 ? matvec_kernel<DIM, T, 3> : matvec_kernel<DIM, T, 2>) : matvec_kernel<DIM, T, 1>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (DIM == 3) {  // tiles to fill the CTAs this kernel keeps resident
    static int resident = 0;
    if (!resident) resident = resident_ctas(kern, Op::THREADS, smem);
    if (resident > 0) a.tm = Op::map(g, zlen_for(g, resident));
  }
  kern<<<dim3(a.tm.ntiles, ncopies), Op::THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_matvec(cudaStream_t s, const Grid& g, const double* C, bool f64, const void* E,
                          const uint8_t* mask, const void* u, void* y, int ncopies, int zlen, const int* stop) {
  if (g.dim == 2)
    return f64 ? matvec_impl<2, double>(s, g, C, E, mask, u, y, ncopies, zlen, stop)
               : matvec_impl<2, float>(s, g, C, E, mask, u, y, ncopies, zlen, stop);
  return f64 ? matvec_impl<3, double>(s, g, C, E, mask, u, y, ncopies, zlen, stop)
             : matvec_impl<3, float>(s, g, C, E, mask, u, y, ncopies, zlen, stop);
}

cudaError_t launch_matvec_dots(cudaStream_t s, const Grid& g, const double* C, const float* E32, const uint8_t* mask,
                               const float* u, float* y, int ncopies, int zlen, const int* stop, double* part,
                               MgCtl* ctl, int what) {
  if (g.dim != 3) return cudaErrorInvalidValue;
  return matvec_impl<3, float>(s, g, C, E32, mask, u, y, ncopies, zlen, stop, what, part, ctl);
}

// ---------------------------------------------------------------------------
// The same operator in double-word FP32 arithmetic (df32.cuh) on FP64 data:
// u and y are double, the moduli and C are double-words (about 48 significant
// bits).  Each operation runs on the FP32 pipes (11 FP32 operations per
// addition with the sloppy sum below, 9 per multiplication) instead of GB300's
// FP64 pipe at 1/64 of the FP32 rate; the result agrees with the FP64 operator
// to about 1e-13 of the element force scale.

__global__ void dw_moduli_kernel(const double* __restrict__ E64, df32* __restrict__ Edw, long long ne) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne;
       e += (long long)gridDim.x * blockDim.x)
    Edw[e] = df32::of(E64[e]);
}

// The operator's sums use the sloppy double-word addition: its error is
// bounded by the operands (about 1e-13 of the element force scale here), far
// below the tolerances this operator serves, for 11 FP32 operations instead
// of 20.
using DwT = df32f;

template <int DIM>
struct MvDwArgs {
  Grid g;
  TileMapG tm;
  const DwT* E;
  const uint8_t* mask;
  const double* u;
  double* y;
  long long stride;
  const int* stop;
  CMat<DIM, DwT> C;
};

template <int DIM, int MINB = 1>
__global__ void __launch_bounds__(TileOp<DIM, DwT>::THREADS, MINB)
    matvec_dw_kernel(const __grid_constant__ MvDwArgs<DIM> a) {
  if (halted(a.stop)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const double* u = a.u + blockIdx.y * a.stride;
  double* y = a.y + blockIdx.y * a.stride;
  auto load = [&](long long node, int comp, bool) -> DwT {
    return ((a.mask[node] >> comp) & 1) ? DwT() : DwT::of(u[node * DIM + comp]);
  };
  if constexpr (DIM == 3) {
    TileOp<3, DwT>::apply1_pre(
        a.g, a.tm, blockIdx.x, a.E, a.C, smem_raw, load,
        [&](long long node) -> uint8_t { return node >= 0 ? a.mask[node] : (uint8_t)0; },
        [&](long long node, const DwT(&yv)[3], const DwT(&)[3], uint8_t mk) {
#pragma unroll
          for (int r = 0; r < 3; r++) y[node * 3 + r] = ((mk >> r) & 1) ? u[node * 3 + r] : yv[r].to_double();
        });
  } else {
    TileOp<DIM, DwT>::template apply<1>(
        a.g, a.tm, blockIdx.x, a.E, a.C, smem_raw, 1, [&](long long node, int comp, bool own) {
          return load(node, comp, own);
        },
        [&](long long node, int, const DwT(&yv)[DIM], const DwT(&)[DIM]) {
          const uint8_t mk = a.mask[node];
#pragma unroll
          for (int r = 0; r < DIM; r++)
            y[node * DIM + r] = ((mk >> r) & 1) ? u[node * DIM + r] : yv[r].to_double();
        });
  }
}

template <int DIM>
static cudaError_t matvec_dw_impl(cudaStream_t s, const Grid& g, const double* C, const DwT* E,
                                  const uint8_t* mask, const double* u, double* y, int ncopies, int zlen,
                                  const int* stop) {
  using Op = TileOp<DIM, DwT>;
  MvDwArgs<DIM> a;
  a.g = g;
  a.tm = Op::map(g, zlen);
  a.E = E;
  a.mask = mask;
  a.u = u;
  a.y = y;
  a.stride = g.nn * DIM;
  a.stop = stop;
  constexpr int n = DIM == 2 ? 25 : 324;
  for (int i = 0; i < n; i++) a.C.k[i] = DwT::of(C[i]);
  const size_t smem = Op::smem_bytes();
  auto kern = DIM == 3 ? matvec_dw_kernel<DIM, 2> : matvec_dw_kernel<DIM, 1>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (DIM == 3) {
    static int resident = 0;
    if (!resident) resident = resident_ctas(kern, Op::THREADS, smem);
    if (resident > 0) a.tm = Op::map(g, zlen_for(g, resident));
  }
  kern<<<dim3(a.tm.ntiles, ncopies), Op::THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_dw_moduli(cudaStream_t s, const double* E64, void* Edw, long long ne) {
  dw_moduli_kernel<<<grid_for(ne), 256, 0, s>>>(E64, (df32*)Edw, ne);
  return cudaGetLastError();
}

cudaError_t launch_matvec_dw(cudaStream_t s, const Grid& g, const double* C, const void* Edw, const uint8_t* mask,
                             const double* u, double* y, int ncopies, int zlen, const int* stop) {
  // the moduli are stored as df32; DwT has the same layout (hi, lo)
  if (g.dim == 2) return matvec_dw_impl<2>(s, g, C, (const DwT*)Edw, mask, u, y, ncopies, zlen, stop);
  return matvec_dw_impl<3>(s, g, C, (const DwT*)Edw, mask, u, y, ncopies, zlen, stop);
}

// ---------------------------------------------------------------------------
// Multigrid finest-level sweep on the FP32 strain-form operator, one pass per
// case (blockIdx.y):
//   mode 1: y = a u + c w + om D^-1 (b - K u)   (Chebyshev smoothing step; w
//           may be null, and y may alias w, which is read at the own DOF only)
//   mode 2: y = b - K u                          (residual)
// K u with the fixed entries of u read as 0; y = 0 on fixed DOFs.  The
// operator value never leaves registers, so a step reads u, b (and w) and the
// l1 scale once and writes y once.

template <int DIM>
struct SweepArgs {
  Grid g;
  TileMapG tm;
  const float* E;
  const uint8_t* mask;
  const float* invd;
  const float* u;
  const float* w;
  const float* b;
  float* y;
  long long stride;
  const int* stop;
  int mode;
  float a, c, om;
  // PCG dot products formed in the epilogue (3D): dots >= 0 adds b.y and b.b
  // (r.z and r.r when b is the finest right-hand side r and y = z) and
  // completes them as pcg_dots_complete(what = dots)
  int dots;
  double* part;
  MgCtl* ctl;
  CMat<DIM, float> C;
};

template <int DIM, int MINB = 1>
__global__ void __launch_bounds__(TileOp<DIM, float>::THREADS, MINB)
    mg_sweep_kernel(const __grid_constant__ SweepArgs<DIM> a) {
  if (halted(a.stop)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const float* u = a.u + blockIdx.y * a.stride;
  const float* b = a.b + blockIdx.y * a.stride;
  const float* w = a.w ? a.w + blockIdx.y * a.stride : nullptr;
  float* y = a.y + blockIdx.y * a.stride;
  auto load = [&](long long node, int comp, bool) -> float {
    return ((a.mask[node] >> comp) & 1) ? 0.f : u[node * DIM + comp];
  };
  if constexpr (DIM == 3) {
    float d0 = 0.f, d1 = 0.f;  // this thread's share of the fused dot products
    // the output node's right-hand side, l1 scale, x_{k-2} term and fixed bits
    // are loaded before the layer's arithmetic
    struct Pre {
      float b[3], d[3], w[3];
      uint8_t mk;
    };
    TileOp<3, float>::apply1_pre(
        a.g, a.tm, blockIdx.x, a.E, a.C, smem_raw, load,
        [&](long long node) -> Pre {
          Pre q;
          q.mk = 0;
#pragma unroll
          for (int r = 0; r < 3; r++) q.b[r] = q.d[r] = q.w[r] = 0.f;
          if (node >= 0) {
            q.mk = a.mask[node];
#pragma unroll
            for (int r = 0; r < 3; r++) {
              q.b[r] = b[node * 3 + r];
              if (a.mode == 1) q.d[r] = a.invd[node * 3 + r];
              if (a.mode == 1 && w) q.w[r] = w[node * 3 + r];
            }
          }
          return q;
        },
        [&](long long node, const float(&kv)[3], const float(&us)[3], const Pre& q) {
#pragma unroll
          for (int r = 0; r < 3; r++) {
            const float res = q.b[r] - kv[r];
            float out = res;
            if (a.mode == 1) {
              out = fmaf(a.a, us[r], a.om * q.d[r] * res);
              if (w) out = fmaf(a.c, q.w[r], out);
            }
            const float yv = ((q.mk >> r) & 1) ? 0.f : out;
            y[node * 3 + r] = yv;
            if (a.dots >= 0) {
              d0 = fmaf(q.b[r], yv, d0);
              d1 = fmaf(q.b[r], q.b[r], d1);
            }
          }
        });
    if (a.dots >= 0) {
      double acc[2] = {(double)d0, (double)d1};
      pcg_dots_complete(acc, a.part, a.ctl, a.dots);
    }
  } else {
    TileOp<DIM, float>::template apply<1>(
        a.g, a.tm, blockIdx.x, a.E, a.C, smem_raw, 1, [&](long long node, int comp, bool own) {
          return load(node, comp, own);
        },
        [&](long long node, int, const float(&kv)[DIM], const float(&us)[DIM]) {
          const uint8_t mk = a.mask[node];
#pragma unroll
          for (int r = 0; r < DIM; r++) {
            const long long i = node * DIM + r;
            const float res = b[i] - kv[r];
            float out = res;
            if (a.mode == 1) {
              out = fmaf(a.a, us[r], a.om * a.invd[i] * res);
              if (w) out = fmaf(a.c, w[i], out);
            }
            y[i] = ((mk >> r) & 1) ? 0.f : out;
          }
        });
  }
}

template <int DIM>
static cudaError_t sweep_impl(cudaStream_t s, const Grid& g, const double* C, const float* E, const uint8_t* mask,
                              const float* invd, const float* u, const float* w, const float* b, float* y,
                              int ncopies, int zlen, int mode, float ca, float cc, float om, const int* stop,
                              int dots, double* part, MgCtl* ctl) {
  using Op = TileOp<DIM, float>;
  SweepArgs<DIM> a;
  a.g = g;
  a.tm = Op::map(g, zlen);
  a.E = E;
  a.mask = mask;
  a.invd = invd;
  a.u = u;
  a.w = w;
  a.b = b;
  a.y = y;
  a.stride = g.nn * DIM;
  a.stop = stop;
  a.mode = mode;
  a.a = ca;
  a.c = cc;
  a.om = om;
  a.dots = DIM == 3 ? dots : -1;
  a.part = part;
  a.ctl = ctl;
  fill_c<DIM, float>(a.C, C);
  const size_t smem = Op::smem_bytes();
  // H8: 3 resident CTAs per SM, tiles matched to them (measured fastest)
  auto kern = DIM == 3 ? mg_sweep_kernel<DIM, 3> : mg_sweep_kernel<DIM, 1>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (DIM == 3) {  // tiles to fill the CTAs this kernel keeps resident
    static int res = 0;
    if (!res) res = resident_ctas(kern, Op::THREADS, smem);
    if (res > 0) a.tm = Op::map(g, zlen_for(g, res));
  }
  kern<<<dim3(a.tm.ntiles, ncopies), Op::THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_mg_sweep(cudaStream_t s, const Grid& g, const double* C, const float* E, const uint8_t* mask,
                            const float* invd, const float* u, const float* w, const float* b, float* y,
                            int ncopies, int zlen, int mode, float ca, float cc, float om, const int* stop,
                            int dots, double* part, MgCtl* ctl) {
  return g.dim == 2 ? sweep_impl<2>(s, g, C, E, mask, invd, u, w, b, y, ncopies, zlen, mode, ca, cc, om, stop, -1,
                                    part, ctl)
                    : sweep_impl<3>(s, g, C, E, mask, invd, u, w, b, y, ncopies, zlen, mode, ca, cc, om, stop, dots,
                                    part, ctl);
}

// ---------------------------------------------------------------------------
// FP64 true-residual update.

template <typename T>
__global__ void merge_kernel(double* x64, T* xl, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    x64[i] += (double)xl[i];
    xl[i] = T(0);
  }
}

template <int DIM, typename T>
struct ResArgs {
  Grid g;
  TileMapG tm;
  int nc, nv;
  const double* E64;
  const uint8_t* mask;
  const T* invd;
  const double* f;
  const double* x64;
  T* r;
  T* z;
  double* part;  // [16][gridDim.x]: rr_true[8], rz[8]
  CMat<DIM, double> C;
};

template <int DIM, typename T>
__global__ void __launch_bounds__(TileOp<DIM, double>::THREADS)
    residual_kernel(const __grid_constant__ ResArgs<DIM, T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double sRed[32 * 16];
  double acc[16];
#pragma unroll
  for (int i = 0; i < 16; i++) acc[i] = 0.0;
  TileOp<DIM, double>::template apply<kMaxCases>(
      a.g, a.tm, blockIdx.x, a.E64, a.C, smem_raw, a.nc,
      [&](long long node, int v, bool) -> double {
        return ((a.mask[node] >> (v % DIM)) & 1) ? 0.0 : a.x64[(long long)v * a.g.nn + node];
      },
      [&](long long node, int cs, const double(&yv)[DIM], const double(&)[DIM]) {
        const uint8_t mk = a.mask[node];
        double srr = 0.0, srz = 0.0;
#pragma unroll
        for (int r = 0; r < DIM; r++) {
          const long long idx = (long long)(cs * DIM + r) * a.g.nn + node;
          const double r64 = ((mk >> r) & 1) ? 0.0 : a.f[idx] - yv[r];
          const T rt = (T)r64;
          const T zt = rt * a.invd[(long long)r * a.g.nn + node];
          a.r[idx] = rt;
          a.z[idx] = zt;
          srr += r64 * r64;
          srz += (double)rt * (double)zt;
        }
        addto<16>(acc, cs, srr);
        addto<16>(acc, 8 + cs, srz);
      });
  block_sum<16>(acc, sRed);
  if (threadIdx.x == 0)
    for (int i = 0; i < 16; i++) a.part[(size_t)i * gridDim.x + blockIdx.x] = acc[i];
}

// Sums the residual partials in block order and advances the CG state.
__global__ void residual_finalize_kernel(const double* part, int nblocks, int nc, CgState* cs,
                                         const double* tol2ff, int init) {
  __shared__ double sRed[32 * 16];
  double tot[16];
  for (int i = 0; i < 16; i++) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += part[(size_t)i * nblocks + b];
    tot[i] = s;
  }
  block_sum<16>(tot, sRed);
  if (threadIdx.x != 0) return;
  if (init) {
    cs->it = 0;
    cs->pbuf = 0;
    cs->flags = 0;
    cs->updates = 0;
  }
  cs->need = 0;
  cs->updates += 1;
  for (int c = 0; c < kMaxCases; c++) {
    const double rr = tot[c], rz = tot[8 + c];
    if (init) {
      cs->state[c] = c < nc ? 0 : 1;
      cs->stall[c] = 0;
      cs->rr_ref[c] = rr;
      cs->rr_true[c] = rr;
      cs->beta[c] = 0.0;
      cs->rz[c] = rz;
      if (c < nc && rr <= tol2ff[c]) cs->state[c] = 1;
      continue;
    }
    if (c >= nc) continue;
    cs->rr_true[c] = rr;
    if (cs->state[c] != 0) continue;
    // stagnation: the true residual no longer halves between updates
    cs->stall[c] = rr > 0.25 * cs->rr_ref[c] ? cs->stall[c] + 1 : 0;
    cs->rr_ref[c] = rr;
    const double rz_old = cs->rz[c];
    cs->beta[c] = rz_old != 0.0 ? rz / rz_old : 0.0;
    cs->rz[c] = rz;
    if (rr <= tol2ff[c]) cs->state[c] = 1;
    else if (cs->stall[c] >= 6) cs->state[c] = 3;
  }
}

template <int DIM, typename T>
static cudaError_t residual_impl(cudaStream_t s, const Solver& S, bool init, int* nl) {
  using Op = TileOp<DIM, double>;
  const long long nvals = S.g.nn * S.nc * DIM;
  *nl = 0;
  if (!init) {
    merge_kernel<T><<<grid_for(nvals), 256, 0, s>>>(S.x64, (T*)S.xl, nvals);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    (*nl)++;
  }
  ResArgs<DIM, T> a;
  a.g = S.g;
  a.tm = Op::map(S.g, S.zlen);
  a.nc = S.nc;
  a.nv = S.nc * DIM;
  a.E64 = S.E64;
  a.mask = S.mask;
  a.invd = (const T*)S.invdiag;
  a.f = S.f;
  a.x64 = S.x64;
  a.r = (T*)S.r;
  a.z = (T*)S.z;
  a.part = S.part;
  fill_c<DIM, double>(a.C, S.C);
  const size_t smem = Op::smem_bytes(S.nc);
  auto kern = residual_kernel<DIM, T>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<a.tm.ntiles, Op::THREADS, smem, s>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  residual_finalize_kernel<<<1, 256, 0, s>>>(S.part, a.tm.ntiles, S.nc, S.cs, S.tol2ff_dev, init ? 1 : 0);
  *nl += 2;
  return cudaGetLastError();
}

cudaError_t launch_true_residual(cudaStream_t s, const Solver& S, bool f64, bool init, int* nl) {
  if (S.g.dim == 2)
    return f64 ? residual_impl<2, double>(s, S, init, nl) : residual_impl<2, float>(s, S, init, nl);
  return f64 ? residual_impl<3, double>(s, S, init, nl) : residual_impl<3, float>(s, S, init, nl);
}

// ---------------------------------------------------------------------------
// Compliance and sensitivities.  ce_e = sum_k u_e^T K0 u_e = g^T C g, in FP64
// in 2D; in 3D in double-word FP32 arithmetic (df32.cuh, about 1e-14 relative:
// GB300's FP64 pipe made the FP64 energy of 1.5 M elements take 0.53 ms), summed
// over the cases in FP64.  The compliance f.u stays FP64.

template <int DIM>
struct SensArgs {
  Grid g;
  int nc, nv;
  const double* x64;
  const double* f;
  const double* rho;
  double penal, dE;
  double* ce;
  double* dc;
  double* part;
  CMat<DIM, double> C;
  CMat<DIM, df32> Cdw;
};

template <int DIM>
__global__ void __launch_bounds__(256) sens_kernel(const __grid_constant__ SensArgs<DIM> a) {
  __shared__ double sRed[32];
  const Grid& g = a.g;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < g.ne;
       e += (long long)gridDim.x * blockDim.x) {
    const int ex = (int)(e % g.ex), ey = (int)((e / g.ex) % g.ey);
    const int ez = DIM == 3 ? (int)(e / ((long long)g.ex * g.ey)) : 0;
    double ce = 0.0;
    for (int cs = 0; cs < a.nc; cs++) {
      if constexpr (DIM == 2) {
        double ux[4], uy[4];
#pragma unroll
        for (int m = 0; m < 4; m++) {
          const long long node = (ex + cofs(m, 0)) + (long long)g.nx * (ey + cofs(m, 1));
          ux[m] = a.x64[(long long)(cs * 2) * g.nn + node];
          uy[m] = a.x64[(long long)(cs * 2 + 1) * g.nn + node];
        }
        ce += q4_energy(ux, uy, a.C);
      } else {
        df32 u[8][3];
#pragma unroll
        for (int m = 0; m < 8; m++) {
          const long long node = (ex + cofs(m, 0)) +
                                 (long long)g.nx * ((ey + cofs(m, 1)) + (long long)g.ny * (ez + cofs(m, 2)));
#pragma unroll
          for (int s = 0; s < 3; s++) u[m][s] = df32::of(a.x64[(long long)(cs * 3 + s) * g.nn + node]);
        }
        ce += h8_energy(u, a.Cdw).to_double();
      }
    }
    const double r = a.rho[e];
    const double rp1 = a.penal == 3.0 ? r * r : pow(r, a.penal - 1.0);
    a.ce[e] = ce;
    a.dc[e] = -a.penal * rp1 * a.dE * ce;
  }
  // compliance: sum of f . u over all DOF values
  double c[1] = {0.0};
  const long long nvals = g.nn * a.nv;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nvals;
       i += (long long)gridDim.x * blockDim.x)
    c[0] = fma(a.f[i], a.x64[i], c[0]);
  block_sum<1>(c, sRed);
  if (threadIdx.x == 0) a.part[blockIdx.x] = c[0];
}

__global__ void final_sum_kernel(const double* part, int n, double* out) {
  __shared__ double sRed[32];
  double s[1] = {0.0};
  for (int i = threadIdx.x; i < n; i += blockDim.x) s[0] += part[i];
  block_sum<1>(s, sRed);
  if (threadIdx.x == 0) out[0] = s[0];
}

template <int DIM>
static cudaError_t sens_impl(cudaStream_t s, const Grid& g, int nc, const double* C, const double* x64,
                             const double* f, const double* rho, double penal, double dE, double* ce,
                             double* dc, double* part, double* out_c) {
  SensArgs<DIM> a;
  a.g = g;
  a.nc = nc;
  a.nv = nc * DIM;
  a.x64 = x64;
  a.f = f;
  a.rho = rho;
  a.penal = penal;
  a.dE = dE;
  a.ce = ce;
  a.dc = dc;
  a.part = part;
  fill_c<DIM, double>(a.C, C);
  for (int i = 0; i < (DIM == 2 ? 25 : 324); i++) a.Cdw.k[i] = df32::of(C[i]);
  const int grid = grid_for(g.ne > g.nn * nc * DIM ? g.ne : g.nn * nc * DIM);
  sens_kernel<DIM><<<grid, 256, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  final_sum_kernel<<<1, 256, 0, s>>>(part, grid, out_c);
  return cudaGetLastError();
}

cudaError_t launch_sens(cudaStream_t s, const Grid& g, int nc, const double* C, const double* x64,
                        const double* f, const double* rho, double penal, double dE, double* ce,
                        double* dc, double* part, double* out_c) {
  return g.dim == 2 ? sens_impl<2>(s, g, nc, C, x64, f, rho, penal, dE, ce, dc, part, out_c)
                    : sens_impl<3>(s, g, nc, C, x64, f, rho, penal, dE, ce, dc, part, out_c);
}

// ---------------------------------------------------------------------------
// Launchers: moduli, diagonal, layouts.

cudaError_t launch_young(cudaStream_t s, const double* rho, float* E32, double* E64, long long ne,
                         double E0, double Emin, double penal) {
  young_kernel<<<grid_for(ne), 256, 0, s>>>(rho, E32, E64, ne, E0, Emin, penal);
  return cudaGetLastError();
}

template <int DIM>
static cudaError_t diag_impl(cudaStream_t s, const Grid& g, const double* K0, const double* E64,
                             const uint8_t* mask, float* inv32, double* inv64) {
  DiagArgs<DIM> a;
  a.g = g;
  a.E64 = E64;
  a.mask = mask;
  a.inv32 = inv32;
  a.inv64 = inv64;
  constexpr int nd = DIM * (DIM == 2 ? 4 : 8);
  for (int i = 0; i < nd; i++) a.kd[i] = K0[i * nd + i];
  diag_kernel<DIM><<<grid_for(g.nn), 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_diag(cudaStream_t s, const Grid& g, const double* K0, const double* E64,
                        const uint8_t* mask, float* inv32, double* inv64) {
  return g.dim == 2 ? diag_impl<2>(s, g, K0, E64, mask, inv32, inv64)
                    : diag_impl<3>(s, g, K0, E64, mask, inv32, inv64);
}

cudaError_t launch_to_internal(cudaStream_t s, const double* src, double* dst, long long nn, int dim,
                               int nc, const uint8_t* mask, int zero_fixed) {
  to_internal_kernel<<<grid_for(nn * dim * nc), 256, 0, s>>>(src, dst, nn, dim, nc, mask, zero_fixed);
  return cudaGetLastError();
}

cudaError_t launch_to_abi(cudaStream_t s, const double* src, double* dst, long long nn, int dim, int nc) {
  to_abi_kernel<<<grid_for(nn * dim * nc), 256, 0, s>>>(src, dst, nn, dim, nc);
  return cudaGetLastError();
}

}  // namespace tp

namespace tp {
cudaError_t launch_cg_segment2(cudaStream_t s, const Solver& S, bool f64, int nsm, int* grid_out);
cudaError_t launch_cg_segment3(cudaStream_t s, const Solver& S, bool f64, int nsm, int* grid_out);
cudaError_t launch_cg_segment(cudaStream_t s, const Solver& S, bool f64, int nsm, int* grid_out) {
  return S.g.dim == 2 ? launch_cg_segment2(s, S, f64, nsm, grid_out) : launch_cg_segment3(s, S, f64, nsm, grid_out);
}
}  // namespace tp
