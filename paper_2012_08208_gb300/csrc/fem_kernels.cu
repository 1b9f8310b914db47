// Matrix-free finite-element kernels of the GB300 SIMP library:
//   * modified-SIMP moduli E_e = Emin + rho_e^p (E0 - Emin)
//   * the density-penalised operator y = sum_e E_e K0 u_e (Q4 / H8), node-owner
//     gather from a shared-memory tile (no atomics, deterministic)
//   * Jacobi diagonal
//   * the persistent Jacobi-preconditioned CG (one cooperative launch per solve,
//     all load cases in lock-step, FP64 dot products, FP64 reliable updates)
//   * compliance and element sensitivities
// The discrete system is that of Section 3.1 (Eq. "fe_form") with the SIMP
// penalisation of Eq. "simp_fn"; the CG replaces the sparse LU of Section 4.3.
#include <cstdio>

#include "tile.cuh"

namespace tp {

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
  using G = TileGeom<DIM>;
  const Grid& g = a.g;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < g.nn;
       n += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(n % g.nx), y = (int)((n / g.nx) % g.ny), z = (int)(n / ((long long)g.nx * g.ny));
    double d[DIM];
#pragma unroll
    for (int r = 0; r < DIM; r++) d[r] = 0.0;
#pragma unroll
    for (int cn = 0; cn < G::NCORN; cn++) {
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
      a.inv64[n * DIM + r] = v;
      a.inv32[n * DIM + r] = (float)v;
    }
  }
}

__global__ void to_internal_kernel(const double* __restrict__ src, double* dst, long long nn, int dim,
                                   int nc, const uint8_t* mask, int zero_fixed) {
  const long long total = nn * dim * nc;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long node = i / (dim * nc);
    const int v = (int)(i - node * dim * nc);
    const int c = v / dim, comp = v - c * dim;
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
    dst[i] = src[(node * nc + c) * dim + comp];
  }
}

// ---------------------------------------------------------------------------
// Standalone operator application (boundary-conditioned): y = K u on free DOFs
// with fixed entries of u read as 0, y = u on fixed DOFs.

template <int DIM, typename T>
struct MvArgs {
  Grid g;
  TileMap<DIM> tm;
  const T* E;
  const uint8_t* mask;
  const T* u;
  T* y;
  long long stride;
  KMat<DIM, T> k;
};

template <int DIM, typename T>
__global__ void __launch_bounds__(kThreads) matvec_kernel(const __grid_constant__ MvArgs<DIM, T> a) {
  using G = TileGeom<DIM>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sP = reinterpret_cast<T*>(smem_raw);
  T* sE = sP + G::HN * DIM;
  const T* u = a.u + blockIdx.y * a.stride;
  T* y = a.y + blockIdx.y * a.stride;
  int x0, y0, z0;
  tile_origin<DIM>(a.tm, blockIdx.x, x0, y0, z0);
  load_E<DIM, T>(a.g, x0, y0, z0, a.E, sE);
  load_halo<DIM, T>(a.g, x0, y0, z0, DIM, sP, [&](long long node, int v, bool) -> T {
    return ((a.mask[node] >> v) & 1) ? T(0) : u[node * DIM + v];
  });
  __syncthreads();
  for (int ln = threadIdx.x; ln < G::TN; ln += blockDim.x) {
    int tx, ty, tz;
    long long node;
    if (!own_node<DIM>(a.g, ln, x0, y0, z0, tx, ty, tz, node)) continue;
    T acc[DIM];
    node_apply<DIM, T>(sP, sE, DIM, 0, tx, ty, tz, a.k, acc);
    const uint8_t mk = a.mask[node];
#pragma unroll
    for (int r = 0; r < DIM; r++) y[node * DIM + r] = ((mk >> r) & 1) ? u[node * DIM + r] : acc[r];
  }
}

// ---------------------------------------------------------------------------
// Compliance and sensitivities (FP64).

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
  KMat<DIM, double> kD;
};

template <int DIM>
__global__ void __launch_bounds__(kThreads) sens_kernel(const __grid_constant__ SensArgs<DIM> a) {
  using G = TileGeom<DIM>;
  __shared__ double sRed[32];
  const Grid& g = a.g;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < g.ne;
       e += (long long)gridDim.x * blockDim.x) {
    const int ex = (int)(e % g.ex), ey = (int)((e / g.ex) % g.ey);
    const int ez = DIM == 3 ? (int)(e / ((long long)g.ex * g.ey)) : 0;
    double ce = 0.0;
    for (int cs = 0; cs < a.nc; cs++) {
      double u[G::ND];
#pragma unroll
      for (int m = 0; m < G::NCORN; m++) {
        const long long node =
            (ex + cofs(m, 0)) + (long long)g.nx * ((ey + cofs(m, 1)) + (long long)g.ny * (ez + (DIM == 3 ? cofs(m, 2) : 0)));
#pragma unroll
        for (int s = 0; s < DIM; s++) u[DIM * m + s] = a.x64[node * a.nv + cs * DIM + s];
      }
      double t = 0.0;
#pragma unroll
      for (int i = 0; i < G::ND; i++) {
        double si = 0.0;
#pragma unroll
        for (int j = 0; j < G::ND; j++) si = fma(a.kD.k[i * G::ND + j], u[j], si);
        t = fma(u[i], si, t);
      }
      ce += t;
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

// ---------------------------------------------------------------------------
// Host launchers.

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
  constexpr int nd = TileGeom<DIM>::ND;
  for (int i = 0; i < nd; i++) a.kd[i] = K0[i * nd + i];
  diag_kernel<DIM><<<grid_for(g.nn), 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_diag(cudaStream_t s, const Grid& g, const double* K0, const double* E64,
                        const uint8_t* mask, float* inv32, double* inv64) {
  return g.dim == 2 ? diag_impl<2>(s, g, K0, E64, mask, inv32, inv64)
                    : diag_impl<3>(s, g, K0, E64, mask, inv32, inv64);
}

template <int DIM, typename T>
static cudaError_t matvec_impl(cudaStream_t s, const Grid& g, const double* K0, const void* E,
                               const uint8_t* mask, const void* u, void* y, int ncopies) {
  using G = TileGeom<DIM>;
  MvArgs<DIM, T> a;
  a.g = g;
  a.tm = tile_map<DIM>(g);
  a.E = (const T*)E;
  a.mask = mask;
  a.u = (const T*)u;
  a.y = (T*)y;
  a.stride = g.nn * DIM;
  fill_k<DIM, T>(a.k, K0);
  const size_t smem = (size_t)(G::HN * DIM + G::EN) * sizeof(T);
  dim3 grid(a.tm.ntiles, ncopies);
  matvec_kernel<DIM, T><<<grid, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_matvec(cudaStream_t s, const Grid& g, const double* K0, bool f64, const void* E,
                          const uint8_t* mask, const void* u, void* y, int ncopies) {
  if (g.dim == 2)
    return f64 ? matvec_impl<2, double>(s, g, K0, E, mask, u, y, ncopies)
               : matvec_impl<2, float>(s, g, K0, E, mask, u, y, ncopies);
  return f64 ? matvec_impl<3, double>(s, g, K0, E, mask, u, y, ncopies)
             : matvec_impl<3, float>(s, g, K0, E, mask, u, y, ncopies);
}

cudaError_t launch_pcg2(cudaStream_t s, const PcgLaunch& L, bool f64, int nsm, int* grid_out);
cudaError_t launch_pcg3(cudaStream_t s, const PcgLaunch& L, bool f64, int nsm, int* grid_out);

cudaError_t launch_pcg(cudaStream_t s, const PcgLaunch& L, bool f64, int nsm, int* grid_out) {
  return L.g.dim == 2 ? launch_pcg2(s, L, f64, nsm, grid_out) : launch_pcg3(s, L, f64, nsm, grid_out);
}

template <int DIM>
static cudaError_t sens_impl(cudaStream_t s, const Grid& g, int nc, const double* K0, const double* x64,
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
  fill_k<DIM, double>(a.kD, K0);
  const int grid = grid_for(g.ne > g.nn * nc * DIM ? g.ne : g.nn * nc * DIM);
  sens_kernel<DIM><<<grid, kThreads, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  final_sum_kernel<<<1, 256, 0, s>>>(part, grid, out_c);
  return cudaGetLastError();
}

cudaError_t launch_sens(cudaStream_t s, const Grid& g, int nc, const double* K0, const double* x64,
                        const double* f, const double* rho, double penal, double dE, double* ce,
                        double* dc, double* part, double* out_c) {
  return g.dim == 2 ? sens_impl<2>(s, g, nc, K0, x64, f, rho, penal, dE, ce, dc, part, out_c)
                    : sens_impl<3>(s, g, nc, K0, x64, f, rho, penal, dE, ce, dc, part, out_c);
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
