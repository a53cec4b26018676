// Right-hand side with plate data, E = -grad(phi) (Sec. 2.2), the adjoint
// coefficient gradient, and the coarsest-grid direct solve (Sec. 3.2: a
// sequential direct solver on the coarsest mesh; here a dense Cholesky
// factorisation in one thread block, turned into an explicit inverse so the
// per-V-cycle coarse solve is one dense matrix-vector product).
#include "gmg_internal.cuh"

namespace gmg {

namespace {

inline unsigned flat_blocks(size_t n) {
  size_t b = (n + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  if (b == 0) b = 1;
  return (unsigned)b;
}

__global__ void k_rhs(Grid3 g, const double* __restrict__ a, const double* __restrict__ f, double* __restrict__ b,
                      double g_bot, double g_top, int homogeneous) {
  const size_t n = g.n(), pl = g.plane();
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
    double v = f[p];
    if (!homogeneous) {  // plate planes by comparison, not by dividing the index
      if (p < pl) v += a[p] * g.cp * g_bot;
      if (p >= n - pl) v += a[p] * g.cp * g_top;
    }
    b[p] = v;
  }
}

// The same on double2 pieces (n even, f and b 16-byte aligned), two pieces a
// trip with both loads issued first: a copy this simple is bound by the loads
// each thread keeps in flight.
__global__ void k_rhs2(Grid3 g, const double* __restrict__ a, const double2* __restrict__ f,
                       double2* __restrict__ b, double g_bot, double g_top, int homogeneous) {
  const size_t n2 = g.n() / 2, pl = g.plane(), n = g.n();
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const double cb = g.cp * g_bot, ct = g.cp * g_top;
  auto fix = [&](size_t q, double2 v) {  // q: the piece's first cell
    if (!homogeneous) {
      if (q < pl) {
        v.x += a[q] * cb;
        v.y += a[q + 1] * cb;
      }
      if (q >= n - pl) {
        v.x += a[q] * ct;
        v.y += a[q + 1] * ct;
      }
    }
    return v;
  };
  size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  for (; p + stride < n2; p += 2 * stride) {
    const double2 v0 = f[p], v1 = f[p + stride];
    b[p] = fix(2 * p, v0);
    b[p + stride] = fix(2 * (p + stride), v1);
  }
  if (p < n2) b[p] = fix(2 * p, f[p]);
}

template <typename TE>
__global__ void k_field(Grid3 g, double ihx2, double ihy2, double ihz2, float fhx, float fhy, float fhz,
                        const double* __restrict__ phi, TE* __restrict__ ex, TE* __restrict__ ey,
                        TE* __restrict__ ez, double g_bot, double g_top) {
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y * 8 + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  const size_t pl = g.plane();
  const size_t p = ((size_t)k * g.ny + j) * g.nx + i;
  const double c = phi[p];
  const double xm = (i > 0) ? phi[p - 1] : c;                 // mirror ghost (zero flux)
  const double xp = (i < g.nx - 1) ? phi[p + 1] : c;
  const double ym = (j > 0) ? phi[p - g.nx] : c;
  const double yp = (j < g.ny - 1) ? phi[p + g.nx] : c;
  // plate ghost 2g - phi; k is the same for the whole block, so only the two
  // plate planes run the ghost arithmetic
  double zm, zp;
  if (k > 0 && k < g.nz - 1) {
    zm = phi[p - pl];
    zp = phi[p + pl];
  } else {
    zm = (k > 0) ? phi[p - pl] : 2.0 * g_bot - c;
    zp = (k < g.nz - 1) ? phi[p + pl] : 2.0 * g_top - c;
  }
  if constexpr (sizeof(TE) == 4) {
    // FP32 output: the FP64 differences are rounded once to FP32 (on the
    // integer pipe, bit-identical to the conversion instruction) and scaled in
    // FP32; the error stays at two FP32 roundings and the FP64 pipe runs only
    // the three differences.
    ex[p] = f64_to_f32(xm - xp) * fhx;
    ey[p] = f64_to_f32(ym - yp) * fhy;
    ez[p] = f64_to_f32(zm - zp) * fhz;
  } else {
    ex[p] = (TE)(-(xp - xm) * ihx2);
    ey[p] = (TE)(-(yp - ym) * ihy2);
    ez[p] = (TE)(-(zp - zm) * ihz2);
  }
}

// a and f of eq. (e18) from the densities, one thread per cell; the second
// differences of n_e take the densities' zero-flux ghosts (ghost = cell).
__global__ void k_assemble(Grid3 g, DensityCoef dc, const double* __restrict__ ne, const double* __restrict__ np,
                           double* __restrict__ a, double* __restrict__ f) {
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y * 8 + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  const size_t pl = g.plane();
  const size_t p = ((size_t)k * g.ny + j) * g.nx + i;
  const double c = ne[p], ni = np[p];
  const double xm = i > 0 ? ne[p - 1] : c, xp = i < g.nx - 1 ? ne[p + 1] : c;
  const double ym = j > 0 ? ne[p - g.nx] : c, yp = j < g.ny - 1 ? ne[p + g.nx] : c;
  const double zm = k > 0 ? ne[p - pl] : c, zp = k < g.nz - 1 ? ne[p + pl] : c;
  const double lap = dc.dx_ih2 * ((xp - 2.0 * c) + xm) + dc.dy_ih2 * ((yp - 2.0 * c) + ym) +
                     dc.dz_ih2 * ((zp - 2.0 * c) + zm);
  a[p] = 1.0 + (dc.half_tau_e_eps0_mu_p * ni + dc.half_tau_e_eps0_mu_e * c);
  f[p] = dc.e_over_eps0 * ((ni - c) - dc.half_tau * lap);
}

__global__ void k_adjoint_grad(Grid3 g, const double* __restrict__ phi, const double* __restrict__ lam,
                               double* __restrict__ out, double g_bot, double g_top) {
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y * 8 + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  const size_t pl = g.plane();
  const size_t p = ((size_t)k * g.ny + j) * g.nx + i;
  const double fp = phi[p], lp = lam[p];
  double s = 0.0;
  // d a_f / d a_p = 1/2 on interior faces; (a_f/h^2) per unit a_p is 0.5/h^2 = c
  if (i > 0) s += g.cx * (lp - lam[p - 1]) * (fp - phi[p - 1]);
  if (i < g.nx - 1) s += g.cx * (lp - lam[p + 1]) * (fp - phi[p + 1]);
  if (j > 0) s += g.cy * (lp - lam[p - g.nx]) * (fp - phi[p - g.nx]);
  if (j < g.ny - 1) s += g.cy * (lp - lam[p + g.nx]) * (fp - phi[p + g.nx]);
  if (k > 0) s += g.cz * (lp - lam[p - pl]) * (fp - phi[p - pl]);
  else s += g.cp * lp * (fp - g_bot);
  if (k < g.nz - 1) s += g.cz * (lp - lam[p + pl]) * (fp - phi[p + pl]);
  else s += g.cp * lp * (fp - g_top);
  out[p] = -s;
}

// Dense coarsest operator, one thread per row.
__global__ void k_coarse_assemble(Grid3 g, const double* __restrict__ a, double* __restrict__ A) {
  const int n = (int)g.n();
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n) return;
  const int i = row % g.nx, j = (row / g.nx) % g.ny, k = row / (g.nx * g.ny);
  const int pl = g.nx * g.ny;
  double* Ar = A + (size_t)row * n;
  for (int c = 0; c < n; ++c) Ar[c] = 0.0;
  const double ap = a[row];
  double d = 0.0;
  auto face = [&](int q, double cc) {
    const double v = (ap + a[q]) * cc;
    Ar[q] = -v;
    d += v;
  };
  if (i > 0) face(row - 1, g.cx);
  if (i < g.nx - 1) face(row + 1, g.cx);
  if (j > 0) face(row - g.nx, g.cy);
  if (j < g.ny - 1) face(row + g.nx, g.cy);
  if (k > 0) face(row - pl, g.cz);
  else d += ap * g.cp;
  if (k < g.nz - 1) face(row + pl, g.cz);
  else d += ap * g.cp;
  Ar[row] = d;
}

// Cholesky A = L L^T in place (lower triangle), then Ainv = L^{-T} L^{-1}.
// One block; n <= 1024.  status[0] = 0 or 1 + index of a non-positive pivot.
__global__ void __launch_bounds__(1024) k_coarse_factor(int n, double* __restrict__ A, double* __restrict__ W,
                                                        double* __restrict__ Ainv, float* __restrict__ Ainv32,
                                                        int* __restrict__ status) {
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      double s = A[(size_t)j * n + j];
      for (int k = 0; k < j; ++k) s -= A[(size_t)j * n + k] * A[(size_t)j * n + k];
      if (!(s > 0.0) || !isfinite(s)) bad = 1 + j;
      else A[(size_t)j * n + j] = sqrt(s);
    }
    __syncthreads();
    if (bad) break;
    const double ljj = A[(size_t)j * n + j];
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) {
      double s = A[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) s -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
      A[(size_t)i * n + j] = s / ljj;
    }
    __syncthreads();
  }
  if (bad) {
    if (threadIdx.x == 0) status[0] = bad;
    return;
  }
  // W = L^{-1}: column c solves L y = e_c by forward substitution.
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    for (int i = 0; i < c; ++i) W[(size_t)i * n + c] = 0.0;
    for (int i = c; i < n; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int k = c; k < i; ++k) s -= A[(size_t)i * n + k] * W[(size_t)k * n + c];
      W[(size_t)i * n + c] = s / A[(size_t)i * n + i];
    }
  }
  __syncthreads();
  // Ainv = W^T W
  for (size_t e = threadIdx.x; e < (size_t)n * n; e += blockDim.x) {
    const int r = (int)(e / n), c = (int)(e % n);
    const int k0 = r > c ? r : c;
    double s = 0.0;
    for (int k = k0; k < n; ++k) s += W[(size_t)k * n + r] * W[(size_t)k * n + c];
    Ainv[e] = s;
    if (Ainv32) Ainv32[e] = (float)s;
  }
  if (threadIdx.x == 0) status[0] = 0;
}

// x = Ainv b, one warp per row.
template <typename T>
__global__ void k_coarse_apply(int n, const double* __restrict__ Ainv, const T* __restrict__ b, T* __restrict__ x) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= n) return;
  double s = 0.0;
  for (int c = lane; c < n; c += 32) s += Ainv[(size_t)warp * n + c] * (double)b[c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) x[warp] = (T)s;
}

}  // namespace

cudaError_t launch_rhs(const Grid3& g, const double* a, const double* f, double* b, double g_bot, double g_top,
                       int homogeneous, cudaStream_t s) {
  // a plane holds an even number of cells when nx is even, so a piece never straddles a plate plane
  if (g.n() % 2 == 0 && g.nx % 2 == 0 && ((uintptr_t)f & 15) == 0 && ((uintptr_t)b & 15) == 0) {
    k_rhs2<<<flat_blocks(g.n() / 2), 256, 0, s>>>(g, a, reinterpret_cast<const double2*>(f),
                                                 reinterpret_cast<double2*>(b), g_bot, g_top, homogeneous);
    return cudaGetLastError();
  }
  k_rhs<<<flat_blocks(g.n()), 256, 0, s>>>(g, a, f, b, g_bot, g_top, homogeneous);
  return cudaGetLastError();
}

cudaError_t launch_field(const Grid3& g, double hx, double hy, double hz, const double* phi, void* ex, void* ey,
                         void* ez, int out_fp32, double g_bot, double g_top, cudaStream_t s) {
  dim3 grid((unsigned)((g.nx + 31) / 32), (unsigned)((g.ny + 7) / 8), (unsigned)g.nz);
  const double ix = 0.5 / hx, iy = 0.5 / hy, iz = 0.5 / hz;
  if (out_fp32)
    k_field<float><<<grid, dim3(32, 8), 0, s>>>(g, ix, iy, iz, (float)ix, (float)iy, (float)iz, phi, (float*)ex,
                                                (float*)ey, (float*)ez, g_bot, g_top);
  else
    k_field<double><<<grid, dim3(32, 8), 0, s>>>(g, ix, iy, iz, (float)ix, (float)iy, (float)iz, phi,
                                                 (double*)ex, (double*)ey, (double*)ez, g_bot, g_top);
  return cudaGetLastError();
}

cudaError_t launch_assemble(const Grid3& g, const DensityCoef& dc, const double* ne, const double* np, double* a,
                            double* f, cudaStream_t s) {
  dim3 grid((unsigned)((g.nx + 31) / 32), (unsigned)((g.ny + 7) / 8), (unsigned)g.nz);
  k_assemble<<<grid, dim3(32, 8), 0, s>>>(g, dc, ne, np, a, f);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_grad(const Grid3& g, const double* phi, const double* lam, double* out, double g_bot,
                                double g_top, cudaStream_t s) {
  dim3 grid((unsigned)((g.nx + 31) / 32), (unsigned)((g.ny + 7) / 8), (unsigned)g.nz);
  k_adjoint_grad<<<grid, dim3(32, 8), 0, s>>>(g, phi, lam, out, g_bot, g_top);
  return cudaGetLastError();
}

cudaError_t launch_coarse_assemble(const Grid3& g, const double* a, double* A, cudaStream_t s) {
  const int n = (int)g.n();
  k_coarse_assemble<<<(n + 127) / 128, 128, 0, s>>>(g, a, A);
  return cudaGetLastError();
}

cudaError_t launch_coarse_factor(int n, double* A, double* work, double* Ainv, float* Ainv32, int* status,
                                 cudaStream_t s) {
  k_coarse_factor<<<1, 1024, 0, s>>>(n, A, work, Ainv, Ainv32, status);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_coarse_apply(int n, const double* Ainv, const T* b, T* x, cudaStream_t s) {
  const int warps_per_block = 8;
  k_coarse_apply<T><<<(n + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0, s>>>(n, Ainv, b, x);
  return cudaGetLastError();
}
template cudaError_t launch_coarse_apply<float>(int, const double*, const float*, float*, cudaStream_t);
template cudaError_t launch_coarse_apply<double>(int, const double*, const double*, double*, cudaStream_t);

}  // namespace gmg
