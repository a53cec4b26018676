// Stencil kernels of the multigrid levels: operator apply (eq. (e18)), residual
// with the first part of the SSOR preconditioner, red-black Gauss-Seidel
// half-sweeps with the Chebyshev update of eq. (e19) fused in, the fused
// residual + 8-child restriction, and the cell-centred prolongation.
#include <type_traits>

#include "gmg_internal.cuh"

namespace gmg {

namespace {

constexpr int BX = 32, BY = 8;

template <typename A, typename B>
using wider_t = typename std::conditional<std::is_same<A, double>::value || std::is_same<B, double>::value,
                                          double, float>::type;

inline dim3 grid_cells(const Grid3& g) {
  return dim3((unsigned)((g.nx + BX - 1) / BX), (unsigned)((g.ny + BY - 1) / BY), (unsigned)g.nz);
}

// ---------------------------------------------------------------------------
// y = A x
// ---------------------------------------------------------------------------
template <typename C, typename TA, typename TX, typename TY>
__global__ void __launch_bounds__(BX* BY) k_apply(Grid3 g, const TA* __restrict__ a, const TX* __restrict__ x,
                                                  TY* __restrict__ y) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  const size_t p = ((size_t)k * g.ny + j) * g.nx + i;
  C ax;
  stencil_diff<C>(g, a, x, i, j, k, p, ax);
  y[p] = (TY)ax;
}

// ---------------------------------------------------------------------------
// r = b - A x, z = first stage of the smoother preconditioner applied to r
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(BX* BY) k_residual(Grid3 g, const T* __restrict__ a, const T* __restrict__ b,
                                                     const T* __restrict__ x, T* __restrict__ r, T* __restrict__ z,
                                                     int pc) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  const size_t p = ((size_t)k * g.ny + j) * g.nx + i;
  T res = ldg(b + p);
  if (x) {
    T ax;
    stencil_diff<T>(g, a, x, i, j, k, p, ax);
    res -= ax;
  }
  if (r) r[p] = res;
  if (pc == PC_IDENTITY) {
    z[p] = res;
  } else if (pc == PC_JACOBI || (pc == PC_SGS && ((i + j + k) & 1) == 0)) {
    T diag, nsum;
    stencil_split<T, T, T>(g, a, (const T*)nullptr, i, j, k, p, diag, nsum);
    z[p] = res / diag;
  }
}

// ---------------------------------------------------------------------------
// Red-black Gauss-Seidel half-sweep on one colour, Chebyshev update fused.
// Thread (ix, j) of plane k handles cell i = 2 ix + ((j + k + color) & 1).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(BX* BY) k_sgs_half(Grid3 g, const T* __restrict__ a, const T* __restrict__ r,
                                                     T* z, int color, T* __restrict__ d, T* __restrict__ x, T c1,
                                                     T c2, int flags) {
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  const int i = 2 * (int)(blockIdx.x * BX + threadIdx.x) + ((j + k + color) & 1);
  if (i >= g.nx || j >= g.ny) return;
  const size_t p = ((size_t)k * g.ny + j) * g.nx + i;
  T diag, nsum;
  stencil_split<T, T, T>(g, a, (const T*)z, i, j, k, p, diag, nsum);
  const T zp = (ldg(r + p) + nsum) / diag;
  z[p] = zp;
  if (flags & CHEB_UPDATE) {
    const T dp = (flags & CHEB_FIRST) ? c2 * zp : c1 * d[p] + c2 * zp;
    d[p] = dp;
    x[p] = (flags & CHEB_XZERO) ? dp : x[p] + dp;
  }
}

template <typename T>
__global__ void k_cheb_update(size_t n, const T* __restrict__ z, T* __restrict__ d, T* __restrict__ x, T c1, T c2,
                              int flags) {
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
    const T zp = z[p];
    const T dp = (flags & CHEB_FIRST) ? c2 * zp : c1 * d[p] + c2 * zp;
    d[p] = dp;
    x[p] = (flags & CHEB_XZERO) ? dp : x[p] + dp;
  }
}

// ---------------------------------------------------------------------------
// Fused residual + restriction: one thread per coarse cell.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(BX* BY) k_residual_restrict(Grid3 g, const T* __restrict__ a,
                                                              const T* __restrict__ b, const T* __restrict__ x,
                                                              T* __restrict__ coarse) {
  const int nxc = g.nx / 2, nyc = g.ny / 2;
  const int ic = blockIdx.x * BX + threadIdx.x;
  const int jc = blockIdx.y * BY + threadIdx.y;
  const int kc = blockIdx.z;
  if (ic >= nxc || jc >= nyc) return;
  T sum = (T)0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int i = 2 * ic + (c & 1), j = 2 * jc + ((c >> 1) & 1), k = 2 * kc + (c >> 2);
    const size_t p = ((size_t)k * g.ny + j) * g.nx + i;
    T ax;
    stencil_diff<T>(g, a, x, i, j, k, p, ax);
    sum += ldg(b + p) - ax;
  }
  coarse[((size_t)kc * nyc + jc) * nxc + ic] = sum * (T)0.125;
}

// b_c = mean of the 8 children of b (full multigrid carries the right-hand
// side down with the residuals' restriction).
template <typename T>
__global__ void __launch_bounds__(BX* BY) k_restrict_only(Grid3 g, const T* __restrict__ b, T* __restrict__ coarse) {
  const int nxc = g.nx / 2, nyc = g.ny / 2;
  const int ic = blockIdx.x * BX + threadIdx.x;
  const int jc = blockIdx.y * BY + threadIdx.y;
  const int kc = blockIdx.z;
  if (ic >= nxc || jc >= nyc) return;
  T sum = (T)0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int i = 2 * ic + (c & 1), j = 2 * jc + ((c >> 1) & 1), k = 2 * kc + (c >> 2);
    sum += ldg(b + ((size_t)k * g.ny + j) * g.nx + i);
  }
  coarse[((size_t)kc * nyc + jc) * nxc + ic] = sum * (T)0.125;
}

// ---------------------------------------------------------------------------
// x_fine += P e_coarse.  Trilinear: per axis the child takes 3/4 of its
// parent and 1/4 of the neighbour on its side; beyond the domain the
// neighbour is a ghost equal to the parent (Neumann, x/y) or minus the
// parent (homogeneous Dirichlet, z).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(BX* BY) k_prolong_add(Grid3 g, const T* __restrict__ e, T* __restrict__ x,
                                                        int mode) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  const int nxc = g.nx / 2, nyc = g.ny / 2, nzc = g.nz / 2;
  const int ic = i >> 1, jc = j >> 1, kc = k >> 1;
  const size_t p = ((size_t)k * g.ny + j) * g.nx + i;
  auto at = [&](int kk, int jj, int ii) { return ldg(e + ((size_t)kk * nyc + jj) * nxc + ii); };
  if (mode == 1) {
    x[p] += at(kc, jc, ic);
    return;
  }
  // neighbour index and sign per axis
  const int in = (i & 1) ? ic + 1 : ic - 1;
  const int jn = (j & 1) ? jc + 1 : jc - 1;
  const int kn = (k & 1) ? kc + 1 : kc - 1;
  const bool iin = in >= 0 && in < nxc, jin = jn >= 0 && jn < nyc, kin = kn >= 0 && kn < nzc;
  const int ii[2] = {ic, iin ? in : ic};
  const int jj[2] = {jc, jin ? jn : jc};
  const int kk[2] = {kc, kin ? kn : kc};
  const T wz1 = kin ? (T)0.25 : (T)-0.25;  // odd ghost at the plates
  const T wx[2] = {(T)0.75, (T)0.25}, wy[2] = {(T)0.75, (T)0.25}, wz[2] = {(T)0.75, wz1};
  T v = (T)0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int sx = c & 1, sy = (c >> 1) & 1, sz = c >> 2;
    v += wz[sz] * wy[sy] * wx[sx] * at(kk[sz], jj[sy], ii[sx]);
  }
  x[p] += v;
}

__global__ void k_coarsen_coef(Grid3 g, const double* __restrict__ a, double* __restrict__ ac,
                               float* __restrict__ ac32) {
  const int nxc = g.nx / 2, nyc = g.ny / 2, nzc = g.nz / 2;
  const size_t nc = (size_t)nxc * nyc * nzc;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < nc; q += (size_t)gridDim.x * blockDim.x) {
    const int ic = (int)(q % nxc), jc = (int)((q / nxc) % nyc), kc = (int)(q / ((size_t)nxc * nyc));
    double s = 0.0;
    for (int c = 0; c < 8; ++c) {
      const int i = 2 * ic + (c & 1), j = 2 * jc + ((c >> 1) & 1), k = 2 * kc + (c >> 2);
      s += a[((size_t)k * g.ny + j) * g.nx + i];
    }
    s *= 0.125;
    ac[q] = s;
    if (ac32) ac32[q] = (float)s;
  }
}

// FP64 -> FP32 (round to nearest even) on the integer pipe: the copy is then
// bound by HBM alone, not by GB300's FP64 pipe, which runs the conversion
// instruction.
__global__ void k_cast_d2f(size_t n, const double* __restrict__ s, float* __restrict__ d) {
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x)
    d[p] = f64_to_f32(s[p]);
}
__global__ void k_cast_f2d(size_t n, const float* __restrict__ s, double* __restrict__ d) {
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x)
    d[p] = (double)s[p];
}
__global__ void k_copy_d(size_t n, const double* __restrict__ s, double* __restrict__ d) {
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x)
    d[p] = s[p];
}

inline unsigned flat_blocks(size_t n, int threads) {
  size_t b = (n + threads - 1) / threads;
  if (b > 152 * 32) b = 152 * 32;
  if (b == 0) b = 1;
  return (unsigned)b;
}

}  // namespace

Grid3 make_grid(int nx, int ny, int nz, double lx, double ly, double lz) {
  Grid3 g;
  g.nx = nx;
  g.ny = ny;
  g.nz = nz;
  const double hx = lx / nx, hy = ly / ny, hz = lz / nz;
  g.cx = 0.5 / (hx * hx);
  g.cy = 0.5 / (hy * hy);
  g.cz = 0.5 / (hz * hz);
  g.cp = 2.0 / (hz * hz);
  g.fx = (float)g.cx;
  g.fy = (float)g.cy;
  g.fz = (float)g.cz;
  g.fp = (float)g.cp;
  return g;
}

template <typename TA, typename TX, typename TY>
cudaError_t launch_apply(const Grid3& g, const TA* a, const TX* x, TY* y, cudaStream_t s) {
  using C = wider_t<wider_t<TA, TX>, TY>;
  k_apply<C, TA, TX, TY><<<grid_cells(g), dim3(BX, BY), 0, s>>>(g, a, x, y);
  return cudaGetLastError();
}
template cudaError_t launch_apply<double, double, double>(const Grid3&, const double*, const double*, double*,
                                                          cudaStream_t);
template cudaError_t launch_apply<double, float, double>(const Grid3&, const double*, const float*, double*,
                                                         cudaStream_t);
template cudaError_t launch_apply<float, float, float>(const Grid3&, const float*, const float*, float*,
                                                       cudaStream_t);

template <typename T>
cudaError_t launch_residual(const Grid3& g, const T* a, const T* b, const T* x, T* r, T* z, int pc,
                            cudaStream_t s) {
  if constexpr (std::is_same<T, double>::value) {
    // the plain FP64 residual (no preconditioner output): every face product once
    if (x && r && !z && pc == PC_NONE) return launch_residual64_tiled(g, a, b, x, r, s);
  }
  k_residual<T><<<grid_cells(g), dim3(BX, BY), 0, s>>>(g, a, b, x, r, z, pc);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sgs_half(const Grid3& g, const T* a, const T* r, T* z, int color, T* d, T* x, double c1,
                            double c2, int flags, cudaStream_t s) {
  dim3 grid((unsigned)(((g.nx + 1) / 2 + BX - 1) / BX), (unsigned)((g.ny + BY - 1) / BY), (unsigned)g.nz);
  k_sgs_half<T><<<grid, dim3(BX, BY), 0, s>>>(g, a, r, z, color, d, x, (T)c1, (T)c2, flags);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cheb_update(size_t n, const T* z, T* d, T* x, double c1, double c2, int flags,
                               cudaStream_t s) {
  k_cheb_update<T><<<flat_blocks(n, 256), 256, 0, s>>>(n, z, d, x, (T)c1, (T)c2, flags);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_residual_restrict(const Grid3& g, const T* a, const T* b, const T* x, T* coarse,
                                     cudaStream_t s) {
  dim3 grid((unsigned)((g.nx / 2 + BX - 1) / BX), (unsigned)((g.ny / 2 + BY - 1) / BY), (unsigned)(g.nz / 2));
  if (!x) {  // x = 0: b itself
    k_restrict_only<T><<<grid, dim3(BX, BY), 0, s>>>(g, b, coarse);
    return cudaGetLastError();
  }
  if constexpr (std::is_same<T, float>::value) {
    if (pair_aligned(a) && pair_aligned(b) && pair_aligned(x) && cells_fit_int32(g))
      return launch_restrict_pairs(g, a, b, x, coarse, s);
  }
  k_residual_restrict<T><<<grid, dim3(BX, BY), 0, s>>>(g, a, b, x, coarse);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prolong_add(const Grid3& g, const T* e, T* x, int mode, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) {
    if (pair_aligned(x) && cells_fit_int32(g)) return launch_prolong_pairs(g, e, x, mode, s);
  }
  k_prolong_add<T><<<grid_cells(g), dim3(BX, BY), 0, s>>>(g, e, x, mode);
  return cudaGetLastError();
}

cudaError_t launch_coarsen_coef(const Grid3& g, const double* a, double* ac, float* ac32, cudaStream_t s) {
  k_coarsen_coef<<<flat_blocks(g.n() / 8, 256), 256, 0, s>>>(g, a, ac, ac32);
  return cudaGetLastError();
}
cudaError_t launch_cast_d2f(size_t n, const double* src, float* dst, cudaStream_t s) {
  k_cast_d2f<<<flat_blocks(n, 256), 256, 0, s>>>(n, src, dst);
  return cudaGetLastError();
}
cudaError_t launch_cast_f2d(size_t n, const float* src, double* dst, cudaStream_t s) {
  k_cast_f2d<<<flat_blocks(n, 256), 256, 0, s>>>(n, src, dst);
  return cudaGetLastError();
}
cudaError_t launch_copy_d(size_t n, const double* src, double* dst, cudaStream_t s) {
  k_copy_d<<<flat_blocks(n, 256), 256, 0, s>>>(n, src, dst);
  return cudaGetLastError();
}

#define GMG_INST(T)                                                                                         \
  template cudaError_t launch_residual<T>(const Grid3&, const T*, const T*, const T*, T*, T*, int,          \
                                          cudaStream_t);                                                    \
  template cudaError_t launch_sgs_half<T>(const Grid3&, const T*, const T*, T*, int, T*, T*, double, double, \
                                          int, cudaStream_t);                                               \
  template cudaError_t launch_cheb_update<T>(size_t, const T*, T*, T*, double, double, int, cudaStream_t);  \
  template cudaError_t launch_residual_restrict<T>(const Grid3&, const T*, const T*, const T*, T*,          \
                                                   cudaStream_t);                                           \
  template cudaError_t launch_prolong_add<T>(const Grid3&, const T*, T*, int, cudaStream_t);
GMG_INST(float)
GMG_INST(double)
#undef GMG_INST

}  // namespace gmg
