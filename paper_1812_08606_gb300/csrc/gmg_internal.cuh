// Internal declarations shared by the CUDA translation units of libgmg.
//
// Every field is a contiguous [nz][ny][nx] array (x fastest).  The operator
// is the 7-point finite-volume stencil of eq. (e18), Sec. 2.2:
//   (A x)_p = sum_{interior faces f=(p,q)} a_f (x_p - x_q)/h_f^2
//           + sum_{plate faces of p} 2 a_p x_p / hz^2,   a_f = (a_p + a_q)/2,
// with zero flux through the x/y side walls (eq. (eM)).  Kernels form the face
// coefficients on the fly from the cell coefficient a.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace gmg {

// Grid of one multigrid level plus the stencil scale factors.
struct Grid3 {
  int nx, ny, nz;
  double cx, cy, cz;  // 0.5 / h^2 per axis: a_f / h^2 = (a_p + a_q) * c
  double cp;          // 2 / hz^2: plate-face coefficient per unit a_p
  // FP32 copies: an FP32 kernel must not convert from double per cell (on
  // GB300 every FP64 instruction, conversions included, runs at 1/64 rate).
  float fx, fy, fz, fp;
  __host__ __device__ size_t n() const { return (size_t)nx * ny * nz; }
  __host__ __device__ size_t plane() const { return (size_t)nx * ny; }
};

// Stencil scale factors in the arithmetic type C.
template <typename C>
struct GridCoef;
template <>
struct GridCoef<float> {
  __device__ __forceinline__ static float x(const Grid3& g) { return g.fx; }
  __device__ __forceinline__ static float y(const Grid3& g) { return g.fy; }
  __device__ __forceinline__ static float z(const Grid3& g) { return g.fz; }
  __device__ __forceinline__ static float p(const Grid3& g) { return g.fp; }
};
template <>
struct GridCoef<double> {
  __device__ __forceinline__ static double x(const Grid3& g) { return g.cx; }
  __device__ __forceinline__ static double y(const Grid3& g) { return g.cy; }
  __device__ __forceinline__ static double z(const Grid3& g) { return g.cz; }
  __device__ __forceinline__ static double p(const Grid3& g) { return g.cp; }
};

Grid3 make_grid(int nx, int ny, int nz, double lx, double ly, double lz);

// Face form of a level's operator (the coarse levels of the series-parallel
// coarsening, k_faces.cu): matrix entries (coefficient / h^2) of the low faces
// of every cell, kx (0 at i = 0), ky (0 at j = 0), kz (the bottom plate's
// entry at k = 0), and the top plate's entries ktop (nx * ny).
template <typename T>
struct Faces {
  const T* kx = nullptr;
  const T* ky = nullptr;
  const T* kz = nullptr;
  const T* ktop = nullptr;
};

// Smoother-preconditioner choice, matching gmg_smoother_pc.
enum PcKind : int { PC_SGS = 0, PC_JACOBI = 1, PC_IDENTITY = 2, PC_NONE = 3 };

// Flags of the Chebyshev update fused into the smoother kernels.  The fused
// kernel also takes CHEB_LAST (the last step of a smoothing: d is dead after
// it and not written) and CHEB_EIG (a step of the eigen estimate's Krylov
// basis: b is taken as zero and not read, d is read unless CHEB_FIRST and
// never written, x_out = ce x_in + c1 d - c2 B^{-1} A x_in).
enum ChebFlags : int { CHEB_UPDATE = 1, CHEB_FIRST = 2, CHEB_XZERO = 4, CHEB_LAST = 8, CHEB_EIG = 16 };

// ----------------------------------------------------------------------------
// Device helpers
// ----------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }
// The grid's cells, with four planes to spare, index in 32 bits: the pair and
// transfer kernels then form offsets with 32-bit arithmetic.
inline bool cells_fit_int32(const Grid3& g) { return (size_t)(g.nz + 4) * g.plane() < ((size_t)1 << 31); }


// Exact FP32 -> FP64 conversion from the IEEE-754 bit fields, on the integer
// pipe only (GB300 runs the conversion instruction on the FP64 pipe, at 1/64
// of the FP32 rate).  Normal numbers: exponent rebiased from 127 to 1023, the
// 23 mantissa bits moved to the top of the 52-bit field.  Subnormal numbers
// m 2^-149 are normalised first (leading bit of m moved to bit 23); zero,
// infinity and NaN map to their FP64 forms (a NaN comes out quiet, payload kept).
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned sign = u & 0x80000000u;
  const unsigned e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  const int sh = __clz(m | 1u) - 8;               // subnormal: shift that puts the leading bit at 23
  const unsigned ms = (m << sh) & 0x7fffffu;
  const unsigned ef = e == 0xffu ? 0x7ffu : (e != 0u ? e + 896u : 897u - (unsigned)sh);
  const unsigned mf = e == 0xffu ? (m ? m | 0x400000u : 0u) : (e != 0u ? m : ms);  // NaN: quiet bit set
  const bool zero = e == 0u && m == 0u;
  const unsigned hi = zero ? sign : (sign | (ef << 20) | (mf >> 3));
  const unsigned lo = zero ? 0u : (mf << 29);
  return __hiloint2double((int)hi, (int)lo);
}

// FP64 -> FP32 with round to nearest, ties to even, from the IEEE-754 bit
// fields on the integer pipe only; bit-identical to the conversion instruction
// (which GB300 runs on the FP64 pipe).  The 53-bit significand M (implicit bit
// included) is shifted right to the FP32 grid: by 29 bits for a normal FP32
// result (exponent rebiased from 1023 to 127), by more for a subnormal one
// (units of 2^-149); the dropped bits decide the rounding, and a carry out of
// the mantissa moves into the exponent (the largest finite FP32 rounds up to
// infinity that way).  Infinity and NaN keep their class (a NaN comes out
// quiet, the top 22 payload bits kept); FP64 subnormals round to a signed zero.
__device__ __forceinline__ float f64_to_f32(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu);
  const int ef = e - 896;  // FP32 biased exponent of a normal result
  if (ef >= 1 && ef <= 254) {
    // the common case in 32-bit words: kept = top 23 of the 52 mantissa bits,
    // rest = the 29 dropped ones; round up when rest + (kept odd) > half
    const unsigned kept = ((hi & 0xfffffu) << 3) | (lo >> 29), rest = lo & 0x1fffffffu;
    const unsigned up = rest + (kept & 1u) > 0x10000000u ? 1u : 0u;
    return __uint_as_float(sign | (((unsigned)ef << 23) + kept + up));
  }
  const unsigned long long m = ((unsigned long long)(hi & 0xfffffu) << 32) | lo;
  if (e == 0x7ff) return __uint_as_float(sign | 0x7f800000u | (m ? 0x400000u | (unsigned)(m >> 29) : 0u));
  if (ef >= 255) return __uint_as_float(sign | 0x7f800000u);  // beyond FP32: infinity
  const int sh = 926 - e;                                    // subnormal result: 30 or more
  if (e == 0 || sh > 54) return __uint_as_float(sign);       // below half the smallest subnormal
  const unsigned long long sig = m | (1ULL << 52);
  const unsigned long long kept = sig >> sh, rest = sig & ((1ULL << sh) - 1ULL), half = 1ULL << (sh - 1);
  const unsigned up = (rest > half || (rest == half && (kept & 1ULL))) ? 1u : 0u;
  return __uint_as_float(sign | ((unsigned)kept + up));
}
__device__ __forceinline__ double to_f64(float f) { return f32_to_f64(f); }
__device__ __forceinline__ double to_f64(double d) { return d; }

// Diagonal D_p and the neighbour sum N_p = sum_f c_f x_q (so (A x)_p = D_p x_p - N_p),
// and the difference form sum_f c_f (x_p - x_q) + plate terms, which keeps the
// accuracy of A x for smooth x.  C is the arithmetic type.
template <typename C, typename TA, typename TX>
__device__ __forceinline__ void stencil_diff(const Grid3& g, const TA* __restrict__ a,
                                             const TX* __restrict__ x, int i, int j, int k,
                                             size_t p, C& ax) {
  const C ap = (C)ldg(a + p);
  const C xp = (C)ldg(x + p);
  const size_t pl = g.plane();
  C acc = (C)0;
  if (i > 0) acc += (ap + (C)ldg(a + p - 1)) * GridCoef<C>::x(g) * (xp - (C)ldg(x + p - 1));
  if (i < g.nx - 1) acc += (ap + (C)ldg(a + p + 1)) * GridCoef<C>::x(g) * (xp - (C)ldg(x + p + 1));
  if (j > 0) acc += (ap + (C)ldg(a + p - g.nx)) * GridCoef<C>::y(g) * (xp - (C)ldg(x + p - g.nx));
  if (j < g.ny - 1) acc += (ap + (C)ldg(a + p + g.nx)) * GridCoef<C>::y(g) * (xp - (C)ldg(x + p + g.nx));
  if (k > 0) acc += (ap + (C)ldg(a + p - pl)) * GridCoef<C>::z(g) * (xp - (C)ldg(x + p - pl));
  else acc += ap * GridCoef<C>::p(g) * xp;
  if (k < g.nz - 1) acc += (ap + (C)ldg(a + p + pl)) * GridCoef<C>::z(g) * (xp - (C)ldg(x + p + pl));
  else acc += ap * GridCoef<C>::p(g) * xp;
  ax = acc;
}

// Diagonal and neighbour sum (N z)_p; z may be null (treated as zero).
template <typename C, typename TA, typename TZ>
__device__ __forceinline__ void stencil_split(const Grid3& g, const TA* __restrict__ a,
                                              const TZ* z, int i, int j, int k,
                                              size_t p, C& diag, C& nsum) {
  const C ap = (C)ldg(a + p);
  const size_t pl = g.plane();
  C d = (C)0, s = (C)0;
  if (i > 0) { C c = (ap + (C)ldg(a + p - 1)) * GridCoef<C>::x(g); d += c; if (z) s += c * (C)z[p - 1]; }
  if (i < g.nx - 1) { C c = (ap + (C)ldg(a + p + 1)) * GridCoef<C>::x(g); d += c; if (z) s += c * (C)z[p + 1]; }
  if (j > 0) { C c = (ap + (C)ldg(a + p - g.nx)) * GridCoef<C>::y(g); d += c; if (z) s += c * (C)z[p - g.nx]; }
  if (j < g.ny - 1) { C c = (ap + (C)ldg(a + p + g.nx)) * GridCoef<C>::y(g); d += c; if (z) s += c * (C)z[p + g.nx]; }
  if (k > 0) { C c = (ap + (C)ldg(a + p - pl)) * GridCoef<C>::z(g); d += c; if (z) s += c * (C)z[p - pl]; }
  else d += ap * GridCoef<C>::p(g);
  if (k < g.nz - 1) { C c = (ap + (C)ldg(a + p + pl)) * GridCoef<C>::z(g); d += c; if (z) s += c * (C)z[p + pl]; }
  else d += ap * GridCoef<C>::p(g);
  diag = d;
  nsum = s;
}

// ----------------------------------------------------------------------------
// Host launchers (all enqueue on `s`; return the launch error)
// ----------------------------------------------------------------------------

// y = A x.  TA/TX/TY in {float,double}; arithmetic in double if any is double.
template <typename TA, typename TX, typename TY>
cudaError_t launch_apply(const Grid3& g, const TA* a, const TX* x, TY* y, cudaStream_t s);

// r = b - A x (x may be null = zero; r may be null = not stored) and, for the
// smoother, z = first part of B^{-1} r: red cells r/D (SGS), all cells r/D
// (Jacobi), z = r (identity), nothing (PC_NONE).
template <typename T>
cudaError_t launch_residual(const Grid3& g, const T* a, const T* b, const T* x, T* r, T* z, int pc,
                            cudaStream_t s);

// One Gauss-Seidel half-sweep on the cells of `color` ((i+j+k)&1 == color):
// z_p = (r_p + (N z)_p) / D_p, with the Chebyshev update fused (flags).
template <typename T>
cudaError_t launch_sgs_half(const Grid3& g, const T* a, const T* r, T* z, int color, T* d, T* x,
                            double c1, double c2, int flags, cudaStream_t s);

// One Chebyshev step with the red-black SSOR preconditioner in one pass
// (FP32): x_out = x_in + d, d = c1 d + c2 B^{-1}(b - A x_in); xin null means
// x_in = 0.  x_out must not alias x_in; d is updated in place.  ce is read
// only with CHEB_EIG.
// With tma_status non-null the step runs, where tma_smoother_eligible allows
// it, on the kernel fed by bulk-tensor copies (k_smooth_tma.cu), which counts
// in *tma_status the waits for its copies that ran out (none when correct).
// launch_cheb_sgs_tma returns cudaErrorNotSupported, having launched nothing,
// when the driver gives no tensor-map encoder or an encoding fails.
bool fused_smoother_eligible(const Grid3& g);
cudaError_t launch_cheb_sgs_fused(const Grid3& g, const float* a, const float* b, const float* xin, float* xout,
                                  float* d, double c1, double c2, double ce, int flags, int* tma_status,
                                  cudaStream_t s);
// The copy-fed kernel's conditions: a smoothing step (not CHEB_EIG), nx a
// multiple of 4 (16-byte rows) and at least 64, ny at least 26, a, b, x_in
// and d 16-byte aligned, x_out 8-byte aligned.
bool tma_smoother_eligible(const Grid3& g, const float* a, const float* b, const float* xin, const float* xout,
                           const float* d, int flags);
cudaError_t launch_cheb_sgs_tma(const Grid3& g, const float* a, const float* b, const float* xin, float* xout,
                                float* d, double c1, double c2, int flags, int* status, cudaStream_t s);
// The same step on a face-form level (all face arrays 8-byte aligned).
cudaError_t launch_cheb_sgs_fused_faces(const Grid3& g, const Faces<float>& F, const float* b, const float* xin,
                                        float* xout, float* d, double c1, double c2, double ce, int flags,
                                        cudaStream_t s);

// Pointwise Chebyshev update on all cells: d = c1 d + c2 z; x += d.
template <typename T>
cudaError_t launch_cheb_update(size_t n, const T* z, T* d, T* x, double c1, double c2, int flags,
                               cudaStream_t s);

// coarse = mean over the 8 children of (b - A x) on the fine grid g (x null:
// of b itself).
template <typename T>
cudaError_t launch_residual_restrict(const Grid3& g, const T* a, const T* b, const T* x, T* coarse,
                                     cudaStream_t s);

// x_fine += P e_coarse; mode 0 trilinear, 1 constant.
template <typename T>
cudaError_t launch_prolong_add(const Grid3& g_fine, const T* e, T* x, int mode, cudaStream_t s);

// The cell-pair kernels read and write FP32 arrays as float2: every such array
// must start on an 8-byte boundary (their launchers refuse others with
// cudaErrorMisalignedAddress and launch nothing).
inline bool pair_aligned(const void* p) { return ((uintptr_t)p & 7) == 0; }

// FP32 forms of the two transfers above with one thread per fine cell pair
// (k_transfer.cu); the FP32 instantiations of launch_residual_restrict and
// launch_prolong_add use them for 8-byte aligned arrays and fall back to the
// one-cell kernels otherwise.  g is the fine grid (all dimensions even).
cudaError_t launch_restrict_pairs(const Grid3& g, const float* a, const float* b, const float* x, float* coarse,
                                  cudaStream_t s);
cudaError_t launch_prolong_pairs(const Grid3& g, const float* e, float* x, int mode, cudaStream_t s);

// ---- Face-form levels and the operator-dependent prolongation (k_faces.cu) ----
// y = A x, r/z of the smoother residual, a red-black half-sweep and the fused
// residual + restriction, as the cell-form launchers above but on faces.
template <typename T, typename TX, typename TY>
cudaError_t launch_apply_faces(const Grid3& g, const Faces<T>& F, const TX* x, TY* y, cudaStream_t s);
template <typename T>
cudaError_t launch_residual_faces(const Grid3& g, const Faces<T>& F, const T* b, const T* x, T* r, T* z, int pc,
                                  cudaStream_t s);
template <typename T>
cudaError_t launch_sgs_half_faces(const Grid3& g, const Faces<T>& F, const T* r, T* z, int color, T* d, T* x,
                                  double c1, double c2, int flags, cudaStream_t s);
template <typename T>
cudaError_t launch_residual_restrict_faces(const Grid3& g, const Faces<T>& F, const T* b, const T* x, T* coarse,
                                           cudaStream_t s);
// The coarse level's faces (kx, ky, kz, ktop, coarse size) from fine grid g
// whose operator is the cell coefficient a (non-null) or the faces F.
template <typename T>
cudaError_t launch_coarsen_faces(const Grid3& g, const T* a, const Faces<T>& F, T* kx, T* ky, T* kz, T* ktop,
                                 cudaStream_t s);
// Parent weights (wx | wy | wz, 3 n) of the prolongation into grid g, from its
// operator (cell coefficient a or faces F).
template <typename T>
cudaError_t launch_prolong_weights(const Grid3& g, const T* a, const Faces<T>& F, T* w, cudaStream_t s);
// x_fine += P e with those weights; g is the fine grid.
template <typename T>
cudaError_t launch_prolong_opdep(const Grid3& g, const T* e, T* x, const T* w, cudaStream_t s);
// FP64 face entries of a cell-form level (eq. (e18)).
template <typename T>
cudaError_t launch_faces_of_cells(const Grid3& g, const T* a, double* kx, double* ky, double* kz, double* ktop,
                                  cudaStream_t s);
// Dense coarsest operator (n x n, FP64) from faces.
template <typename T>
cudaError_t launch_coarse_assemble_faces(const Grid3& g, const Faces<T>& F, double* A, cudaStream_t s);

// coarse coefficient = mean of the 8 children (FP64), plus an FP32 copy if c32.
cudaError_t launch_coarsen_coef(const Grid3& g_fine, const double* a, double* ac, float* ac32,
                                cudaStream_t s);
cudaError_t launch_cast_d2f(size_t n, const double* src, float* dst, cudaStream_t s);
cudaError_t launch_cast_f2d(size_t n, const float* src, double* dst, cudaStream_t s);
cudaError_t launch_copy_d(size_t n, const double* src, double* dst, cudaStream_t s);

// b = f (+ plate terms 2 a_p g / hz^2 on the first and last layer unless homogeneous).
cudaError_t launch_rhs(const Grid3& g, const double* a, const double* f, double* b, double g_bot,
                       double g_top, int homogeneous, cudaStream_t s);

// E = -grad phi, central differences with boundary ghosts.
cudaError_t launch_field(const Grid3& g, double hx, double hy, double hz, const double* phi,
                         void* ex, void* ey, void* ez, int out_fp32, double g_bot, double g_top,
                         cudaStream_t s);

// dL/da from phi and lambda.
// a and f of the elliptic step from the densities (eqs. (semi2), (e18)).
struct DensityCoef {
  double half_tau_e_eps0_mu_e, half_tau_e_eps0_mu_p;  // (e/eps0)(tau/2)|mu|
  double e_over_eps0, half_tau;
  double dx_ih2, dy_ih2, dz_ih2;                      // D_alpha / h_alpha^2
};
cudaError_t launch_assemble(const Grid3& g, const DensityCoef& dc, const double* ne, const double* np, double* a,
                            double* f, cudaStream_t s);
// One explicit transport stage (k_transport.cu): constants in the grid's units.
struct TransportCoef {
  double mu_e, mu_p;              // mobility magnitudes
  double diff_x, diff_y, diff_z;  // electron diffusion
  double ion_ap, ion_bp;          // alpha(|E|) = ion_ap exp(-ion_bp / |E|)
  double g_bottom, g_top;         // plate potentials (the field's ghosts)
  double kx, ky, kz;              // 1/h^2: the drift divergence of the scaled face fluxes
  double ih2x, ih2y, ih2z;        // 1/(2h): the central-difference field
  double dih2x, dih2y, dih2z;     // D_alpha / h_alpha^2
  double dmx, dmy, dmz;           // D_alpha / mu_e (0 when mu_e = 0): diffusion folded into the face values
};
// r = b - A x in FP64 with each face product formed once (32 x 8 column tiles
// marching in z); the outer solver's true residual.
cudaError_t launch_residual64_tiled(const Grid3& g, const double* a, const double* b, const double* x, double* r,
                                   cudaStream_t s);
// rate_mode 0: the ionization rate computed in place; 1: also stored to rate[];
// 2: read from rate[] (written by a mode-1 stage with the same phi).
cudaError_t launch_transport(const Grid3& g, const TransportCoef& tc, const double* base_e, const double* base_p,
                             const double* ev_e, const double* ev_p, const double* phi, double c, double* out_e,
                             double* out_p, double* rate, int rate_mode, cudaStream_t s);
cudaError_t launch_adjoint_grad(const Grid3& g, const double* phi, const double* lam, double* out,
                                double g_bot, double g_top, cudaStream_t s);

// u_i = splitmix64-based start vector in [-1, 1).
cudaError_t launch_hash_vector(size_t n, double* u, cudaStream_t s);
cudaError_t launch_hash_vector(size_t n, float* u, cudaStream_t s);

// ---- Reductions (deterministic: fixed block count and summation order) ----
int reduce_blocks(size_t n);  // number of partial sums a reduction over n produces

// partial[b*k + i] = block b's part of sum_p w_p v_i,p  (i < k <= 8), V row stride ldv.
template <typename T>
cudaError_t launch_multi_dot(size_t n, const T* w, const T* V, size_t ldv, int k, double* partial,
                             cudaStream_t s);
// Fused classical Gram-Schmidt passes over k <= 32 vectors: partial sums of
// h = V^T w (h_prev null) or of h = V^T (w - V h_prev); and w -= V (h1 + h2)
// with partial sums of ||w||^2.  Partials: [block * k + i] / [block].
constexpr int kCgsMaxVectors = 32;
template <typename T>
cudaError_t launch_cgs_dots(size_t n, const T* w, const T* V, size_t ldv, int k, const double* h_prev,
                            double* partial, cudaStream_t s);
template <typename T>
cudaError_t launch_cgs_update(size_t n, T* w, const T* V, size_t ldv, int k, const double* h1, const double* h2,
                              double* partial, cudaStream_t s);
// Gram matrix of nv (2..kGramMaxVectors) FP32 vectors of length n, row stride
// ldv: partial[b * nv(nv+1)/2 + q] = block b's part of (v_i, v_j), q over the
// upper triangle i <= j row by row.
constexpr int kGramMaxVectors = 12;
cudaError_t launch_gram(size_t n, const float* V, size_t ldv, int nv, double* partial, cudaStream_t s);
// out = alpha t + beta v + gamma u (u null: the last term is left out).
template <typename T>
cudaError_t launch_three_term(size_t n, const T* t, const T* v, const T* u, T* out, double alpha, double beta,
                              double gamma, cudaStream_t s);
// out[i] = sum_b partial[b*k + i] (+ out[i] if accumulate) for i < k; one block per output.
cudaError_t launch_finalize(const double* partial, int nblocks, int k, double* out, int accumulate,
                            cudaStream_t s);
// out[0] = sqrt(sum_b partial[b]); out[1] = (out[0] != 0) ? 1/out[0] : 0.
cudaError_t launch_finalize_norm(const double* partial, int nblocks, double* out, cudaStream_t s);
// w -= sum_i h[i] v_i  (i < k <= 64), h read from device memory.
template <typename T>
cudaError_t launch_multi_axpy(size_t n, T* w, const T* V, size_t ldv, int k, const double* h, cudaStream_t s);
// dst = src * scale[0] (scale read from device memory).
template <typename T>
cudaError_t launch_scale(size_t n, const T* src, T* dst, const double* scale, cudaStream_t s);
// dst = src * alpha (alpha by value).
cudaError_t launch_scale_value(size_t n, const double* src, double* dst, double alpha, cudaStream_t s);
// out[0..2k] = h1[0..k), h2[0..k), *nrm (device to device; k <= 64).
cudaError_t launch_gather_column(const double* h1, const double* h2, const double* nrm, int k, double* out,
                                 cudaStream_t s);
// bytes (a multiple of 4, at most 1 MB) from device memory to mapped pinned
// host memory (its device address), by a one-block kernel instead of a copy engine.
cudaError_t launch_words_to_host(const void* src, void* dst_mapped, size_t bytes, cudaStream_t s);
// dst = src * s, dst32 = FP32 rounding of dst; s = *scale (device) or alpha when
// scale is null; dst may be src.
cudaError_t launch_scale_round(size_t n, const double* src, double* dst, float* dst32, const double* scale,
                               double alpha, cudaStream_t s);
// x += sum_i y[i] z_i, Z row stride ldz, k <= 64, y on the device.
template <typename TZ>
cudaError_t launch_update_solution(size_t n, double* x, const TZ* Z, size_t ldz, int k,
                                   const double* y, cudaStream_t s);
// partial[b*2 + 0] = min over block of a; partial[b*2+1] = count of non-finite / non-positive.
// One fused modified Gram-Schmidt pass: w -= (*hi) vi (vi null: none), then the
// partial sums of (w, vnext) (vnext null: ||w||^2), one per reduce block.
template <typename T>
cudaError_t launch_mgs_step(size_t n, T* w, const T* vi, const T* vnext, const double* hi, double* partial,
                            cudaStream_t s);
// out = a1 v1 + a2 v2 + a3 v3 (FP64 out; null vectors drop their terms; out may alias v3).
template <typename T1, typename T2>
cudaError_t launch_lin3(size_t n, double a1, const T1* v1, double a2, const T2* v2, double a3, const double* v3,
                        double* out, cudaStream_t s);
cudaError_t launch_coef_check(size_t n, const double* a, double* partial, cudaStream_t s);
cudaError_t launch_finalize_check(const double* partial, int nblocks, double* out, cudaStream_t s);

// ---- Double-float outer operator (mixed precision) ----
// Stencil scale factors as (hi, lo) FP32 pairs.
struct DfCoef {
  float xh, xl, yh, yl, zh, zl, ph, pl;
};
DfCoef make_df_coef(const Grid3& g);
// w = A z with a stored as (hi, lo) pairs, z FP32, w FP64; double-float arithmetic.
cudaError_t launch_apply_df64(const Grid3& g, const DfCoef& c, const float2* a2, const float* z, double* w,
                              cudaStream_t s);
// a2 = (fl32(a), fl32(a - fl32(a))).
cudaError_t launch_split(size_t n, const double* a, float2* a2, cudaStream_t s);

// ---- Coarsest level: dense SPD operator, Cholesky, explicit inverse ----
// A (n x n, row-major, n = g.n()) from the coarse coefficient.
cudaError_t launch_coarse_assemble(const Grid3& g, const double* a, double* A, cudaStream_t s);
// In place: A -> L (lower Cholesky factor), then Ainv = A^{-1} (FP64) and, if Ainv32 is not null, an FP32 copy.
// status[0] = 0 on success, 1 + column if a pivot was not positive.
cudaError_t launch_coarse_factor(int n, double* A, double* work, double* Ainv, float* Ainv32,
                                 int* status, cudaStream_t s);
// x = Ainv b (dense matvec): b and x in level precision, the FP64 inverse and
// FP64 sums (an FP32 inverse of the ill-conditioned coarsest operator would
// lose up to cond(A) x 2^-24 of the coarse correction).
template <typename T>
cudaError_t launch_coarse_apply(int n, const double* Ainv, const T* b, T* x, cudaStream_t s);

}  // namespace gmg
