// FP64 vector kernels of the FGMRES outer loop (Algorithm 1, Sec. 3.1):
// deterministic multi-dot reductions for the Gram-Schmidt coefficients
// h_{i,j} = (w, v_i), the multi-axpy w -= sum_i h_{i,j} v_i, norms and
// scaling for v_{j+1} = w / h_{j+1,j}, and the solution update x = x0 + Z_k y_k.
// Reductions use a fixed number of blocks and a fixed summation order, so a
// result does not depend on scheduling.
#include <type_traits>

#include "gmg_internal.cuh"

namespace gmg {

namespace {

constexpr int RT = 256;          // reduction block size
constexpr int MAX_RBLOCKS = 1024;


__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum a per-thread value over the block; result valid in thread 0.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    t = (lane < NT / 32) ? sh[lane] : 0.0;
    t = warp_sum(t);
  }
  __syncthreads();
  return t;
}

// T = double: FP64 products and sums.  T = float (the FP32 eigen estimate of
// the mixed-precision set-up): per-thread FP32 sums, FP64 across threads.
template <int K, typename T>
__global__ void __launch_bounds__(RT) k_multi_dot(size_t n, const T* __restrict__ w, const T* __restrict__ V,
                                                  size_t ldv, double* __restrict__ partial) {
  __shared__ double sh[RT / 32];
  T acc[K];
#pragma unroll
  for (int i = 0; i < K; ++i) acc[i] = (T)0;
  for (size_t p = blockIdx.x * (size_t)RT + threadIdx.x; p < n; p += (size_t)gridDim.x * RT) {
    const T wp = w[p];
#pragma unroll
    for (int i = 0; i < K; ++i) acc[i] = fma(wp, V[i * ldv + p], acc[i]);
  }
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const double t = block_sum<RT>((double)acc[i], sh);
    if (threadIdx.x == 0) partial[(size_t)blockIdx.x * K + i] = t;
  }
}

// ---- Modified Gram-Schmidt, one fused pass per basis vector ----
// w -= h_i v_i (h_i read from device memory; vi null: no update) and the
// partial sums of (w, v_next) with the updated w (vnext null: ||w||^2).  Each
// pass reads w, v_i and v_next once and writes w, so MGS moves about 32 bytes
// per element per basis vector and takes 2 FMA: on GB300, whose FP64 rate is
// 1/64 of FP32, that is cheaper than the 4 FMA per element per vector of CGS2.
template <typename T>
__global__ void __launch_bounds__(RT) k_mgs_step(size_t n, T* __restrict__ w, const T* __restrict__ vi,
                                                 const T* __restrict__ vnext, const double* __restrict__ hi,
                                                 double* __restrict__ partial) {
  __shared__ double sh[RT / 32];
  const T h = vi ? (T)*hi : (T)0;
  T acc = (T)0;
  for (size_t p = blockIdx.x * (size_t)RT + threadIdx.x; p < n; p += (size_t)gridDim.x * RT) {
    T wp = w[p];
    if (vi) {
      wp = fma(-h, vi[p], wp);
      w[p] = wp;
    }
    acc = fma(wp, vnext ? vnext[p] : wp, acc);
  }
  const double t = block_sum<RT>((double)acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// ---- Fused classical Gram-Schmidt passes (K <= CGS_KMAX vectors) ----
// K is a template parameter: a loop over a runtime count would issue every
// unrolled (predicated-off) load and FMA, which on GB300's 1/64-rate FP64 pipe
// costs as much as the real ones.
// Pass 1: partial sums of h1 = V^T w.  Pass 2 (h != null): partial sums of
// h2 = V^T (w - V h), forming w - V h on the fly without storing it.
template <int K, typename T>
__global__ void __launch_bounds__(RT) k_cgs_dots(size_t n, const T* __restrict__ w, const T* __restrict__ V,
                                                 size_t ldv, const double* __restrict__ h,
                                                 double* __restrict__ partial) {
  __shared__ double sh[RT / 32];
  __shared__ T hs[K];
  if (threadIdx.x < K) hs[threadIdx.x] = h ? (T)h[threadIdx.x] : (T)0;
  __syncthreads();
  T acc[K];
#pragma unroll
  for (int i = 0; i < K; ++i) acc[i] = (T)0;
  for (size_t p = blockIdx.x * (size_t)RT + threadIdx.x; p < n; p += (size_t)gridDim.x * RT) {
    T v[K];
#pragma unroll
    for (int i = 0; i < K; ++i) v[i] = V[i * ldv + p];
    T wp = w[p];
    if (h) {
#pragma unroll
      for (int i = 0; i < K; ++i) wp = fma(-hs[i], v[i], wp);
    }
#pragma unroll
    for (int i = 0; i < K; ++i) acc[i] = fma(wp, v[i], acc[i]);
  }
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const double t = block_sum<RT>((double)acc[i], sh);
    if (threadIdx.x == 0) partial[(size_t)blockIdx.x * K + i] = t;
  }
}

// Pass 3: w -= V (h1 + h2) in place, and partial sums of ||w||^2.
template <int K, typename T>
__global__ void __launch_bounds__(RT) k_cgs_update(size_t n, T* __restrict__ w, const T* __restrict__ V, size_t ldv,
                                                   const double* __restrict__ h1, const double* __restrict__ h2,
                                                   double* __restrict__ partial) {
  __shared__ double sh[RT / 32];
  __shared__ T hs[K];
  if (threadIdx.x < K) hs[threadIdx.x] = (T)(h1[threadIdx.x] + h2[threadIdx.x]);
  __syncthreads();
  T acc = (T)0;
  for (size_t p = blockIdx.x * (size_t)RT + threadIdx.x; p < n; p += (size_t)gridDim.x * RT) {
    T wp = w[p];
#pragma unroll
    for (int i = 0; i < K; ++i) wp = fma(-hs[i], V[i * ldv + p], wp);
    w[p] = wp;
    acc = fma(wp, wp, acc);
  }
  const double t = block_sum<RT>((double)acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// FP32 forms of the two CGS kernels on float4 pieces (n and the row stride
// multiples of 4, rows 16-byte aligned): a quarter of the load instructions for
// the same bytes, so the passes run closer to HBM bandwidth.  K <= 16.
template <int K>
__global__ void __launch_bounds__(RT) k_cgs_dots_f4(size_t n4, const float4* __restrict__ w,
                                                    const float4* __restrict__ V, size_t ldv4,
                                                    const double* __restrict__ h, double* __restrict__ partial) {
  __shared__ double sh[RT / 32];
  __shared__ float hs[K];
  if (threadIdx.x < K) hs[threadIdx.x] = h ? (float)h[threadIdx.x] : 0.f;
  __syncthreads();
  float acc[K];
#pragma unroll
  for (int i = 0; i < K; ++i) acc[i] = 0.f;
  for (size_t p = blockIdx.x * (size_t)RT + threadIdx.x; p < n4; p += (size_t)gridDim.x * RT) {
    float4 v[K];
#pragma unroll
    for (int i = 0; i < K; ++i) v[i] = V[i * ldv4 + p];
    float4 wp = w[p];
    if (h) {
#pragma unroll
      for (int i = 0; i < K; ++i) {
        wp.x = fmaf(-hs[i], v[i].x, wp.x);
        wp.y = fmaf(-hs[i], v[i].y, wp.y);
        wp.z = fmaf(-hs[i], v[i].z, wp.z);
        wp.w = fmaf(-hs[i], v[i].w, wp.w);
      }
    }
#pragma unroll
    for (int i = 0; i < K; ++i)
      acc[i] = fmaf(wp.w, v[i].w, fmaf(wp.z, v[i].z, fmaf(wp.y, v[i].y, fmaf(wp.x, v[i].x, acc[i]))));
  }
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const double t = block_sum<RT>((double)acc[i], sh);
    if (threadIdx.x == 0) partial[(size_t)blockIdx.x * K + i] = t;
  }
}

template <int K>
__global__ void __launch_bounds__(RT) k_cgs_update_f4(size_t n4, float4* __restrict__ w, const float4* __restrict__ V,
                                                      size_t ldv4, const double* __restrict__ h1,
                                                      const double* __restrict__ h2, double* __restrict__ partial) {
  __shared__ double sh[RT / 32];
  __shared__ float hs[K];
  if (threadIdx.x < K) hs[threadIdx.x] = (float)(h1[threadIdx.x] + h2[threadIdx.x]);
  __syncthreads();
  float acc = 0.f;
  for (size_t p = blockIdx.x * (size_t)RT + threadIdx.x; p < n4; p += (size_t)gridDim.x * RT) {
    float4 wp = w[p];
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const float4 v = V[i * ldv4 + p];
      wp.x = fmaf(-hs[i], v.x, wp.x);
      wp.y = fmaf(-hs[i], v.y, wp.y);
      wp.z = fmaf(-hs[i], v.z, wp.z);
      wp.w = fmaf(-hs[i], v.w, wp.w);
    }
    w[p] = wp;
    acc = fmaf(wp.w, wp.w, fmaf(wp.z, wp.z, fmaf(wp.y, wp.y, fmaf(wp.x, wp.x, acc))));
  }
  const double t = block_sum<RT>((double)acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// ---- Gram matrix of a few FP32 vectors (the eigen estimate's Krylov basis) ----
// partial[b * NP + q], q running over the upper triangle i <= j row by row:
// block b's part of (v_i, v_j).  One pass reads each vector once, in float2
// pieces: the NP accumulators and two values per vector fit two blocks per
// SM.  Per-thread FP32 sums (reduce_blocks gives each thread at most about a
// thousand elements at the sizes of a level) and FP32 sums over a warp, then
// FP64 over the block's warps and over blocks: the NP block sums cost one
// barrier, not 2 NP, and no FP64 shuffle chains on the 1/64-rate FP64 pipe.
template <int NP>
__device__ __forceinline__ void gram_block_sums(const float (&acc)[NP], double* __restrict__ out) {
  __shared__ float red[RT / 32][NP];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    float t = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) red[warp][q] = t;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < NP; q += RT) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < RT / 32; ++w) t += (double)red[w][q];
    out[q] = t;
  }
}
template <int NV>
__global__ void __launch_bounds__(RT, 2) k_gram_f2(size_t n2, const float2* __restrict__ V, size_t ldv2,
                                                   double* __restrict__ partial) {
  constexpr int NP = NV * (NV + 1) / 2;
  float acc[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) acc[q] = 0.f;
  for (size_t p = blockIdx.x * (size_t)RT + threadIdx.x; p < n2; p += (size_t)gridDim.x * RT) {
    float2 v[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = V[i * ldv2 + p];
    int q = 0;
#pragma unroll
    for (int i = 0; i < NV; ++i)
#pragma unroll
      for (int j = i; j < NV; ++j, ++q) acc[q] = fmaf(v[i].y, v[j].y, fmaf(v[i].x, v[j].x, acc[q]));
  }
  gram_block_sums<NP>(acc, partial + (size_t)blockIdx.x * NP);
}

// The same on single elements (n or the row stride odd).
template <int NV>
__global__ void __launch_bounds__(RT) k_gram(size_t n, const float* __restrict__ V, size_t ldv,
                                             double* __restrict__ partial) {
  constexpr int NP = NV * (NV + 1) / 2;
  float acc[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) acc[q] = 0.f;
  for (size_t p = blockIdx.x * (size_t)RT + threadIdx.x; p < n; p += (size_t)gridDim.x * RT) {
    float v[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = V[i * ldv + p];
    int q = 0;
#pragma unroll
    for (int i = 0; i < NV; ++i)
#pragma unroll
      for (int j = i; j < NV; ++j, ++q) acc[q] = fmaf(v[i], v[j], acc[q]);
  }
  gram_block_sums<NP>(acc, partial + (size_t)blockIdx.x * NP);
}

// out = alpha t + beta v + gamma u (u null: gamma = 0), FP32 arithmetic.
template <typename T>
__global__ void k_three_term(size_t n, const T* __restrict__ t, const T* __restrict__ v, const T* __restrict__ u,
                             T* __restrict__ out, T alpha, T beta, T gamma) {
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
    T r = fma(alpha, t[p], beta * v[p]);
    if (u) r = fma(gamma, u[p], r);
    out[p] = r;
  }
}

__global__ void __launch_bounds__(RT) k_finalize(const double* __restrict__ partial, int nblocks, int k,
                                                 double* __restrict__ out, int accumulate) {
  __shared__ double sh[RT / 32];
  const int i = blockIdx.x;
  double v = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += RT) v += partial[(size_t)b * k + i];
  v = block_sum<RT>(v, sh);
  if (threadIdx.x == 0) out[i] = accumulate ? out[i] + v : v;
}

__global__ void __launch_bounds__(RT) k_finalize_norm(const double* __restrict__ partial, int nblocks,
                                                      double* __restrict__ out) {
  __shared__ double sh[RT / 32];
  double v = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += RT) v += partial[b];
  v = block_sum<RT>(v, sh);
  if (threadIdx.x == 0) {
    const double nrm = sqrt(v);
    out[0] = nrm;
    out[1] = (nrm != 0.0) ? 1.0 / nrm : 0.0;
  }
}

template <typename T>
__global__ void __launch_bounds__(RT) k_multi_axpy(size_t n, T* __restrict__ w, const T* __restrict__ V, size_t ldv,
                                                   int k, const double* __restrict__ h) {
  __shared__ T hs[64];
  if (threadIdx.x < k) hs[threadIdx.x] = (T)h[threadIdx.x];
  __syncthreads();
  for (size_t p = blockIdx.x * (size_t)RT + threadIdx.x; p < n; p += (size_t)gridDim.x * RT) {
    T v = w[p];
    for (int i = 0; i < k; ++i) v = fma(-hs[i], V[i * ldv + p], v);
    w[p] = v;
  }
}

template <typename T>
__global__ void k_scale(size_t n, const T* __restrict__ src, T* __restrict__ dst, const double* __restrict__ scale) {
  const T s = (T)scale[0];
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x)
    dst[p] = src[p] * s;
}

// FP32 dst = src * scale[0] on float4 pieces (n4 = n / 4; both arrays 16-byte aligned).
__global__ void k_scale_f4(size_t n4, const float4* __restrict__ src, float4* __restrict__ dst,
                           const double* __restrict__ scale) {
  const float s = (float)scale[0];
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n4; p += (size_t)gridDim.x * blockDim.x) {
    const float4 v = src[p];
    dst[p] = make_float4(v.x * s, v.y * s, v.z * s, v.w * s);
  }
}

__global__ void k_scale_value(size_t n, const double* __restrict__ src, double* __restrict__ dst, double s) {
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x)
    dst[p] = src[p] * s;
}

// dst = src * s (s = *scale, or alpha when scale is null) and dst32 = dst rounded
// to FP32: the new Arnoldi vector and the mixed-precision preconditioner's
// input in one pass (dst may be src).
__global__ void k_scale_round(size_t n, const double* src, double* dst, float* __restrict__ dst32,
                              const double* __restrict__ scale, double alpha) {
  const double s = scale ? scale[0] : alpha;
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
    const double v = src[p] * s;
    dst[p] = v;
    dst32[p] = f64_to_f32(v);
  }
}

template <typename TZ>
__global__ void __launch_bounds__(RT) k_update_solution(size_t n, double* __restrict__ x,
                                                        const TZ* __restrict__ Z, size_t ldz, int k,
                                                        const double* __restrict__ y) {
  __shared__ double ys[64];
  if (threadIdx.x < k) ys[threadIdx.x] = y[threadIdx.x];
  __syncthreads();
  for (size_t p = blockIdx.x * (size_t)RT + threadIdx.x; p < n; p += (size_t)gridDim.x * RT) {
    double v = x[p];
    for (int i = 0; i < k; ++i) v = fma(ys[i], to_f64(Z[i * ldz + p]), v);  // exact widening
    x[p] = v;
  }
}

// The same update for a fixed number of vectors: the K loads of an element are
// independent and issued together, and the sum runs as two interleaved FMA
// chains (even and odd i) added at the end.
template <int K, typename TZ>
__global__ void __launch_bounds__(RT) k_update_solution_k(size_t n, double* __restrict__ x,
                                                          const TZ* __restrict__ Z, size_t ldz,
                                                          const double* __restrict__ y) {
  __shared__ double ys[K];
  if (threadIdx.x < K) ys[threadIdx.x] = y[threadIdx.x];
  __syncthreads();
  for (size_t p = blockIdx.x * (size_t)RT + threadIdx.x; p < n; p += (size_t)gridDim.x * RT) {
    TZ zv[K];
#pragma unroll
    for (int i = 0; i < K; ++i) zv[i] = Z[i * ldz + p];
    double s0 = x[p], s1 = 0.0;
#pragma unroll
    for (int i = 0; i < K; i += 2) {
      s0 = fma(ys[i], to_f64(zv[i]), s0);
      if (i + 1 < K) s1 = fma(ys[i + 1], to_f64(zv[i + 1]), s1);
    }
    x[p] = s0 + s1;
  }
}

// The same update for FP32 Z (the mixed FGMRES): the sum s = Z y is formed in
// double-float arithmetic on the FP32 pipe and added to x with one FP64 add.
// Each y_i is split once per block into y_hi + y_lo (FP32, 48 bits together);
// y_hi z is exact as ph + pe (pe by FMA), y_lo z is rounded, and the terms are
// added with the two-sum of Knuth, so s carries about 2^-47 of the largest term
// (FP64 FMAs: about 2^-52).  The correction is added to an FP64 x, which keeps
// its own 53 bits; with GB300's FP64 rate at 1/64 of FP32, the K FP64 FMAs per
// element of the FP64 form bind it to the FP64 pipe.
template <int K>
__global__ void __launch_bounds__(RT) k_update_solution_df(size_t n, double* __restrict__ x,
                                                           const float* __restrict__ Z, size_t ldz,
                                                           const double* __restrict__ y) {
  __shared__ float yh[K], yl[K];
  if (threadIdx.x < K) {
    const double v = y[threadIdx.x];
    const float h = (float)v;
    yh[threadIdx.x] = h;
    yl[threadIdx.x] = (float)(v - (double)h);
  }
  __syncthreads();
  for (size_t p = blockIdx.x * (size_t)RT + threadIdx.x; p < n; p += (size_t)gridDim.x * RT) {
    float zv[K];
#pragma unroll
    for (int i = 0; i < K; ++i) zv[i] = Z[i * ldz + p];
    float sh = 0.f, sl = 0.f;
#pragma unroll
    for (int i = 0; i < K; ++i) {
      // rounded-operation intrinsics: no contraction into FMAs may change ph or the two-sum
      const float ph = __fmul_rn(yh[i], zv[i]);
      const float pl = fmaf(yl[i], zv[i], fmaf(yh[i], zv[i], -ph));
      const float t = __fadd_rn(sh, ph), bb = __fsub_rn(t, sh);
      const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bb)), __fsub_rn(ph, bb));
      sl = __fadd_rn(sl, __fadd_rn(err, pl));
      sh = t;
    }
    x[p] += f32_to_f64(sh) + f32_to_f64(sl);
  }
}

// out = a1 v1 + a2 v2 + a3 v3 in FP64 (the vector updates of CG, FCG, CGS and
// BiCGSTAB); FP32 terms are widened exactly, a null vector drops its term, and
// out may be v3 or a double v1 / v2 (each element is read before it is written).
template <typename T1, typename T2>
__global__ void __launch_bounds__(RT) k_lin3(size_t n, double a1, const T1* v1, double a2, const T2* v2, double a3,
                                             const double* v3, double* out) {
  for (size_t p = blockIdx.x * (size_t)RT + threadIdx.x; p < n; p += (size_t)gridDim.x * RT) {
    double s = 0.0;
    if (v1) s = a1 * to_f64(v1[p]);
    if (v2) s = fma(a2, to_f64(v2[p]), s);
    if (v3) s = fma(a3, v3[p], s);
    out[p] = s;
  }
}

__global__ void __launch_bounds__(RT) k_coef_check(size_t n, const double* __restrict__ a,
                                                   double* __restrict__ partial) {
  __shared__ double sh[RT / 32];
  __shared__ double shm[RT / 32];
  // On the integer pipe: a double is positive and finite exactly when its bit
  // pattern, as a signed 64-bit integer, lies strictly between 0 and that of
  // +infinity, and such doubles order like their patterns (NaN and negatives fail).
  long long mnb = __double_as_longlong(1.0e300);
  int badc = 0;
  for (size_t p = blockIdx.x * (size_t)RT + threadIdx.x; p < n; p += (size_t)gridDim.x * RT) {
    const long long b = __double_as_longlong(a[p]);
    if (b > 0 && b < 0x7FF0000000000000LL)
      mnb = b < mnb ? b : mnb;
    else
      ++badc;
  }
  double mn = __longlong_as_double(mnb), bad = (double)badc;
  // block min
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mn = fmin(mn, __shfl_down_sync(0xffffffffu, mn, o));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) shm[warp] = mn;
  __syncthreads();
  if (warp == 0) {
    double t = (lane < RT / 32) ? shm[lane] : 1.0e300;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = fmin(t, __shfl_down_sync(0xffffffffu, t, o));
    mn = t;
  }
  __syncthreads();
  const double nb = block_sum<RT>(bad, sh);
  if (threadIdx.x == 0) {
    partial[2 * (size_t)blockIdx.x] = mn;
    partial[2 * (size_t)blockIdx.x + 1] = nb;
  }
}

__global__ void k_finalize_check(const double* __restrict__ partial, int nblocks, double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double mn = 1.0e300, bad = 0.0;
  for (int b = 0; b < nblocks; ++b) {
    mn = fmin(mn, partial[2 * b]);
    bad += partial[2 * b + 1];
  }
  out[0] = mn;
  out[1] = bad;
}

// splitmix64 (Steele, Lea, Flood, OOPSLA 2014) at counter p: state = (p+1) * gamma.
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t p) {
  uint64_t z = (p + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_hash_vector(size_t n, double* __restrict__ u) {
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
    const uint64_t bits = splitmix64_at((uint64_t)p) >> 11;
    u[p] = (double)bits * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
  }
}

// FP32 start vector: the top 24 bits of the same splitmix64 draws, so the
// value is the FP64 start vector truncated to FP32 precision (no FP64 math).
__global__ void k_hash_vector_f32(size_t n, float* __restrict__ u) {
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
    const uint32_t bits = (uint32_t)(splitmix64_at((uint64_t)p) >> 40);
    u[p] = (float)bits * (1.0f / 16777216.0f) * 2.0f - 1.0f;
  }
}

inline unsigned flat_blocks(size_t n) {
  size_t b = (n + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  if (b == 0) b = 1;
  return (unsigned)b;
}

}  // namespace

int reduce_blocks(size_t n) {
  size_t b = (n + (size_t)RT * 8 - 1) / ((size_t)RT * 8);
  if (b > MAX_RBLOCKS) b = MAX_RBLOCKS;
  if (b < 1) b = 1;
  return (int)b;
}

template <typename T>
cudaError_t launch_multi_dot(size_t n, const T* w, const T* V, size_t ldv, int k, double* partial, cudaStream_t s) {
  const int nb = reduce_blocks(n);
  switch (k) {
#define GMG_CASE(K) \
  case K: k_multi_dot<K, T><<<nb, RT, 0, s>>>(n, w, V, ldv, partial); break;
    GMG_CASE(1) GMG_CASE(2) GMG_CASE(3) GMG_CASE(4) GMG_CASE(5) GMG_CASE(6) GMG_CASE(7) GMG_CASE(8)
#undef GMG_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_finalize(const double* partial, int nblocks, int k, double* out, int accumulate,
                            cudaStream_t s) {
  k_finalize<<<k, RT, 0, s>>>(partial, nblocks, k, out, accumulate);
  return cudaGetLastError();
}

cudaError_t launch_finalize_norm(const double* partial, int nblocks, double* out, cudaStream_t s) {
  k_finalize_norm<<<1, RT, 0, s>>>(partial, nblocks, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_multi_axpy(size_t n, T* w, const T* V, size_t ldv, int k, const double* h, cudaStream_t s) {
  if (k < 1 || k > 64) return cudaErrorInvalidValue;
  k_multi_axpy<T><<<reduce_blocks(n), RT, 0, s>>>(n, w, V, ldv, k, h);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scale(size_t n, const T* src, T* dst, const double* scale, cudaStream_t s) {
  if (std::is_same<T, float>::value && n % 4 == 0 && ((uintptr_t)src & 15) == 0 && ((uintptr_t)dst & 15) == 0) {
    k_scale_f4<<<flat_blocks(n / 4), 256, 0, s>>>(n / 4, reinterpret_cast<const float4*>(src),
                                                 reinterpret_cast<float4*>(dst), scale);
    return cudaGetLastError();
  }
  k_scale<T><<<flat_blocks(n), 256, 0, s>>>(n, src, dst, scale);
  return cudaGetLastError();
}

#define GMG_CASES32(X)                                                                                   \
  X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16) X(17) X(18) X(19) \
  X(20) X(21) X(22) X(23) X(24) X(25) X(26) X(27) X(28) X(29) X(30) X(31) X(32)
#define GMG_CASES16(X) \
  X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16)

namespace {
template <typename T>
bool f4_ok(size_t n, const T* w, const T* V, size_t ldv, int k) {
  return std::is_same<T, float>::value && k <= 16 && n % 4 == 0 && ldv % 4 == 0 && ((uintptr_t)w & 15) == 0 &&
         ((uintptr_t)V & 15) == 0;
}
}  // namespace

template <typename T>
cudaError_t launch_cgs_dots(size_t n, const T* w, const T* V, size_t ldv, int k, const double* h, double* partial,
                            cudaStream_t s) {
  const int nb = reduce_blocks(n);
  if (f4_ok(n, w, V, ldv, k)) {
    const float4* w4 = reinterpret_cast<const float4*>(w);
    const float4* V4 = reinterpret_cast<const float4*>(V);
    switch (k) {
#define GMG_CASE(K) \
  case K: k_cgs_dots_f4<K><<<nb, RT, 0, s>>>(n / 4, w4, V4, ldv / 4, h, partial); break;
      GMG_CASES16(GMG_CASE)
#undef GMG_CASE
      default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
  switch (k) {
#define GMG_CASE(K) \
  case K: k_cgs_dots<K, T><<<nb, RT, 0, s>>>(n, w, V, ldv, h, partial); break;
    GMG_CASES32(GMG_CASE)
#undef GMG_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cgs_update(size_t n, T* w, const T* V, size_t ldv, int k, const double* h1, const double* h2,
                              double* partial, cudaStream_t s) {
  const int nb = reduce_blocks(n);
  if (f4_ok(n, w, V, ldv, k)) {
    float4* w4 = reinterpret_cast<float4*>(w);
    const float4* V4 = reinterpret_cast<const float4*>(V);
    switch (k) {
#define GMG_CASE(K) \
  case K: k_cgs_update_f4<K><<<nb, RT, 0, s>>>(n / 4, w4, V4, ldv / 4, h1, h2, partial); break;
      GMG_CASES16(GMG_CASE)
#undef GMG_CASE
      default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
  switch (k) {
#define GMG_CASE(K) \
  case K: k_cgs_update<K, T><<<nb, RT, 0, s>>>(n, w, V, ldv, h1, h2, partial); break;
    GMG_CASES32(GMG_CASE)
#undef GMG_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

#define GMG_INST(T)                                                                                           \
  template cudaError_t launch_cgs_dots<T>(size_t, const T*, const T*, size_t, int, const double*, double*,   \
                                          cudaStream_t);                                                     \
  template cudaError_t launch_cgs_update<T>(size_t, T*, const T*, size_t, int, const double*, const double*, \
                                            double*, cudaStream_t);                                          \
  template cudaError_t launch_multi_dot<T>(size_t, const T*, const T*, size_t, int, double*, cudaStream_t);  \
  template cudaError_t launch_multi_axpy<T>(size_t, T*, const T*, size_t, int, const double*, cudaStream_t); \
  template cudaError_t launch_scale<T>(size_t, const T*, T*, const double*, cudaStream_t);
GMG_INST(float)
GMG_INST(double)
#undef GMG_INST

cudaError_t launch_gram(size_t n, const float* V, size_t ldv, int nv, double* partial, cudaStream_t s) {
  const int nb = reduce_blocks(n);
  if (n % 2 == 0 && ldv % 2 == 0 && ((uintptr_t)V & 7) == 0) {
    const float2* V2 = reinterpret_cast<const float2*>(V);
    switch (nv) {
#define GMG_CASE(K) \
  case K: k_gram_f2<K><<<nb, RT, 0, s>>>(n / 2, V2, ldv / 2, partial); break;
      GMG_CASE(2) GMG_CASE(3) GMG_CASE(4) GMG_CASE(5) GMG_CASE(6) GMG_CASE(7) GMG_CASE(8) GMG_CASE(9)
      GMG_CASE(10) GMG_CASE(11) GMG_CASE(12)
#undef GMG_CASE
      default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
  switch (nv) {
#define GMG_CASE(K) \
  case K: k_gram<K><<<nb, RT, 0, s>>>(n, V, ldv, partial); break;
    GMG_CASE(2) GMG_CASE(3) GMG_CASE(4) GMG_CASE(5) GMG_CASE(6) GMG_CASE(7) GMG_CASE(8) GMG_CASE(9)
    GMG_CASE(10) GMG_CASE(11) GMG_CASE(12)
#undef GMG_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_three_term(size_t n, const T* t, const T* v, const T* u, T* out, double alpha, double beta,
                              double gamma, cudaStream_t s) {
  k_three_term<T><<<flat_blocks(n), 256, 0, s>>>(n, t, v, u, out, (T)alpha, (T)beta, (T)gamma);
  return cudaGetLastError();
}
template cudaError_t launch_three_term<float>(size_t, const float*, const float*, const float*, float*, double,
                                              double, double, cudaStream_t);

cudaError_t launch_scale_value(size_t n, const double* src, double* dst, double alpha, cudaStream_t s) {
  k_scale_value<<<flat_blocks(n), 256, 0, s>>>(n, src, dst, alpha);
  return cudaGetLastError();
}

// out = [h1[0..k), h2[0..k), *nrm]: one Hessenberg column kept on the device.
__global__ void k_gather_column(const double* __restrict__ h1, const double* __restrict__ h2,
                                const double* __restrict__ nrm, int k, double* __restrict__ out) {
  for (int i = threadIdx.x; i <= 2 * k; i += blockDim.x) out[i] = i < k ? h1[i] : (i < 2 * k ? h2[i - k] : nrm[0]);
}

cudaError_t launch_gather_column(const double* h1, const double* h2, const double* nrm, int k, double* out,
                                 cudaStream_t s) {
  if (k < 1 || k > 64) return cudaErrorInvalidValue;
  k_gather_column<<<1, 128, 0, s>>>(h1, h2, nrm, k, out);
  return cudaGetLastError();
}

// A few words from device memory into mapped pinned host memory, written by
// the kernel itself: the copy engines may be busy with large transfers of
// another stream, and a small copy queued behind them would stall the host
// for their whole duration.
__global__ void k_words_to_host(const unsigned* __restrict__ src, unsigned* dst, int words) {
  for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
}

cudaError_t launch_words_to_host(const void* src, void* dst_mapped, size_t bytes, cudaStream_t s) {
  if (bytes % 4 != 0 || bytes > (size_t)1 << 20) return cudaErrorInvalidValue;
  if (bytes == 0) return cudaSuccess;
  k_words_to_host<<<1, 256, 0, s>>>((const unsigned*)src, (unsigned*)dst_mapped, (int)(bytes / 4));
  return cudaGetLastError();
}

// The same on pairs (n2 = n / 2; src, dst 16-byte and dst32 8-byte aligned).
__global__ void k_scale_round2(size_t n2, const double2* src, double2* dst, float2* __restrict__ dst32,
                               const double* __restrict__ scale, double alpha) {
  const double s = scale ? scale[0] : alpha;
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n2; p += (size_t)gridDim.x * blockDim.x) {
    const double2 v = src[p];
    const double2 r = make_double2(v.x * s, v.y * s);
    dst[p] = r;
    dst32[p] = make_float2(f64_to_f32(r.x), f64_to_f32(r.y));
  }
}

cudaError_t launch_scale_round(size_t n, const double* src, double* dst, float* dst32, const double* scale,
                               double alpha, cudaStream_t s) {
  if (n % 2 == 0 && ((uintptr_t)src & 15) == 0 && ((uintptr_t)dst & 15) == 0 && ((uintptr_t)dst32 & 7) == 0) {
    k_scale_round2<<<flat_blocks(n / 2), 256, 0, s>>>(n / 2, reinterpret_cast<const double2*>(src),
                                                     reinterpret_cast<double2*>(dst),
                                                     reinterpret_cast<float2*>(dst32), scale, alpha);
    return cudaGetLastError();
  }
  k_scale_round<<<flat_blocks(n), 256, 0, s>>>(n, src, dst, dst32, scale, alpha);
  return cudaGetLastError();
}

template <typename TZ>
cudaError_t launch_update_solution(size_t n, double* x, const TZ* Z, size_t ldz, int k, const double* y,
                                   cudaStream_t s) {
  if (k < 1 || k > 64) return cudaErrorInvalidValue;
  const int nb = reduce_blocks(n);
  if constexpr (std::is_same<TZ, float>::value) {
    switch (k) {
#define GMG_CASE(K) \
  case K: k_update_solution_df<K><<<nb, RT, 0, s>>>(n, x, Z, ldz, y); return cudaGetLastError();
      GMG_CASES32(GMG_CASE)
#undef GMG_CASE
      default: break;  // past 32 vectors: the FP64 form below
    }
  }
  switch (k) {
#define GMG_CASE(K) \
  case K: k_update_solution_k<K, TZ><<<nb, RT, 0, s>>>(n, x, Z, ldz, y); break;
    GMG_CASES32(GMG_CASE)
#undef GMG_CASE
    default: k_update_solution<TZ><<<nb, RT, 0, s>>>(n, x, Z, ldz, k, y);
  }
  return cudaGetLastError();
}
template cudaError_t launch_update_solution<float>(size_t, double*, const float*, size_t, int, const double*,
                                                   cudaStream_t);
template cudaError_t launch_update_solution<double>(size_t, double*, const double*, size_t, int, const double*,
                                                    cudaStream_t);

template <typename T1, typename T2>
cudaError_t launch_lin3(size_t n, double a1, const T1* v1, double a2, const T2* v2, double a3, const double* v3,
                        double* out, cudaStream_t s) {
  k_lin3<T1, T2><<<flat_blocks(n), RT, 0, s>>>(n, a1, v1, a2, v2, a3, v3, out);
  return cudaGetLastError();
}
template cudaError_t launch_lin3<double, double>(size_t, double, const double*, double, const double*, double,
                                                 const double*, double*, cudaStream_t);
template cudaError_t launch_lin3<float, double>(size_t, double, const float*, double, const double*, double,
                                                const double*, double*, cudaStream_t);
template cudaError_t launch_lin3<float, float>(size_t, double, const float*, double, const float*, double,
                                               const double*, double*, cudaStream_t);

template <typename T>
cudaError_t launch_mgs_step(size_t n, T* w, const T* vi, const T* vnext, const double* hi, double* partial,
                            cudaStream_t s) {
  k_mgs_step<T><<<reduce_blocks(n), RT, 0, s>>>(n, w, vi, vnext, hi, partial);
  return cudaGetLastError();
}
template cudaError_t launch_mgs_step<double>(size_t, double*, const double*, const double*, const double*, double*,
                                             cudaStream_t);
template cudaError_t launch_mgs_step<float>(size_t, float*, const float*, const float*, const double*, double*,
                                            cudaStream_t);

cudaError_t launch_coef_check(size_t n, const double* a, double* partial, cudaStream_t s) {
  k_coef_check<<<reduce_blocks(n), RT, 0, s>>>(n, a, partial);
  return cudaGetLastError();
}

cudaError_t launch_finalize_check(const double* partial, int nblocks, double* out, cudaStream_t s) {
  k_finalize_check<<<1, 32, 0, s>>>(partial, nblocks, out);
  return cudaGetLastError();
}

cudaError_t launch_hash_vector(size_t n, double* u, cudaStream_t s) {
  k_hash_vector<<<flat_blocks(n), 256, 0, s>>>(n, u);
  return cudaGetLastError();
}

cudaError_t launch_hash_vector(size_t n, float* u, cudaStream_t s) {
  k_hash_vector_f32<<<flat_blocks(n), 256, 0, s>>>(n, u);
  return cudaGetLastError();
}

}  // namespace gmg
