// The Arnoldi matrix-vector product w = A z_j of the mixed-precision FGMRES
// (Algorithm 1, Sec. 3.1) in double-float arithmetic.
//
// z_j is the FP32 output of the V-cycle; the coefficient a and the result w
// are FP64.  GB300 executes FP64 instructions (conversions included) at 1/64
// of the FP32 rate, so the 7-point operator of eq. (e18) is evaluated with
// pairs of FP32 numbers (hi + lo, a 48-bit significand) built from
// error-free transformations: Knuth's TwoSum, Dekker's FastTwoSum and the
// FMA-based exact product.  The coefficient is stored split as (hi, lo)
// FP32 pairs, the differences z_p - z_q are exact, and every product and sum
// carries its rounding error; only the final (double)hi + (double)lo uses
// the FP64 pipe.  The result agrees with an FP64 evaluation to about 1e-14
// relative, far below the 1e-8 stopping tolerance.
#include "gmg_internal.cuh"

namespace gmg {

namespace {

struct df {
  float h, l;
};

// s + e = a + b exactly (Knuth).
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}

// s + e = a + b exactly when |a| >= |b| (Dekker).
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}

__device__ __forceinline__ df df_add(df a, df b) {
  const df s = two_sum(a.h, b.h);
  return fast_two_sum(s.h, s.l + (a.l + b.l));
}

__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);  // exact rounding error of the leading product
  e = fmaf(a.h, b.l, fmaf(a.l, b.h, e));
  return fast_two_sum(p, e);
}

__global__ void __launch_bounds__(256) k_apply_df64(Grid3 g, DfCoef c, const float2* __restrict__ a2,
                                                    const float* __restrict__ z, double* __restrict__ w) {
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y * 8 + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  const int nx = g.nx;
  const size_t pl = g.plane();
  const size_t p = ((size_t)k * g.ny + j) * nx + i;
  const float2 apv = __ldg(a2 + p);
  const df ap = {apv.x, apv.y};
  const float zp = __ldg(z + p);
  auto face = [&](size_t q, df acc) {
    const float2 aq = __ldg(a2 + q);
    const df s = df_add(ap, df{aq.x, aq.y});      // a_p + a_q
    const df d = two_sum(zp, -__ldg(z + q));      // z_p - z_q, exact
    return df_add(acc, df_mul(s, d));
  };
  df sx = {0.f, 0.f}, sy = {0.f, 0.f}, sz = {0.f, 0.f}, sp = {0.f, 0.f};
  if (i > 0) sx = face(p - 1, sx);
  if (i < nx - 1) sx = face(p + 1, sx);
  if (j > 0) sy = face(p - nx, sy);
  if (j < g.ny - 1) sy = face(p + nx, sy);
  if (k > 0) sz = face(p - pl, sz);
  else sp = df_add(sp, df_mul(ap, df{zp, 0.f}));
  if (k < g.nz - 1) sz = face(p + pl, sz);
  else sp = df_add(sp, df_mul(ap, df{zp, 0.f}));
  df t = df_mul(sx, df{c.xh, c.xl});
  t = df_add(t, df_mul(sy, df{c.yh, c.yl}));
  t = df_add(t, df_mul(sz, df{c.zh, c.zl}));
  t = df_add(t, df_mul(sp, df{c.ph, c.pl}));
  w[p] = (double)t.h + (double)t.l;
}

// a2[p] = (hi, lo) with hi = fl32(a), lo = fl32(a - hi).
__global__ void k_split(size_t n, const double* __restrict__ a, float2* __restrict__ a2) {
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
    const double v = a[p];
    const float h = (float)v;
    a2[p] = make_float2(h, (float)(v - (double)h));
  }
}

}  // namespace

DfCoef make_df_coef(const Grid3& g) {
  auto split = [](double v, float& h, float& l) {
    h = (float)v;
    l = (float)(v - (double)h);
  };
  DfCoef c;
  split(g.cx, c.xh, c.xl);
  split(g.cy, c.yh, c.yl);
  split(g.cz, c.zh, c.zl);
  split(g.cp, c.ph, c.pl);  // plate face: a_p z_p * 2/hz^2
  return c;
}

cudaError_t launch_apply_df64(const Grid3& g, const DfCoef& c, const float2* a2, const float* z, double* w,
                              cudaStream_t s) {
  dim3 grid((unsigned)((g.nx + 31) / 32), (unsigned)((g.ny + 7) / 8), (unsigned)g.nz);
  k_apply_df64<<<grid, dim3(32, 8), 0, s>>>(g, c, a2, z, w);
  return cudaGetLastError();
}

cudaError_t launch_split(size_t n, const double* a, float2* a2, cudaStream_t s) {
  size_t b = (n + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  if (b == 0) b = 1;
  k_split<<<(unsigned)b, 256, 0, s>>>(n, a, a2);
  return cudaGetLastError();
}

}  // namespace gmg
