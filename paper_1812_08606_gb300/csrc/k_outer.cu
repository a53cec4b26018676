// The Arnoldi matrix-vector product w = A z_j of the mixed-precision FGMRES
// (Algorithm 1, Sec. 3.1) in double-float arithmetic.
//
// z_j is the FP32 output of the V-cycle; the coefficient a and the result w
// are FP64.  GB300 executes FP64 instructions (conversions included) at 1/64
// of the FP32 rate, so the 7-point operator of eq. (e18) is evaluated with
// pairs of FP32 numbers (hi + lo, a 48-bit significand) built from
// error-free transformations: Knuth's TwoSum and the FMA-based exact product.
// The coefficient is stored split as (hi, lo) FP32 pairs and the differences
// z_p - z_q are exact; every product and sum carries its rounding error into
// a low word that is renormalised only by the final FP64 add of the two
// words.  The result agrees with an FP64 evaluation to about 1e-14 relative,
// far below the 1e-8 stopping tolerance.
#include <stdint.h>

#include <algorithm>

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

// acc += (ph + pl): the leading parts are added exactly (TwoSum) and every
// rounding error is gathered in the low word, which is not renormalised until
// the end (the final FP64 add of the two words does that).
__device__ __forceinline__ void acc_add(df& acc, float ph, float pl) {
  const df s = two_sum(acc.h, ph);
  acc.h = s.h;
  acc.l += s.l + pl;
}

// (sh + sl)(dh + dl) to double-float accuracy: the leading product exactly
// by FMA, the cross terms once rounded (sl dl is below the working precision).
__device__ __forceinline__ df mul_df(float sh, float sl, float dh, float dl) {
  const float ph = sh * dh;
  float pl = fmaf(sh, dh, -ph);
  pl = fmaf(sh, dl, fmaf(sl, dh, pl));
  return {ph, pl};
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
  const float2 ap = __ldg(a2 + p);
  const float zp = __ldg(z + p);
  // one interior face: acc += (a_p + a_q)(z_p - z_q); the coefficient sum keeps
  // its low parts, the difference of two floats is exact as a pair
  auto face = [&](size_t q, df& acc) {
    const float2 aq = __ldg(a2 + q);
    df sa = two_sum(ap.x, aq.x);
    sa.l += ap.y + aq.y;
    const df d = two_sum(zp, -__ldg(z + q));
    const df t = mul_df(sa.h, sa.l, d.h, d.l);
    acc_add(acc, t.h, t.l);
  };
  df sx = {0.f, 0.f}, sy = {0.f, 0.f}, sz = {0.f, 0.f}, sp = {0.f, 0.f};
  if (i > 0) face(p - 1, sx);
  if (i < nx - 1) face(p + 1, sx);
  if (j > 0) face(p - nx, sy);
  if (j < g.ny - 1) face(p + nx, sy);
  // plate faces: a_p z_p per plate (the factor 2/hz^2 is in the plate coefficient)
  const df az = mul_df(ap.x, ap.y, zp, 0.f);
  if (k > 0) face(p - pl, sz);
  else acc_add(sp, az.h, az.l);
  if (k < g.nz - 1) face(p + pl, sz);
  else acc_add(sp, az.h, az.l);
  df t = mul_df(sx.h, sx.l, c.xh, c.xl);
  df u = mul_df(sy.h, sy.l, c.yh, c.yl);
  acc_add(t, u.h, u.l);
  u = mul_df(sz.h, sz.l, c.zh, c.zl);
  acc_add(t, u.h, u.l);
  u = mul_df(sp.h, sp.l, c.ph, c.pl);
  acc_add(t, u.h, u.l);
  w[p] = (double)t.h + (double)t.l;
}

// ---------------------------------------------------------------------------
// The same product with one thread per cell pair (2 ip, 2 ip + 1) of a row:
// the double-float arithmetic of both cells runs in packed FP32x2 (each lane
// performs exactly the operations of the one-cell kernel, in the same face
// order), a and z are read as float4 / float2 (the (hi, lo) pairs of both
// cells), x-neighbours come from the neighbouring lanes by shuffle, and the
// planes above and below stay in registers while a block marches along z.
// ---------------------------------------------------------------------------
struct df2 {
  float2 h, l;
};

__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 neg2(float2 a) { return f2(-a.x, -a.y); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ df2 two_sum2(float2 a, float2 b) {
  const float2 s = add2(a, b);
  const float2 bb = sub2(s, a);
  return {s, add2(sub2(a, sub2(s, bb)), sub2(b, bb))};
}
__device__ __forceinline__ void acc_add2(df2& acc, float2 ph, float2 pl) {
  const df2 s = two_sum2(acc.h, ph);
  acc.h = s.h;
  acc.l = add2(acc.l, add2(s.l, pl));
}
__device__ __forceinline__ df2 mul_df2(float2 sh, float2 sl, float2 dh, float2 dl) {
  const float2 ph = mul2(sh, dh);
  float2 pl = fma2(sh, dh, neg2(ph));
  pl = fma2(sh, dl, fma2(sl, dh, pl));
  return {ph, pl};
}
// acc += (a_p + a_q)(z_p - z_q) for both cells
__device__ __forceinline__ void face2(df2& acc, float2 aph, float2 apl, float2 aqh, float2 aql, float2 zp,
                                      float2 zq) {
  df2 sa = two_sum2(aph, aqh);
  sa.l = add2(sa.l, add2(apl, aql));
  const df2 d = two_sum2(zp, neg2(zq));
  const df2 t = mul_df2(sa.h, sa.l, d.h, d.l);
  acc_add2(acc, t.h, t.l);
}

constexpr unsigned FULL = 0xffffffffu;

__global__ void __launch_bounds__(256) k_apply_df64_pairs(Grid3 g, DfCoef c, const float4* __restrict__ a4,
                                                          const float2* __restrict__ z2, double2* __restrict__ w2,
                                                          int kchunk) {
  const int ny = g.ny, nz = g.nz, np = g.nx / 2;  // pairs per row
  const int tx = threadIdx.x;
  const int ip = blockIdx.x * 32 + tx, j = blockIdx.y * 8 + threadIdx.y;
  const int k0 = blockIdx.z * kchunk, k1 = min(nz, k0 + kchunk);
  const bool act = ip < np && j < ny;
  // pair offsets in 32 bits: the launcher keeps (nz + 2) planes of pairs below 2^31
  const int pp = ny * np;  // pairs per plane
  const int q = act ? j * np + ip : 0;
  const bool lds = act && j > 0, ldn = act && j < ny - 1;
  const bool ldl = act && tx == 0 && ip > 0, ldr = act && tx == 31 && ip + 1 < np;
  const bool wl = ip > 0, wr = ip + 1 < np;  // the row continues left of / right of the pair
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  const float2 zz = f2(0.f, 0.f);
  auto la = [&](int k) { return (act && k >= 0 && k < nz) ? __ldg(a4 + (k * pp + q)) : z4; };
  auto lz = [&](int k) { return (act && k >= 0 && k < nz) ? __ldg(z2 + (k * pp + q)) : zz; };
  const float2 cxh = f2(c.xh, c.xh), cxl = f2(c.xl, c.xl), cyh = f2(c.yh, c.yh), cyl = f2(c.yl, c.yl);
  const float2 czh = f2(c.zh, c.zh), czl = f2(c.zl, c.zl), cph = f2(c.ph, c.ph), cpl = f2(c.pl, c.pl);
  float4 am = la(k0 - 1), ac = la(k0);
  float2 zm = lz(k0 - 1), zc = lz(k0);
  for (int k = k0; k < k1; ++k) {
    const float4 ap = la(k + 1);
    const float2 zp = lz(k + 1);
    const int o = k * pp + q;
    const float4 as = lds ? __ldg(a4 + o - np) : z4, an = ldn ? __ldg(a4 + o + np) : z4;
    const float2 zs = lds ? __ldg(z2 + o - np) : zz, zn = ldn ? __ldg(z2 + o + np) : zz;
    // the left pair's second cell and the right pair's first cell
    float alh = __shfl_up_sync(FULL, ac.z, 1), all = __shfl_up_sync(FULL, ac.w, 1);
    float zl = __shfl_up_sync(FULL, zc.y, 1);
    float arh = __shfl_down_sync(FULL, ac.x, 1), arl = __shfl_down_sync(FULL, ac.y, 1);
    float zr = __shfl_down_sync(FULL, zc.x, 1);
    if (ldl) {
      const float4 t = __ldg(a4 + o - 1);
      alh = t.z;
      all = t.w;
      zl = __ldg(z2 + o - 1).y;
    }
    if (ldr) {
      const float4 t = __ldg(a4 + o + 1);
      arh = t.x;
      arl = t.y;
      zr = __ldg(z2 + o + 1).x;
    }
    // a side wall: the missing neighbour copies the cell, so its face adds an exact zero
    if (!wl) {
      alh = ac.x;
      all = ac.y;
      zl = zc.x;
    }
    if (!wr) {
      arh = ac.z;
      arl = ac.w;
      zr = zc.y;
    }
    if (act) {
      const float2 aph = f2(ac.x, ac.z), apl = f2(ac.y, ac.w);
      df2 sx = {zz, zz}, sy = {zz, zz}, sz = {zz, zz}, sp = {zz, zz};
      face2(sx, aph, apl, f2(alh, ac.x), f2(all, ac.y), zc, f2(zl, zc.x));
      face2(sx, aph, apl, f2(ac.z, arh), f2(ac.w, arl), zc, f2(zc.y, zr));
      if (j > 0) face2(sy, aph, apl, f2(as.x, as.z), f2(as.y, as.w), zc, zs);
      if (j < ny - 1) face2(sy, aph, apl, f2(an.x, an.z), f2(an.y, an.w), zc, zn);
      const df2 az = mul_df2(aph, apl, zc, zz);
      if (k > 0) face2(sz, aph, apl, f2(am.x, am.z), f2(am.y, am.w), zc, zm);
      else acc_add2(sp, az.h, az.l);
      if (k < nz - 1) face2(sz, aph, apl, f2(ap.x, ap.z), f2(ap.y, ap.w), zc, zp);
      else acc_add2(sp, az.h, az.l);
      df2 t = mul_df2(sx.h, sx.l, cxh, cxl);
      df2 u = mul_df2(sy.h, sy.l, cyh, cyl);
      acc_add2(t, u.h, u.l);
      u = mul_df2(sz.h, sz.l, czh, czl);
      acc_add2(t, u.h, u.l);
      u = mul_df2(sp.h, sp.l, cph, cpl);
      acc_add2(t, u.h, u.l);
      w2[o] = make_double2((double)t.h.x + (double)t.l.x, (double)t.h.y + (double)t.l.y);
    }
    am = ac;
    ac = ap;
    zm = zc;
    zc = zp;
  }
}

// a2[p] = (hi, lo) with hi = fl32(a), lo = fl32(a - hi).
__global__ void k_split(size_t n, const double* __restrict__ a, float2* __restrict__ a2) {
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
    const double v = a[p];
    const float h = f64_to_f32(v);  // conversions on the integer pipe; only the subtraction is FP64
    a2[p] = make_float2(h, f64_to_f32(v - f32_to_f64(h)));
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
  // pair kernel: even rows, 16-byte (a, w) / 8-byte (z) alignment of the pair arrays, and fewer than 2^31
  // cell pairs in nz + 2 planes (32-bit offsets)
  const bool pairs_fit = (size_t)(g.nz + 2) * (g.plane() / 2) < ((size_t)1 << 31);
  if (g.nx % 2 == 0 && pairs_fit && ((uintptr_t)a2 & 15) == 0 && ((uintptr_t)z & 7) == 0 &&
      ((uintptr_t)w & 15) == 0) {
    const int gx = (g.nx / 2 + 31) / 32, gy = (g.ny + 7) / 8;
    const long long xy = (long long)gx * gy, target = 152LL * 8 * 2;
    int zc = (int)std::max(1LL, std::min((target + xy - 1) / xy, (long long)std::max(1, g.nz / 4)));
    const int kchunk = (g.nz + zc - 1) / zc;
    zc = (g.nz + kchunk - 1) / kchunk;
    k_apply_df64_pairs<<<dim3((unsigned)gx, (unsigned)gy, (unsigned)zc), dim3(32, 8), 0, s>>>(
        g, c, reinterpret_cast<const float4*>(a2), reinterpret_cast<const float2*>(z), reinterpret_cast<double2*>(w),
        kchunk);
    return cudaGetLastError();
  }
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
