// FP32 grid transfers of the V-cycle (Appendix A), laid out for coalesced
// 64-bit access:
//
//   restriction:   b_c = mean over the 8 children of (b - A x)        (fused residual)
//   prolongation:  x += P e_c, cell-centred trilinear (3/4, 1/4 per axis) or
//                  piecewise constant
//
// The operator is the 7-point stencil of eq. (e18).  Both kernels give each
// thread one fine cell pair (2 ic, 2 ic + 1) of one row, i.e. one coarse
// x-index ic, so a warp reads and writes 64 consecutive cells as float2 and
// the x-neighbours of a pair come from the neighbouring lanes by shuffle.  A
// block of 32 x 8 threads covers 64 x 8 fine cells and marches through a
// range of z-planes, keeping the planes above and below in registers.
#include <algorithm>

#include "gmg_internal.cuh"

namespace gmg {

namespace {

constexpr int TP = 32;  // pairs per row = lanes
constexpr int TR = 8;   // fine rows per block (even)
constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, f2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Number of blocks along z for `planes` planes: about two waves of 8 blocks per
// SM in total, at least `min_planes` planes per block.
int z_chunks(long long xy_blocks, int planes, int min_planes) {
  const long long target = 152LL * 8 * 2;
  long long c = (target + xy_blocks - 1) / xy_blocks;
  c = std::max(1LL, std::min(c, (long long)std::max(1, planes / min_planes)));
  return (int)c;
}

// ---------------------------------------------------------------------------
// Fused residual + restriction.  Thread (tx, ty): pair ip = bx 32 + tx and the
// two fine rows j0 = 2 jc, j0 + 1 of coarse row jc = by 8 + ty; coarse planes
// [kc0, kc1).  Per fine plane the thread forms r of its four cells (each row
// is the other's y-neighbour, so only the rows j0 - 1 and j0 + 2 are loaded
// besides its own) and adds them to a running sum; after the second plane of a
// coarse plane it writes the mean of the eight children.
// ---------------------------------------------------------------------------
struct RowWin {  // one fine row's x and a at planes k-1, k, k+1
  float2 xm, xc, xp, am, ac, ap;
};

__device__ __forceinline__ float2 pair_residual(const Grid3& g, const RowWin& w, float2 bb, float xl, float al,
                                               float xr, float ar, float mxl, float mxr, float2 as, float2 xs,
                                               float ms, float2 an, float2 xn, float mn, bool zlo, bool zhi) {
  const float2 z2 = f2(0.f, 0.f);
  const float2 fx2 = f2(g.fx, g.fx), fy2 = f2(g.fy, g.fy), fz2 = f2(g.fz, g.fz), fp2 = f2(g.fp, g.fp);
  const float2 ac = w.ac, xc = w.xc;
  const float2 fxm = mul2(add2(ac, f2(al, ac.x)), f2(mxl, 1.f));
  const float2 fxp = mul2(add2(ac, f2(ac.y, ar)), f2(1.f, mxr));
  float2 sx = mul2(fxm, sub2(xc, f2(xl, xc.x)));
  sx = fma2(fxp, sub2(xc, f2(xc.y, xr)), sx);
  float2 sy = mul2(mul2(add2(ac, as), f2(ms, ms)), sub2(xc, xs));
  sy = fma2(mul2(add2(ac, an), f2(mn, mn)), sub2(xc, xn), sy);
  const float2 plate = add2(zlo ? z2 : ac, zhi ? z2 : ac);
  float2 sz = mul2(fp2, mul2(plate, xc));
  if (zlo) sz = fma2(fz2, mul2(add2(ac, w.am), sub2(xc, w.xm)), sz);
  if (zhi) sz = fma2(fz2, mul2(add2(ac, w.ap), sub2(xc, w.xp)), sz);
  return sub2(bb, fma2(fx2, sx, fma2(fy2, sy, sz)));
}

__global__ void __launch_bounds__(TP* TR, 3) k_restrict_pairs(Grid3 g, const float* __restrict__ a,
                                                           const float* __restrict__ b,
                                                           const float* __restrict__ x, float* __restrict__ coarse,
                                                           int kchunk) {
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int nxc = nx / 2, nyc = ny / 2, nzc = nz / 2;
  const int tx = threadIdx.x;
  const int ip = blockIdx.x * TP + tx;
  const int jc = blockIdx.y * TR + threadIdx.y;  // coarse row
  const int j0 = 2 * jc;                          // its first fine row
  const int kc0 = blockIdx.z * kchunk, kc1 = min(nzc, kc0 + kchunk);
  const bool act = ip < nxc && jc < nyc;
  const int i0 = 2 * ip;
  // offsets in 32 bits: the launcher keeps nz + 4 planes of cells below 2^31
  const int pl2 = (int)(g.plane() >> 1);
  const int rs = nx >> 1;                          // pairs per row
  const int q = act ? (j0 * nx + i0) >> 1 : 0;    // pair offset of row j0 in a plane
  const float2* A2 = reinterpret_cast<const float2*>(a);
  const float2* X2 = reinterpret_cast<const float2*>(x);
  const float2* B2 = reinterpret_cast<const float2*>(b);
  const float mxl = i0 > 0 ? 1.f : 0.f, mxr = i0 + 2 < nx ? 1.f : 0.f;
  const float ms = j0 > 0 ? 1.f : 0.f, mn = j0 + 2 < ny ? 1.f : 0.f;  // faces below row j0, above row j0 + 1
  const bool ldl = act && tx == 0 && i0 > 0;            // left neighbour outside the warp
  const bool ldr = act && tx == TP - 1 && i0 + 2 < nx;  // right neighbour outside the warp
  const bool lds = act && j0 > 0, ldn = act && j0 + 2 < ny;
  const float2 z2 = f2(0.f, 0.f);
  auto load = [&](const float2* P, int k, int row) {
    return (act && k >= 0 && k < nz) ? __ldg(P + (k * pl2 + q + row * rs)) : z2;
  };

  const int k0 = 2 * kc0, k1 = 2 * kc1;
  RowWin w0{load(X2, k0 - 1, 0), load(X2, k0, 0), load(X2, k0 + 1, 0),
            load(A2, k0 - 1, 0), load(A2, k0, 0), load(A2, k0 + 1, 0)};
  RowWin w1{load(X2, k0 - 1, 1), load(X2, k0, 1), load(X2, k0 + 1, 1),
            load(A2, k0 - 1, 1), load(A2, k0, 1), load(A2, k0 + 1, 1)};
  float s = 0.f;
  for (int k = k0; k < k1; ++k) {
    const float2 xq0 = load(X2, k + 2, 0), aq0 = load(A2, k + 2, 0);
    const float2 xq1 = load(X2, k + 2, 1), aq1 = load(A2, k + 2, 1);
    const int o = k * pl2 + q;
    const float2 b0 = act ? __ldg(B2 + o) : z2, b1 = act ? __ldg(B2 + o + rs) : z2;
    const float2 xs = lds ? __ldg(X2 + o - rs) : z2, as = lds ? __ldg(A2 + o - rs) : z2;
    const float2 xn = ldn ? __ldg(X2 + o + 2 * rs) : z2, an = ldn ? __ldg(A2 + o + 2 * rs) : z2;
    // x-neighbours: lane - 1 holds cell i0 - 1 in .y, lane + 1 holds i0 + 2 in .x
    float xl0 = __shfl_up_sync(FULL, w0.xc.y, 1), al0 = __shfl_up_sync(FULL, w0.ac.y, 1);
    float xr0 = __shfl_down_sync(FULL, w0.xc.x, 1), ar0 = __shfl_down_sync(FULL, w0.ac.x, 1);
    float xl1 = __shfl_up_sync(FULL, w1.xc.y, 1), al1 = __shfl_up_sync(FULL, w1.ac.y, 1);
    float xr1 = __shfl_down_sync(FULL, w1.xc.x, 1), ar1 = __shfl_down_sync(FULL, w1.ac.x, 1);
    if (tx == 0) {
      xl0 = ldl ? __ldg(x + 2 * o - 1) : 0.f;
      al0 = ldl ? __ldg(a + 2 * o - 1) : 0.f;
      xl1 = ldl ? __ldg(x + 2 * (o + rs) - 1) : 0.f;
      al1 = ldl ? __ldg(a + 2 * (o + rs) - 1) : 0.f;
    }
    if (tx == TP - 1) {
      xr0 = ldr ? __ldg(x + 2 * o + 2) : 0.f;
      ar0 = ldr ? __ldg(a + 2 * o + 2) : 0.f;
      xr1 = ldr ? __ldg(x + 2 * (o + rs) + 2) : 0.f;
      ar1 = ldr ? __ldg(a + 2 * (o + rs) + 2) : 0.f;
    }
    if (act) {
      const bool zlo = k > 0, zhi = k < nz - 1;
      // row j0: below it row j0 - 1, above it row j0 + 1; row j0 + 1: below j0, above j0 + 2
      const float2 r0 = pair_residual(g, w0, b0, xl0, al0, xr0, ar0, mxl, mxr, as, xs, ms, w1.ac, w1.xc, 1.f, zlo,
                                      zhi);
      const float2 r1 = pair_residual(g, w1, b1, xl1, al1, xr1, ar1, mxl, mxr, w0.ac, w0.xc, 1.f, an, xn, mn, zlo,
                                      zhi);
      s += (r0.x + r0.y) + (r1.x + r1.y);
    }
    if (k & 1) {
      if (act) coarse[((k >> 1) * nyc + jc) * nxc + ip] = 0.125f * s;
      s = 0.f;
    }
    w0.xm = w0.xc; w0.xc = w0.xp; w0.xp = xq0;
    w0.am = w0.ac; w0.ac = w0.ap; w0.ap = aq0;
    w1.xm = w1.xc; w1.xc = w1.xp; w1.xp = xq1;
    w1.am = w1.ac; w1.ac = w1.ap; w1.ap = aq1;
  }
}

// ---------------------------------------------------------------------------
// x += P e.  Thread (tx, ty): pair ip = bx 32 + tx (coarse column ic = ip),
// fine row j = by 8 + ty; coarse planes [kc0, kc1), i.e. fine planes
// [2 kc0, 2 kc1).  Per axis a child takes 3/4 of its parent and 1/4 of the
// neighbour on its side; beyond the domain that neighbour is a ghost equal to
// the parent (Neumann, x/y) or minus the parent (homogeneous Dirichlet, z).
// The thread interpolates its own coarse column in y and z (a window of three
// coarse planes x two coarse rows in registers), then takes the columns ic - 1
// and ic + 1 from the neighbouring lanes; the first and last lane interpolate
// the column just outside the warp themselves.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(TP* TR) k_prolong_pairs(Grid3 g, const float* __restrict__ e,
                                                          float* __restrict__ x, int mode, int kchunk) {
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int nxc = nx / 2, nyc = ny / 2, nzc = nz / 2;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int ip = blockIdx.x * TP + tx;
  const int j = blockIdx.y * TR + ty;
  const int kc0 = blockIdx.z * kchunk, kc1 = min(nzc, kc0 + kchunk);
  const bool act = ip < nxc && j < ny;
  const int jc = j >> 1;
  int jn = (j & 1) ? jc + 1 : jc - 1;
  if (jn < 0 || jn >= nyc) jn = jc;  // Neumann ghost = parent
  // the halo column of the edge lanes
  const int ih = tx == 0 ? ip - 1 : (tx == TP - 1 ? ip + 1 : -1);
  const bool hact = act && ih >= 0 && ih < nxc;
  // offsets in 32 bits: the launcher keeps nz + 4 planes of fine cells below 2^31
  const int pc = nyc * nxc;
  const int rc = act ? jc * nxc : 0, rn = act ? jn * nxc : 0;
  auto ld = [&](bool on, int kc, int row, int col) {
    return (on && kc >= 0 && kc < nzc) ? __ldg(e + (kc * pc + row + col)) : 0.f;
  };
  // window of coarse planes kc - 1, kc, kc + 1: rows (jc, jn), own column and halo column
  float c0m = ld(act, kc0 - 1, rc, ip), n0m = ld(act, kc0 - 1, rn, ip);
  float c0 = ld(act, kc0, rc, ip), n0 = ld(act, kc0, rn, ip);
  float c0p = ld(act, kc0 + 1, rc, ip), n0p = ld(act, kc0 + 1, rn, ip);
  float h0m = ld(hact, kc0 - 1, rc, ih), g0m = ld(hact, kc0 - 1, rn, ih);
  float h0 = ld(hact, kc0, rc, ih), g0 = ld(hact, kc0, rn, ih);
  float h0p = ld(hact, kc0 + 1, rc, ih), g0p = ld(hact, kc0 + 1, rn, ih);
  const int pl2 = (int)(g.plane() >> 1);
  const int q = act ? (j * nx + 2 * ip) >> 1 : 0;
  float2* X2 = reinterpret_cast<float2*>(x);
  for (int kc = kc0; kc < kc1; ++kc) {
    const float c1 = ld(act, kc + 2, rc, ip), n1 = ld(act, kc + 2, rn, ip);
    const float h1 = ld(hact, kc + 2, rc, ih), g1 = ld(hact, kc + 2, rn, ih);
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int k = 2 * kc + half;
      float own, halo;
      if (mode == 1) {
        own = c0;
        halo = h0;
      } else {
        // y first, then z; the z-neighbour plane is below for even k, above for odd k
        const bool kin = half ? kc + 1 < nzc : kc > 0;
        const float wz = kin ? 0.25f : -0.25f;
        const float ycen = fmaf(0.75f, c0, 0.25f * n0), hcen = fmaf(0.75f, h0, 0.25f * g0);
        const float yn = kin ? (half ? fmaf(0.75f, c0p, 0.25f * n0p) : fmaf(0.75f, c0m, 0.25f * n0m)) : ycen;
        const float hn = kin ? (half ? fmaf(0.75f, h0p, 0.25f * g0p) : fmaf(0.75f, h0m, 0.25f * g0m)) : hcen;
        own = fmaf(0.75f, ycen, wz * yn);
        halo = fmaf(0.75f, hcen, wz * hn);
      }
      float left = __shfl_up_sync(FULL, own, 1), right = __shfl_down_sync(FULL, own, 1);
      if (tx == 0) left = halo;
      if (tx == TP - 1) right = halo;
      if (ip == 0) left = own;             // Neumann ghost = parent
      if (ip == nxc - 1) right = own;
      if (act) {
        const int o = k * pl2 + q;
        const float2 v = mode == 1 ? f2(own, own) : f2(fmaf(0.75f, own, 0.25f * left), fmaf(0.75f, own, 0.25f * right));
        X2[o] = add2(X2[o], v);
      }
    }
    c0m = c0; n0m = n0; c0 = c0p; n0 = n0p; c0p = c1; n0p = n1;
    h0m = h0; g0m = g0; h0 = h0p; g0 = g0p; h0p = h1; g0p = g1;
  }
}

}  // namespace

cudaError_t launch_restrict_pairs(const Grid3& g, const float* a, const float* b, const float* x, float* coarse,
                                  cudaStream_t s) {
  if (!pair_aligned(a) || !pair_aligned(b) || !pair_aligned(x) || g.nx % 2 || g.ny % 2)
    return cudaErrorMisalignedAddress;
  if (!cells_fit_int32(g)) return cudaErrorInvalidValue;
  const int gx = (g.nx / 2 + TP - 1) / TP, gy = (g.ny / 2 + TR - 1) / TR;  // one coarse row per thread
  const int nzc = g.nz / 2;
  const int zc = z_chunks((long long)gx * gy, nzc, 4);
  const int kchunk = (nzc + zc - 1) / zc;
  const int gz = (nzc + kchunk - 1) / kchunk;
  k_restrict_pairs<<<dim3((unsigned)gx, (unsigned)gy, (unsigned)gz), dim3(TP, TR), 0, s>>>(g, a, b, x, coarse,
                                                                                          kchunk);
  return cudaGetLastError();
}

cudaError_t launch_prolong_pairs(const Grid3& g, const float* e, float* x, int mode, cudaStream_t s) {
  if (!pair_aligned(x) || g.nx % 2) return cudaErrorMisalignedAddress;
  if (!cells_fit_int32(g)) return cudaErrorInvalidValue;
  const int gx = (g.nx / 2 + TP - 1) / TP, gy = (g.ny + TR - 1) / TR;
  const int nzc = g.nz / 2;
  const int zc = z_chunks((long long)gx * gy, nzc, 4);
  const int kchunk = (nzc + zc - 1) / zc;
  const int gz = (nzc + kchunk - 1) / kchunk;
  k_prolong_pairs<<<dim3((unsigned)gx, (unsigned)gy, (unsigned)gz), dim3(TP, TR), 0, s>>>(g, e, x, mode, kchunk);
  return cudaGetLastError();
}

}  // namespace gmg
