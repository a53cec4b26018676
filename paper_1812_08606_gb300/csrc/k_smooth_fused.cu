// One preconditioned Chebyshev step of the smoother (eqs. (smootheq), (e19),
// Sec. 3.2) with the one-sweep red-black SSOR preconditioner, fused into a
// single pass over the grid:
//
//   r = b - A x_in                         (x_in = 0 on the first pre-smoothing step)
//   z = B^{-1} r:  red  z = r / D,  black z = (r + N z)/D,  red z = (r + N z)/D
//   d = c1 d + c2 z   (d = c2 z on the first step),   x_out = x_in + d
//
// Each thread block owns a 56 x 16 tile of the xy-plane and marches through a
// range of z-planes.  Shared-memory rings hold the last planes of x_in and a
// on the tile plus a 3-cell halo, and of r and z on the tile plus a 2-cell
// halo.  With plane kk just loaded, the block forms r (and the red z) on plane
// kk-1 over the tile + 2 halo, the black z on plane kk-2 over the tile + 1
// halo, and the final red z and the update on plane kk-3 over the tile.  The
// halos are recomputed by neighbouring blocks instead of exchanged, so blocks
// never wait on one another; x_out is a different buffer from x_in, so no
// block reads a value another block has already updated.  d is updated in
// place (each cell reads only its own d).  Global traffic per cell: x_in, a, b,
// d read, x_out and d written (6 words), plus the halo re-reads, which mostly
// hit L2.
#include <algorithm>

#include "gmg_internal.cuh"

namespace gmg {

namespace {

// Block = 32 x 8 threads; thread (tx, ty) owns the cell pair (2 tx, 2 tx + 1)
// of region rows ty, ty + 8, ..., so every thread holds one red and one black cell and the
// residual stage runs in packed FP32x2 arithmetic with 64-bit shared and global
// accesses.  Region: 64 cells (32 pairs) x 22 rows = tile 56 x 16 plus a
// 4-cell halo in x (which keeps the pairs 8-byte aligned in global memory) and
// a 3-cell halo in y.
constexpr int RP = 32, RW = 2 * RP, HX = 4, HY = 3, FTX = RW - 2 * HX, FTY = 16, RH = FTY + 2 * HY;
constexpr int PSZ = RP * RH;                       // pairs per plane of the region
constexpr int NXR = 4, NAR = 5, NRR = 3, NZR = 4, NDR = 3;  // ring depths (planes)
constexpr int BDX = RP, BDY = 8, FTHREADS = BDX * BDY;
// rows per thread of each stage (region rows handled: BDY apart)
constexpr int NLROW = (RH + BDY - 1) / BDY;          // loads, rows 0..21
constexpr int NRROW = (RH - 2 + BDY - 1) / BDY;      // residual, rows 1..20
constexpr int NBROW = (RH - 4 + BDY - 1) / BDY;      // black, rows 2..19
constexpr int NFROW = FTY / BDY;                     // final, rows 3..18
constexpr size_t FUSED_SMEM = (size_t)(NXR + NAR + NRR + NZR + NDR) * PSZ * sizeof(float2);

struct FusedArgs {
  Grid3 g;
  const float* a;
  const float* b;
  const float* xin;  // null: x_in = 0
  float* xout;
  float* d;
  float c1, c2;
  int flags;
  int kchunk;
};

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sc2(float s) { return make_float2(s, s); }
__device__ __forceinline__ float lane(float2 v, int i) { return i ? v.y : v.x; }

// Neighbour sum N = sum_f (a_f/h^2) v_q of one cell (lane li of pair l) from
// pair-packed planes: a (am/ac/ap) and v (vm/vc/vp).  mxl/mxr/mym/myp: face
// masks (0 at a side wall); zlo/zhi: the plane below/above exists.
__device__ __forceinline__ float nsum1(const Grid3& g, const float2* am, const float2* ac, const float2* ap,
                                       const float2* vm, const float2* vc, const float2* vp, int l, int li,
                                       float mxl, float mxr, float mym, float myp, bool zlo, bool zhi) {
  const float2 a2 = ac[l], v2 = vc[l];
  const float a0 = lane(a2, li);
  float al, ar, vl, vr;
  if (li == 0) {
    al = ac[l - 1].y; vl = vc[l - 1].y; ar = a2.y; vr = v2.y;
  } else {
    al = a2.x; vl = v2.x; ar = ac[l + 1].x; vr = vc[l + 1].x;
  }
  float sx = (a0 + al) * mxl * vl;
  sx = fmaf((a0 + ar) * mxr, vr, sx);
  float sy = (a0 + lane(ac[l - RP], li)) * mym * lane(vc[l - RP], li);
  sy = fmaf((a0 + lane(ac[l + RP], li)) * myp, lane(vc[l + RP], li), sy);
  float sz = 0.f;
  if (zlo) sz = (a0 + lane(am[l], li)) * lane(vm[l], li);
  if (zhi) sz = fmaf(a0 + lane(ap[l], li), lane(vp[l], li), sz);
  return fmaf(g.fx, sx, fmaf(g.fy, sy, g.fz * sz));
}

// Rows of a stage handled by one thread: region rows r0 + ty + BDY * m.
template <int NROW>
struct RowSet {
  int l[NROW];      // pair index of the thread's pair in the row (-1: row unused)
  int go[NROW];     // global offset (in cells) of the pair's first cell, plane excluded
  float my0[NROW];  // 1 if the cell has a face to row - 1
  float my1[NROW];  // 1 if the cell has a face to row + 1
  int gy[NROW];
};

template <int NROW>
__device__ __forceinline__ void make_rows(RowSet<NROW>& R, int r0, int rmax, int ty, int tx, int y0, int ny, int nx,
                                          int gx0, bool colok) {
#pragma unroll
  for (int m = 0; m < NROW; ++m) {
    const int ry = r0 + ty + BDY * m, gy = y0 + ry;
    const bool ok = ry <= rmax && colok && gy >= 0 && gy < ny;
    R.l[m] = ok ? ry * RP + tx : -1;
    R.go[m] = gy * nx + gx0;
    R.my0[m] = gy > 0 ? 1.f : 0.f;
    R.my1[m] = gy < ny - 1 ? 1.f : 0.f;
    R.gy[m] = gy;
  }
}

__global__ void __launch_bounds__(FTHREADS, 2) k_cheb_sgs_fused(const FusedArgs P) {
  extern __shared__ float2 sm2[];
  float2* const xs = sm2;
  float2* const as = xs + NXR * PSZ;
  float2* const rs = as + NAR * PSZ;
  float2* const zs = rs + NRR * PSZ;
  float2* const ds = zs + NZR * PSZ;  // 1/D
  const Grid3& g = P.g;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const size_t pl = g.plane();
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int gx0 = blockIdx.x * FTX - HX + 2 * tx;  // first cell of this thread's pair
  const int y0 = blockIdx.y * FTY - HY;            // region row 0
  const int k0 = blockIdx.z * P.kchunk;
  const int k1 = min(nz, k0 + P.kchunk);
  const bool xzero = P.xin == nullptr;
  const bool first = (P.flags & CHEB_FIRST) != 0;
  const bool colin = gx0 >= 0 && gx0 < nx;  // nx even: both cells or neither
  const float2 mxm = make_float2(gx0 > 0 ? 1.f : 0.f, 1.f);       // left faces of the two cells
  const float2 mxp = make_float2(1.f, gx0 + 2 < nx ? 1.f : 0.f);  // right faces
  const int rlo = max(0, k0 - 2), rhi = min(nz, k1 + 2);
  const int blo = max(0, k0 - 1), bhi = min(nz, k1 + 1);
  const float2 fx2 = sc2(g.fx), fy2 = sc2(g.fy), fz2 = sc2(g.fz), fp2 = sc2(g.fp);
  const float2 zero2 = make_float2(0.f, 0.f);

  // r, z and 1/D rings start at zero: cells outside the domain stay zero
  for (int t = ty * BDX + tx; t < (NRR + NZR + NDR) * PSZ; t += FTHREADS) rs[t] = zero2;

  RowSet<NLROW> LD;  // plane loads: rows 0..21
  make_rows(LD, 0, RH - 1, ty, tx, y0, ny, nx, gx0, colin);
  RowSet<NRROW> RR;  // residual: rows 1..20, pairs 1..30
  make_rows(RR, 1, RH - 2, ty, tx, y0, ny, nx, gx0, colin && tx >= 1 && tx <= RP - 2);
  RowSet<NBROW> BR;  // black: rows 2..19, pairs 1..30
  make_rows(BR, 2, RH - 3, ty, tx, y0, ny, nx, gx0, colin && tx >= 1 && tx <= RP - 2);
  RowSet<NFROW> FR;  // final: rows 3..18, pairs 2..29
  make_rows(FR, HY, HY + FTY - 1, ty, tx, y0, ny, nx, gx0, colin && tx >= HX / 2 && tx < RP - HX / 2);
  // rows of the residual stage outside the domain (inside the region) get zeros
  bool rzero[NRROW];
#pragma unroll
  for (int m = 0; m < NRROW; ++m) rzero[m] = RR.l[m] < 0 && 1 + ty + BDY * m <= RH - 2 && tx >= 1 && tx <= RP - 2;

  float2 pa[NLROW], px[NLROW], pb[NRROW], pbn[NRROW], pd[NFROW], pdn[NFROW];
#pragma unroll
  for (int m = 0; m < NLROW; ++m) pa[m] = px[m] = zero2;
#pragma unroll
  for (int m = 0; m < NRROW; ++m) pb[m] = pbn[m] = zero2;
#pragma unroll
  for (int m = 0; m < NFROW; ++m) pd[m] = pdn[m] = zero2;
  auto prefetch_ax = [&](int k) {
#pragma unroll
    for (int m = 0; m < NLROW; ++m) {
      pa[m] = px[m] = zero2;
      if (k >= 0 && k < nz && LD.l[m] >= 0) {
        const size_t q = ((size_t)k * pl + LD.go[m]) >> 1;
        pa[m] = __ldg(reinterpret_cast<const float2*>(P.a) + q);
        if (!xzero) px[m] = __ldg(reinterpret_cast<const float2*>(P.xin) + q);
      }
    }
  };
  prefetch_ax(k0 - 3);

  // ring slot offsets; a ring (depth 5): slot of planes kk-4 .. kk
  int sa[5];
  {
    int base = k0 - 3;
#pragma unroll
    for (int j = 0; j < 5; ++j) sa[j] = (((base - 4 + j) % NAR + NAR) % NAR) * PSZ;
  }
  int sr[3], sd[3];  // r / 1-over-D rings (depth 3): planes kk-3 .. kk-1
#pragma unroll
  for (int j = 0; j < 3; ++j) sr[j] = sd[j] = ((((k0 - 3) - 3 + j) % 3 + 3) % 3) * PSZ;

  for (int kk = k0 - 3; kk <= k1 + 2; ++kk) {
    // slots: a(kk - 4 + j) at sa[j], r(kk - 3 + j) at sr[j], x/z(k) at (k & 3) * PSZ
    if (kk >= 0 && kk < nz) {
      float2* xd = xs + (kk & 3) * PSZ;
      float2* ad = as + sa[4];
#pragma unroll
      for (int m = 0; m < NLROW; ++m) {
        const int ry = ty + BDY * m;
        if (ry < RH) {
          ad[ry * RP + tx] = pa[m];
          xd[ry * RP + tx] = px[m];
        }
      }
    }
    __syncthreads();
    if (kk + 1 <= k1 + 2) prefetch_ax(kk + 1);
    if (kk >= rlo && kk < rhi) {
      const float2* b = reinterpret_cast<const float2*>(P.b) + (((size_t)kk * pl) >> 1);
#pragma unroll
      for (int m = 0; m < NRROW; ++m)
        if (RR.l[m] >= 0) pbn[m] = __ldg(b + (RR.go[m] >> 1));
    }
    if (!first && kk - 2 >= k0 && kk - 2 < k1) {
      const float2* d = reinterpret_cast<const float2*>(P.d) + (((size_t)(kk - 2) * pl) >> 1);
#pragma unroll
      for (int m = 0; m < NFROW; ++m)
        if (FR.l[m] >= 0) pdn[m] = __ldg(d + (FR.go[m] >> 1));
    }

    // ---- r, 1/D (both cells) and the red z on plane kr = kk - 1 ----
    const int kr = kk - 1;
    if (kr >= rlo && kr < rhi) {
      const bool zlo = kr > 0, zhi = kr < nz - 1;
      const float2* ac = as + sa[3];
      const float2* am = as + sa[2];
      const float2* ap = as + sa[4];
      const float2* xc = xs + (kr & 3) * PSZ;
      const float2* xm = xs + ((kr - 1) & 3) * PSZ;
      const float2* xp = xs + ((kr + 1) & 3) * PSZ;
      float2* rd = rs + sr[2];
      float2* zd = zs + (kr & 3) * PSZ;
      float2* dd = ds + sd[2];
#pragma unroll
      for (int m = 0; m < NRROW; ++m) {
        const int l = RR.l[m];
        if (l < 0) {
          if (rzero[m]) {
            const int lz = (1 + ty + BDY * m) * RP + tx;
            rd[lz] = zero2;
            zd[lz] = zero2;
            dd[lz] = zero2;
          }
          continue;
        }
        const float2 my0 = sc2(RR.my0[m]), my1 = sc2(RR.my1[m]);
        const float2 a2 = ac[l], al = ac[l - 1], ar = ac[l + 1];
        const float2 aL = make_float2(al.y, a2.x), aR = make_float2(a2.y, ar.x);
        const float2 fxm = mul2(add2(a2, aL), mxm), fxp = mul2(add2(a2, aR), mxp);
        const float2 fym = mul2(add2(a2, ac[l - RP]), my0), fyp = mul2(add2(a2, ac[l + RP]), my1);
        const float2 fzm = zlo ? add2(a2, am[l]) : zero2, fzp = zhi ? add2(a2, ap[l]) : zero2;
        const float2 plate = add2(zlo ? zero2 : a2, zhi ? zero2 : a2);
        const float2 D =
            fma2(fx2, add2(fxm, fxp), fma2(fy2, add2(fym, fyp), fma2(fz2, add2(fzm, fzp), mul2(fp2, plate))));
        float2 r = pb[m];
        if (!xzero) {
          const float2 x2 = xc[l], xl = xc[l - 1], xr = xc[l + 1];
          const float2 xL = make_float2(xl.y, x2.x), xR = make_float2(x2.y, xr.x);
          float2 sx = mul2(fxm, sub2(x2, xL));
          sx = fma2(fxp, sub2(x2, xR), sx);
          float2 sy = mul2(fym, sub2(x2, xc[l - RP]));
          sy = fma2(fyp, sub2(x2, xc[l + RP]), sy);
          float2 sz = mul2(fp2, mul2(plate, x2));
          if (zlo) sz = fma2(fz2, mul2(fzm, sub2(x2, xm[l])), sz);
          if (zhi) sz = fma2(fz2, mul2(fzp, sub2(x2, xp[l])), sz);
          r = sub2(r, fma2(fx2, sx, fma2(fy2, sy, sz)));
        }
        const float2 di = make_float2(__frcp_rn(D.x), __frcp_rn(D.y));
        rd[l] = r;
        dd[l] = di;
        const int red = (gx0 + RR.gy[m] + kr) & 1;  // 0: the first cell is red
        zd[l] = red ? make_float2(0.f, r.y * di.y) : make_float2(r.x * di.x, 0.f);
      }
    }
    __syncthreads();
    // ---- black z on plane kb = kk - 2 (tile + 1 halo) ----
    const int kb = kk - 2;
    if (kb >= blo && kb < bhi) {
      const bool zlo = kb > 0, zhi = kb < nz - 1;
      const float2* ac = as + sa[2];
      const float2* am = as + sa[1];
      const float2* ap = as + sa[3];
      float2* zc = zs + (kb & 3) * PSZ;
      const float2* zm = zs + ((kb - 1) & 3) * PSZ;
      const float2* zp = zs + ((kb + 1) & 3) * PSZ;
      const float2* rc = rs + sr[1];
      const float2* dc = ds + sd[1];
#pragma unroll
      for (int m = 0; m < NBROW; ++m) {
        const int l = BR.l[m];
        if (l < 0) continue;
        const int li = ((gx0 + BR.gy[m] + kb) & 1) ^ 1;  // lane of the black cell
        const int col = 2 * tx + li;
        if (col < HX - 1 || col > RW - HX) continue;     // region columns 3..60
        const float N = nsum1(g, am, ac, ap, zm, zc, zp, l, li, li ? 1.f : mxm.x, li ? mxp.y : 1.f, BR.my0[m],
                              BR.my1[m], zlo, zhi);
        reinterpret_cast<float*>(zc)[2 * l + li] = (lane(rc[l], li) + N) * lane(dc[l], li);
      }
    }
    __syncthreads();
    // ---- final red z and the Chebyshev update on plane kf = kk - 3 (tile) ----
    const int kf = kk - 3;
    if (kf >= k0 && kf < k1) {
      const bool zlo = kf > 0, zhi = kf < nz - 1;
      const float2* ac = as + sa[1];
      const float2* am = as + sa[0];
      const float2* ap = as + sa[2];
      const float2* zc = zs + (kf & 3) * PSZ;
      const float2* zm = zs + ((kf - 1) & 3) * PSZ;
      const float2* zp = zs + ((kf + 1) & 3) * PSZ;
      const float2* rc = rs + sr[0];
      const float2* dc = ds + sd[0];
      const float2* xc = xs + (kf & 3) * PSZ;
      float2* dg = reinterpret_cast<float2*>(P.d) + (((size_t)kf * pl) >> 1);
      float2* xg = reinterpret_cast<float2*>(P.xout) + (((size_t)kf * pl) >> 1);
      const float2 c2 = sc2(P.c2), c1 = sc2(P.c1);
#pragma unroll
      for (int m = 0; m < NFROW; ++m) {
        const int l = FR.l[m];
        if (l < 0) continue;
        const int li = (gx0 + FR.gy[m] + kf) & 1;  // lane of the red cell
        const float N = nsum1(g, am, ac, ap, zm, zc, zp, l, li, li ? 1.f : mxm.x, li ? mxp.y : 1.f, FR.my0[m],
                              FR.my1[m], zlo, zhi);
        const float zr = (lane(rc[l], li) + N) * lane(dc[l], li);
        const float2 zb = zc[l];
        const float2 z = li ? make_float2(zb.x, zr) : make_float2(zr, zb.y);
        const float2 dv = first ? mul2(c2, z) : fma2(c1, pd[m], mul2(c2, z));
        const int q = FR.go[m] >> 1;
        dg[q] = dv;
        xg[q] = xzero ? dv : add2(xc[l], dv);
      }
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < NRROW; ++m) pb[m] = pbn[m];
#pragma unroll
    for (int m = 0; m < NFROW; ++m) pd[m] = pdn[m];
    // rotate the ring slots to the next plane
    const int na = sa[0];
#pragma unroll
    for (int j = 0; j < 4; ++j) sa[j] = sa[j + 1];
    sa[4] = na;
    const int nr = sr[0], nd = sd[0];
    sr[0] = sr[1]; sr[1] = sr[2]; sr[2] = nr;
    sd[0] = sd[1]; sd[1] = sd[2]; sd[2] = nd;
  }
}

bool g_fused_attr_set = false;

}  // namespace

bool fused_smoother_eligible(const Grid3& g) { return g.nx >= 32 && g.nx % 2 == 0 && g.ny >= 16 && g.nz >= 8; }

cudaError_t launch_cheb_sgs_fused(const Grid3& g, const float* a, const float* b, const float* xin, float* xout,
                                  float* d, double c1, double c2, int flags, cudaStream_t s) {
  if (!g_fused_attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_cheb_sgs_fused, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)FUSED_SMEM);
    if (e != cudaSuccess) return e;
    g_fused_attr_set = true;
  }
  const int tx = (g.nx + FTX - 1) / FTX, ty = (g.ny + FTY - 1) / FTY;
  // enough z-chunks for ~8 blocks per SM, each chunk at least 8 planes
  const int target = 152 * 8;
  int nzc = (target + tx * ty - 1) / (tx * ty);
  nzc = std::max(1, std::min(nzc, g.nz / 8));
  const int kchunk = (g.nz + nzc - 1) / nzc;
  nzc = (g.nz + kchunk - 1) / kchunk;
  FusedArgs P{g, a, b, xin, xout, d, (float)c1, (float)c2, flags, kchunk};
  k_cheb_sgs_fused<<<dim3((unsigned)tx, (unsigned)ty, (unsigned)nzc), dim3(BDX, BDY), FUSED_SMEM, s>>>(P);
  return cudaGetLastError();
}

}  // namespace gmg
