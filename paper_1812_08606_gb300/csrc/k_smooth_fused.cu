// One preconditioned Chebyshev step of the smoother (eqs. (smootheq), (e19),
// Sec. 3.2) with the one-sweep red-black SSOR preconditioner, fused into a
// single pass over the grid:
//
//   r = b - A x_in                         (x_in = 0 on the first pre-smoothing step)
//   z = B^{-1} r:  red  z = r / D,  black z = (r + N z)/D,  red z = (r + N z)/D
//   d = c1 d + c2 z   (d = c2 z on the first step),   x_out = x_in + d
//
// The xy-plane is cut into 56 x 18 tiles; a work unit is one z-plane of one
// tile.  The kernel is persistent: one block per resident slot, each taking an
// equal share of the units (whole tile columns in rounds of one tile per
// block, so that neighbouring tiles advance through z together and re-read
// each other's halos from L2, then an even split of the leftover columns into
// z-segments).  A block marches through each of its z-segments; each thread
// owns one adjacent cell pair (always one red and one black cell) of one
// region row.  With plane t just
// committed, the block forms r, 1/D and the red z on plane t-1 over the tile +
// 2 halo, the black z on plane t-2 over the tile + 1 halo, and the final red z
// plus the update on plane t-3 over the tile.  Along z every value a thread
// needs for its own pair (a, x_in, r, 1/D, red and black z of the neighbouring
// planes) stays in its registers; shared memory holds only what x/y neighbours
// read, and the three stages write slots that nobody reads in the same plane
// iteration, so one barrier per plane suffices.  The halos are recomputed by
// neighbouring blocks instead of exchanged, so blocks never wait on one
// another; x_out is a different buffer from x_in, so no block reads a value
// another block has already updated.  d is updated in place (each cell reads
// only its own d).  Global traffic per cell: x_in, a, b, d read, x_out and d
// written (6 words), plus the halo re-reads, which mostly hit L2.
//
// Away from the ends of a segment and from the plates a plane step needs no
// range checks; those steady steps run two planes at a time.  A warp is one
// region row and the two planes have opposite parity, so the lane holding the
// cell each stage updates is fixed per warp and per plane of the pair: a
// warp-uniform branch picks a copy of the step with that lane known at
// compile time, which removes the lane selects from the stages.
#include <algorithm>
#include <mutex>
#include <type_traits>

#include "gmg_internal.cuh"

namespace gmg {

namespace {

// Block = 32 x 24 threads; thread (tx, ty) owns the cell pair (2 tx, 2 tx + 1)
// of region row ty.  Region: 32 pairs (64 cells) x 24 rows = tile 56 x 18 plus
// a 4-cell halo in x (keeps pairs 8-byte aligned in global memory) and a
// 3-cell halo in y.  Values along z stay in each thread's registers; shared
// memory holds only what x/y neighbours read: a (4 planes), x (2), the red z
// of the residual stage (2) and the black z (2).
constexpr int RP = 32, RW = 2 * RP, HX = 4, HY = 3, FTX = RW - 2 * HX, FTY = 18, RH = FTY + 2 * HY;
constexpr int PPL = RP * RH;  // pairs per region plane = threads per block
constexpr int NAS = 4, NXS = 2, NZS = 2;
constexpr size_t FUSED_SMEM = (size_t)(NAS + NXS) * PPL * sizeof(float2) + (size_t)(2 * NZS) * PPL * sizeof(float);
// The face-form variant also keeps NAS planes of the y-face entries (the cell
// form's a planes hold the x-face entries there).
constexpr size_t FUSED_SMEM_FACE = FUSED_SMEM + (size_t)NAS * PPL * sizeof(float2);

struct FusedArgs {
  Grid3 g;
  const float* a;   // cell form (FACE = false)
  Faces<float> f;   // face form (FACE = true)
  const float* b;
  const float* xin;  // null: x_in = 0
  float* xout;
  float* d;
  float c1, c2;
  float ce;         // the eigen-estimate basis step: coefficient of x_in in x_out
  int flags;
  int tiles_x;      // tiles along x
  long long units;  // tiles x nz (one unit = one z-plane of one tile)
};

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sc2(float s) { return make_float2(s, s); }
__device__ __forceinline__ float lane(float2 v, int i) { return i ? v.y : v.x; }

// Bring a line into L2 ahead of its load (no register, no wait).
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Kind of step, fixed at compile time (each kind is its own kernel, so the
// step carries no runtime tests for it): the first step of a smoothing (d =
// c2 z, d not read), with x_in = 0 (pre-smoothing from zero: x_in not read),
// the last step (d is dead afterwards: not written), and the eigen-estimate
// basis step (b = 0 is not read, d is read unless M_FIRST but never written,
// and x_out = ce x_in + c1 d + c2 z with z = -B^{-1} A x_in).
enum StepMode : int { M_FIRST = 1, M_XZERO = 2, M_LAST = 4, M_EIG = 8 };

// Planes [k0, k1) of tile (bx, by).  Leaves shared memory in use: the caller
// synchronises before the next segment.
//
// FACE: the level's operator is given by face entries (the coarse levels of
// the series-parallel coarsening).  The shared planes of a then hold the
// pairs' x-face entries (left face of each cell), a second set of planes the
// y-face entries (face below each cell), and the register window of a holds
// the z-face entries (face below each cell; the plane above the top one is the
// top plate's entries).  Entries beyond the domain load as zero and a plate's
// neighbour value is zero, so the plate and wall cases need no branches.
//
// INNER: the tile's region (tile + halo) lies inside the domain in x and y
// (inner_tile), so every cell of the region exists and no x or y face of it
// is a wall: the range tests and the wall masks are left out.
template <bool FACE, int MODE, bool INNER>
__device__ __forceinline__ void fused_segment(const FusedArgs& P, float2* smf2, const int bx, const int by,
                                              const int k0, const int k1) {
  float2* const As = smf2;               // NAS planes of a (FACE: x-face entries)
  float2* const Ys = As + NAS * PPL;     // FACE: NAS planes of y-face entries
  float2* const Xs = FACE ? Ys + NAS * PPL : As + NAS * PPL;  // NXS planes of x_in
  float* const Z1s = reinterpret_cast<float*>(Xs + NXS * PPL);  // red z of the residual stage
  float* const ZBs = Z1s + NZS * PPL;                              // black z
  const Grid3& g = P.g;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const size_t pl = g.plane();
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int me = ty * RP + tx;
  const int gx0 = bx * FTX - HX + 2 * tx;
  const int gy = by * FTY - HY + ty;
  constexpr bool xzero = (MODE & M_XZERO) != 0;
  constexpr bool first = (MODE & M_FIRST) != 0;
  constexpr bool eig = (MODE & M_EIG) != 0;
  constexpr bool keep_d = (MODE & M_LAST) == 0 && !eig;
  const bool in = INNER || (gx0 >= 0 && gx0 < nx && gy >= 0 && gy < ny);  // nx even: both cells or neither
  const bool rst = in && tx >= 1 && tx <= RP - 2 && ty >= 1 && ty <= RH - 2;            // residual: tile + 2
  const bool bst = in && ty >= 2 && ty <= RH - 3;                                        // black: tile + 1
  const bool fst = in && tx >= HX / 2 && tx < RP - HX / 2 && ty >= HY && ty < RH - HY;  // final: tile
  // the black stage covers the tile + 1 halo: cells of region columns HX - 1 .. RW - HX
  const bool bcol0 = 2 * tx >= HX - 1 && 2 * tx <= RW - HX, bcol1 = 2 * tx + 1 >= HX - 1 && 2 * tx + 1 <= RW - HX;
  const float mxl = gx0 > 0 ? 1.f : 0.f;       // face left of the first cell
  const float mxr = gx0 + 2 < nx ? 1.f : 0.f;  // face right of the second cell
  const float my0 = gy > 0 ? 1.f : 0.f, my1 = gy < ny - 1 ? 1.f : 0.f;
  // a face value times its wall mask (1 on every face of an inner tile)
  auto wall = [](float v, float m) { return INNER ? v : v * m; };
  auto wall2 = [](float2 v, float2 m) { return INNER ? v : mul2(v, m); };
  const float2 fx2 = sc2(g.fx), fy2 = sc2(g.fy), fz2 = sc2(g.fz), fp2 = sc2(g.fp);
  const float2 zero2 = make_float2(0.f, 0.f);
  const int rlo = max(0, k0 - 2), rhi = min(nz, k1 + 2);
  const int blo = max(0, k0 - 1), bhi = min(nz, k1 + 1);
  // pair offsets in 32 bits (fused_smoother_eligible keeps (nz + 4) planes of pairs below 2^31)
  const int qo = in ? (gy * nx + gx0) >> 1 : 0;  // pair offset in a plane
  const float2* A2 = reinterpret_cast<const float2*>(FACE ? P.f.kz : P.a);  // FACE: z-face entries
  const float2* KX2 = reinterpret_cast<const float2*>(P.f.kx);
  const float2* KY2 = reinterpret_cast<const float2*>(P.f.ky);
  const float2* KT2 = reinterpret_cast<const float2*>(P.f.ktop);
  const float2* X2 = reinterpret_cast<const float2*>(P.xin);
  const float2* B2 = reinterpret_cast<const float2*>(P.b);
  const float2* D2 = reinterpret_cast<const float2*>(P.d);
  const int pl2 = (int)(pl >> 1);

  for (int s = 0; s < NZS; ++s) Z1s[s * PPL + me] = ZBs[s * PPL + me] = 0.f;

  // register windows along z (plane t = current iteration)
  float2 aw0 = zero2, aw1 = zero2, aw2 = zero2, aw3 = zero2, aw4 = zero2;  // a: t-4 .. t
  float2 xw0 = zero2, xw1 = zero2, xw2 = zero2, xw3 = zero2;              // x_in: t-3 .. t
  float2 rw0 = zero2, rw1 = zero2, rw2 = zero2;                           // r: t-3 .. t-1
  float2 dw0 = zero2, dw1 = zero2, dw2 = zero2;                           // 1/D: t-3 .. t-1
  float z1w0 = 0.f, z1w1 = 0.f, z1w2 = 0.f;                               // red z: t-3 .. t-1
  float zbw0 = 0.f, zbw1 = 0.f, zbw2 = 0.f;                               // black z: t-4 .. t-2
  float2 pa = zero2, px = zero2, pb = zero2, pbn = zero2, pd = zero2, pdn = zero2;
  float2 pkx = zero2, pky = zero2;  // FACE: x- and y-face entries of the next plane
  {
    const int k = k0 - 3;
    if (in && k >= 0 && k < nz) {
      pa = __ldg(A2 + (k * pl2 + qo));
      if (!xzero) px = __ldg(X2 + (k * pl2 + qo));
      if constexpr (FACE) {
        pkx = __ldg(KX2 + (k * pl2 + qo));
        pky = __ldg(KY2 + (k * pl2 + qo));
      }
    } else if (FACE && in && k == nz) {
      pa = __ldg(KT2 + qo);
    }
  }

  // One plane step.  LM = 0 or 1: the lane of the cell each stage updates (the
  // red cell at t-1 and t-3, the black cell at t-2; the same lane for all
  // three) is known at compile time; LM = 2: it is computed.  ST: steady state,
  // every plane index of the step lies inside the segment and off the plates.
  auto body = [&](auto LMT, auto STT, const int t) {
    constexpr int LM = decltype(LMT)::value;
    constexpr bool ST = decltype(STT)::value;
    const int L = LM < 2 ? LM : (((gy + t) & 1) ^ 1);
    // ---- commit plane t (prefetched during the previous step) ----
    aw0 = aw1; aw1 = aw2; aw2 = aw3; aw3 = aw4; aw4 = pa;
    xw0 = xw1; xw1 = xw2; xw2 = xw3; xw3 = px;
    if constexpr (FACE) {
      As[(t & 3) * PPL + me] = pkx;
      Ys[(t & 3) * PPL + me] = pky;
    } else {
      As[(t & 3) * PPL + me] = pa;
    }
    Xs[(t & 1) * PPL + me] = px;
    // ---- prefetch for the next step ----
    pa = px = zero2;
    if constexpr (FACE) pkx = pky = zero2;
    const int ot = t * pl2 + qo;  // pair offset of plane t
    if (in && (ST || (t + 1 >= 0 && t + 1 < nz && t + 1 <= k1 + 2))) {
      pa = __ldg(A2 + (ot + pl2));
      if (!xzero) px = __ldg(X2 + (ot + pl2));
      if constexpr (FACE) {
        pkx = __ldg(KX2 + (ot + pl2));
        pky = __ldg(KY2 + (ot + pl2));
      }
    } else if (FACE && !ST && in && t + 1 == nz && t + 1 <= k1 + 2) {
      pa = __ldg(KT2 + qo);  // the top plate's entries, as the z face above plane nz - 1
    }
    if (!eig && rst && (ST || (t >= rlo && t < rhi))) pbn = __ldg(B2 + ot);
    if (fst && !first && (ST || (t - 2 >= k0 && t - 2 < k1))) pdn = __ldg(D2 + (ot - 2 * pl2));
    // From zero (no x_in, r = b) a step has the least work, shorter than the
    // loaded memory latency: bring the plane after next into L2 so that the
    // loads above find their lines there (1.03 -> 0.75 ms at 512^3).  The
    // other kinds hide the latency with their work, and the extra instructions
    // made them 9-13% slower.
    if (xzero && in) {
      if (t + 2 >= 0 && t + 2 < nz) {
        prefetch_l2(A2 + (ot + 2 * pl2));
        if (!xzero) prefetch_l2(X2 + (ot + 2 * pl2));
        if constexpr (FACE) {
          prefetch_l2(KX2 + (ot + 2 * pl2));
          prefetch_l2(KY2 + (ot + 2 * pl2));
        }
      }
      if (!eig && t + 1 >= 0 && t + 1 < nz) prefetch_l2(B2 + (ot + pl2));
      if (!first && t - 1 >= 0 && t - 1 < nz) prefetch_l2(D2 + (ot - pl2));
    }

    // ---- residual stage, plane kr = t - 1: r, 1/D (both cells), red z ----
    const int kr = t - 1;
    {
      float2 r = zero2, di = zero2;
      float z1 = 0.f;
      if (FACE && rst && (ST || (kr >= rlo && kr < rhi))) {
        // face form: D = sum of the six entries; A x with zero beyond the plates
        const float2* xc = Xs + (kr & 1) * PPL;
        const float2 kxo = As[(kr & 3) * PPL + me], kxn = As[(kr & 3) * PPL + me + 1];
        const float2 fxm = kxo, fxp = make_float2(kxo.y, kxn.x);
        const float2 fym = Ys[(kr & 3) * PPL + me], fyp = Ys[(kr & 3) * PPL + me + RP];
        const float2 fzm = aw3, fzp = aw4;  // planes kr and kr + 1
        const float2 D = add2(add2(add2(fxm, fxp), add2(fym, fyp)), add2(fzm, fzp));
        r = pb;
        if (!xzero) {
          const float2 x2 = xw2;  // plane kr
          const float2 xl = xc[me - 1], xr = xc[me + 1];
          const float2 xL = make_float2(xl.y, x2.x), xR = make_float2(x2.y, xr.x);
          float2 ax = mul2(fxm, sub2(x2, xL));
          ax = fma2(fxp, sub2(x2, xR), ax);
          ax = fma2(fym, sub2(x2, xc[me - RP]), ax);
          ax = fma2(fyp, sub2(x2, xc[me + RP]), ax);
          ax = fma2(fzm, sub2(x2, xw1), ax);
          ax = fma2(fzp, sub2(x2, xw3), ax);
          r = sub2(r, ax);
        }
        di = make_float2(__fdividef(1.f, D.x), __fdividef(1.f, D.y));
        z1 = lane(r, L) * lane(di, L);
      } else if (!FACE && rst && (ST || (kr >= rlo && kr < rhi))) {
        const bool zlo = ST || kr > 0, zhi = ST || kr < nz - 1;
        const float2* ac = As + (kr & 3) * PPL;
        const float2* xc = Xs + (kr & 1) * PPL;
        const float2 a2 = aw3;  // plane kr
        const float2 al = ac[me - 1], ar = ac[me + 1];
        const float2 aL = make_float2(al.y, a2.x), aR = make_float2(a2.y, ar.x);
        const float2 fxm = wall2(add2(a2, aL), make_float2(mxl, 1.f));
        const float2 fxp = wall2(add2(a2, aR), make_float2(1.f, mxr));
        const float2 fym = wall2(add2(a2, ac[me - RP]), sc2(my0)), fyp = wall2(add2(a2, ac[me + RP]), sc2(my1));
        const float2 fzm = zlo ? add2(a2, aw2) : zero2, fzp = zhi ? add2(a2, aw4) : zero2;
        float2 D;
        if constexpr (ST) {
          D = fma2(fx2, add2(fxm, fxp), fma2(fy2, add2(fym, fyp), mul2(fz2, add2(fzm, fzp))));
        } else {
          const float2 plate = add2(zlo ? zero2 : a2, zhi ? zero2 : a2);
          D = fma2(fx2, add2(fxm, fxp), fma2(fy2, add2(fym, fyp), fma2(fz2, add2(fzm, fzp), mul2(fp2, plate))));
        }
        r = pb;
        if (!xzero) {
          const float2 x2 = xw2;  // plane kr
          const float2 xl = xc[me - 1], xr = xc[me + 1];
          const float2 xL = make_float2(xl.y, x2.x), xR = make_float2(x2.y, xr.x);
          float2 sx = mul2(fxm, sub2(x2, xL));
          sx = fma2(fxp, sub2(x2, xR), sx);
          float2 sy = mul2(fym, sub2(x2, xc[me - RP]));
          sy = fma2(fyp, sub2(x2, xc[me + RP]), sy);
          float2 sz;
          if constexpr (ST) {
            sz = mul2(fz2, mul2(fzm, sub2(x2, xw1)));
            sz = fma2(fz2, mul2(fzp, sub2(x2, xw3)), sz);
          } else {
            const float2 plate = add2(zlo ? zero2 : a2, zhi ? zero2 : a2);
            sz = mul2(fp2, mul2(plate, x2));
            if (zlo) sz = fma2(fz2, mul2(fzm, sub2(x2, xw1)), sz);
            if (zhi) sz = fma2(fz2, mul2(fzp, sub2(x2, xw3)), sz);
          }
          r = sub2(r, fma2(fx2, sx, fma2(fy2, sy, sz)));
        }
        di = make_float2(__fdividef(1.f, D.x), __fdividef(1.f, D.y));
        z1 = lane(r, L) * lane(di, L);
      }
      rw0 = rw1; rw1 = rw2; rw2 = r;
      dw0 = dw1; dw1 = dw2; dw2 = di;
      z1w0 = z1w1; z1w1 = z1w2; z1w2 = z1;
      Z1s[(kr & 1) * PPL + me] = z1;
    }
    // ---- black stage, plane kb = t - 2: z_B = (r + N z1) / D ----
    const int kb = t - 2;
    {
      float zb = 0.f;
      const bool colok = L ? bcol1 : bcol0;
      if (FACE && bst && colok && (ST || (kb >= blo && kb < bhi))) {
        const float* zc = Z1s + (kb & 1) * PPL;
        const float2 kxo = As[(kb & 3) * PPL + me];
        const float fout = L ? As[(kb & 3) * PPL + me + 1].x : kxo.x;
        float N = kxo.y * z1w1;                          // the face between the pair's cells
        N = fmaf(fout, L ? zc[me + 1] : zc[me - 1], N);
        N = fmaf(lane(Ys[(kb & 3) * PPL + me], L), zc[me - RP], N);
        N = fmaf(lane(Ys[(kb & 3) * PPL + me + RP], L), zc[me + RP], N);
        N = fmaf(lane(aw2, L), z1w0, N);                 // z faces of plane kb (below) and kb + 1 (above)
        N = fmaf(lane(aw3, L), z1w2, N);
        zb = (lane(rw1, L) + N) * lane(dw1, L);
      } else if (!FACE && bst && colok && (ST || (kb >= blo && kb < bhi))) {
        const bool zlo = ST || kb > 0, zhi = ST || kb < nz - 1;
        const float2* ac = As + (kb & 3) * PPL;
        const float* zc = Z1s + (kb & 1) * PPL;
        const float a0 = lane(aw2, L);                  // plane kb
        const float ain = lane(aw2, L ^ 1);             // the red cell of the pair
        const float aout = L ? ac[me + 1].x : ac[me - 1].y;
        const float mout = L ? mxr : mxl;
        float sx = (a0 + ain) * z1w1;                   // z1w1: red z of this pair, plane kb
        sx = fmaf(wall(a0 + aout, mout), L ? zc[me + 1] : zc[me - 1], sx);
        float sy = wall(a0 + lane(ac[me - RP], L), my0) * zc[me - RP];
        sy = fmaf(wall(a0 + lane(ac[me + RP], L), my1), zc[me + RP], sy);
        float sz = 0.f;
        if (zlo) sz = (a0 + lane(aw1, L)) * z1w0;
        if (zhi) sz = fmaf(a0 + lane(aw3, L), z1w2, sz);
        const float N = fmaf(g.fx, sx, fmaf(g.fy, sy, g.fz * sz));
        zb = (lane(rw1, L) + N) * lane(dw1, L);
      }
      zbw0 = zbw1; zbw1 = zbw2; zbw2 = zb;
      ZBs[(kb & 1) * PPL + me] = zb;
    }
    // ---- final stage, plane kf = t - 3: red z and the Chebyshev update ----
    const int kf = t - 3;
    if (fst && (ST || (kf >= k0 && kf < k1))) {
      float N;
      if constexpr (FACE) {
        const float* zc = ZBs + (kf & 1) * PPL;
        const float2 kxo = As[(kf & 3) * PPL + me];
        const float fout = L ? As[(kf & 3) * PPL + me + 1].x : kxo.x;
        N = kxo.y * zbw1;
        N = fmaf(fout, L ? zc[me + 1] : zc[me - 1], N);
        N = fmaf(lane(Ys[(kf & 3) * PPL + me], L), zc[me - RP], N);
        N = fmaf(lane(Ys[(kf & 3) * PPL + me + RP], L), zc[me + RP], N);
        N = fmaf(lane(aw1, L), zbw0, N);               // z faces of plane kf (below) and kf + 1 (above)
        N = fmaf(lane(aw2, L), zbw2, N);
      } else {
        const bool zlo = ST || kf > 0, zhi = ST || kf < nz - 1;
        const float2* ac = As + (kf & 3) * PPL;
        const float* zc = ZBs + (kf & 1) * PPL;
        const float a0 = lane(aw1, L);      // plane kf
        const float ain = lane(aw1, L ^ 1);
        const float aout = L ? ac[me + 1].x : ac[me - 1].y;
        const float mout = L ? mxr : mxl;
        float sx = (a0 + ain) * zbw1;  // zbw1: black z of this pair, plane kf
        sx = fmaf(wall(a0 + aout, mout), L ? zc[me + 1] : zc[me - 1], sx);
        float sy = wall(a0 + lane(ac[me - RP], L), my0) * zc[me - RP];
        sy = fmaf(wall(a0 + lane(ac[me + RP], L), my1), zc[me + RP], sy);
        float sz = 0.f;
        if (zlo) sz = (a0 + lane(aw0, L)) * zbw0;
        if (zhi) sz = fmaf(a0 + lane(aw2, L), zbw2, sz);
        N = fmaf(g.fx, sx, fmaf(g.fy, sy, g.fz * sz));
      }
      const float zr = (lane(rw0, L) + N) * lane(dw0, L);
      const float2 z = L ? make_float2(zbw1, zr) : make_float2(zr, zbw1);
      const float2 c2 = sc2(P.c2);
      const float2 dv = first ? mul2(c2, z) : fma2(sc2(P.c1), pd, mul2(c2, z));
      const int q = kf * pl2 + qo;
      if constexpr (keep_d) reinterpret_cast<float2*>(P.d)[q] = dv;
      if constexpr (eig)
        reinterpret_cast<float2*>(P.xout)[q] = fma2(sc2(P.ce), xw0, dv);
      else
        reinterpret_cast<float2*>(P.xout)[q] = xzero ? dv : add2(xw0, dv);
    }
    pb = pbn;
    pd = pdn;
  };

  // One barrier per plane, at a block-uniform point before each step.  Every
  // shared slot a step writes (a and x of plane t, red z of t-1, black z of
  // t-2) is read by no one in the same step, and every slot it reads was
  // written before the barrier.  Steady steps run in pairs (t even, t + 1);
  // within a warp (one region row) the lane parity of the pair is fixed.
  using I0 = std::integral_constant<int, 0>;
  using I1 = std::integral_constant<int, 1>;
  using IR = std::integral_constant<int, 2>;
  using TS = std::integral_constant<bool, true>;
  using TG = std::integral_constant<bool, false>;
  const int tend = k1 + 2;
  const int s0 = max(k0 + 3, 4), s1 = min(k1, nz - 2);  // steady steps
  const bool godd = (gy & 1) != 0;
  int t = k0 - 3;
  while (t <= tend) {
    if (!(t & 1) && t >= s0 && t + 1 <= s1) {
      // t even: the lane is 1 - parity of gy at t, the parity of gy at t + 1
      __syncthreads();
      if (godd) body(I0{}, TS{}, t); else body(I1{}, TS{}, t);
      __syncthreads();
      if (godd) body(I1{}, TS{}, t + 1); else body(I0{}, TS{}, t + 1);
      t += 2;
    } else {
      __syncthreads();
      body(IR{}, TG{}, t);
      ++t;
    }
  }
}

// Tile (bx, by)'s region, x from bx FTX - HX to bx FTX - HX + RW - 1 and y
// from by FTY - HY to by FTY - HY + RH - 1, lies inside the domain with no
// cell of it on a wall: the first cell is past x = 0 and y = 0 and one cell
// beyond the last is still inside.
__device__ __forceinline__ bool inner_tile(const Grid3& g, int bx, int by) {
  return bx >= 1 && by >= 1 && bx * FTX - HX + RW < g.nx && by * FTY - HY + RH < g.ny;
}

template <bool FACE, int MODE>
__global__ void __launch_bounds__(PPL, 1) k_cheb_sgs_fused(const FusedArgs P) {
  extern __shared__ float2 smf2[];
  const int nz = P.g.nz;
  const long long G = gridDim.x, b = blockIdx.x;
  // whole columns first: tile r G + b in round r < full; then the leftover
  // columns: an equal contiguous share of their (tile, plane) units
  const long long full = P.units / nz / G;
  const long long base = full * G * nz, rest = P.units - base;
  long long u = base + rest * b / G;
  const long long end = base + rest * (b + 1) / G;
  long long r = 0;
  for (;;) {
    int tile, k0, k1;
    if (r < full) {
      tile = (int)(r * G + b);
      k0 = 0;
      k1 = nz;
      ++r;
    } else if (u < end) {
      tile = (int)(u / nz);
      k0 = (int)(u - (long long)tile * nz);
      k1 = (int)min((long long)nz, k0 + (end - u));
      u += k1 - k0;
    } else {
      break;
    }
    const int bx = tile % P.tiles_x, by = tile / P.tiles_x;
    // (the face form has no wall masks: it keeps one form of the segment)
    if (!FACE && inner_tile(P.g, bx, by))
      fused_segment<FACE, MODE, !FACE>(P, smf2, bx, by, k0, k1);
    else
      fused_segment<FACE, MODE, false>(P, smf2, bx, by, k0, k1);
    __syncthreads();
  }
}

// Per device: the kernel's shared-memory attribute is set and its resident
// block count known (0 = not yet).  Guarded by a mutex for host threads.
constexpr int kMaxDevices = 64;
int g_fused_slots[2][kMaxDevices] = {};
std::mutex g_fused_mutex;

// The step kinds the library launches: pre-smoothing from zero (first, x_in =
// 0; also as a one-step smoothing), middle, last, and the eigen-estimate basis
// step without and with d.  The first step with x_in runs as a middle step (or
// a last one) with c1 = 0: fma(0, d, c2 z) = c2 z exactly for finite d, and the
// library keeps d finite (zeroed when allocated, written only by smoothing
// steps).  Compiled as its own kind it ran 38% slower than a middle step that
// moves more bytes (1.42 against 1.04 ms at 512^3, on any data), stalled on
// global loads (4.1 cycles per instruction against 0.5).
constexpr int kModes[] = {M_FIRST | M_XZERO, M_FIRST | M_XZERO | M_LAST, 0, M_LAST, M_FIRST | M_EIG, M_EIG};

template <bool FACE, int MODE>
cudaError_t set_smem() {
  return cudaFuncSetAttribute(k_cheb_sgs_fused<FACE, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(FACE ? FUSED_SMEM_FACE : FUSED_SMEM));
}

// Per device and form: the shared-memory attribute of every step kind is set
// and the resident block count known (0 = not yet).
template <bool FACE>
cudaError_t fused_slots(int* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  const size_t smem = FACE ? FUSED_SMEM_FACE : FUSED_SMEM;
  std::lock_guard<std::mutex> lock(g_fused_mutex);
  int& slots = g_fused_slots[FACE ? 1 : 0][dev];
  if (slots == 0) {
    const cudaError_t es[] = {set_smem<FACE, kModes[0]>(), set_smem<FACE, kModes[1]>(), set_smem<FACE, kModes[2]>(),
                              set_smem<FACE, kModes[3]>(), set_smem<FACE, kModes[4]>(), set_smem<FACE, kModes[5]>()};
    for (cudaError_t q : es)
      if (q != cudaSuccess) return q;
    int sms = 0, per = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cheb_sgs_fused<FACE, 0>, PPL, smem);
    if (e != cudaSuccess) return e;
    slots = std::max(1, sms * std::max(1, per));
  }
  *out = slots;
  return cudaSuccess;
}

template <bool FACE>
cudaError_t launch_fused(const FusedArgs& P0, long long units, cudaStream_t s) {
  int slots = 0;
  const cudaError_t e = fused_slots<FACE>(&slots);
  if (e != cudaSuccess) return e;
  // one block per resident slot, but at least 4 planes per block on small grids
  const long long blocks = std::max(1LL, std::min((long long)slots, units / 4));
  const dim3 grid((unsigned)blocks), block(RP, RH);
  const size_t smem = FACE ? FUSED_SMEM_FACE : FUSED_SMEM;
  FusedArgs P = P0;
  const bool eig = (P.flags & CHEB_EIG) != 0;
  int mode = ((P.flags & CHEB_FIRST) ? M_FIRST : 0) | (P.xin ? 0 : M_XZERO) |
             ((P.flags & CHEB_LAST) && !eig ? M_LAST : 0) | (eig ? M_EIG : 0);
  if ((mode & (M_FIRST | M_XZERO | M_EIG)) == M_FIRST) {  // the first step with x_in: see kModes
    mode &= ~M_FIRST;
    P.c1 = 0.f;
  }
  switch (mode) {
    case M_FIRST | M_XZERO: k_cheb_sgs_fused<FACE, M_FIRST | M_XZERO><<<grid, block, smem, s>>>(P); break;
    case M_FIRST | M_XZERO | M_LAST: k_cheb_sgs_fused<FACE, M_FIRST | M_XZERO | M_LAST><<<grid, block, smem, s>>>(P); break;
    case 0: k_cheb_sgs_fused<FACE, 0><<<grid, block, smem, s>>>(P); break;
    case M_LAST: k_cheb_sgs_fused<FACE, M_LAST><<<grid, block, smem, s>>>(P); break;
    case M_FIRST | M_EIG: k_cheb_sgs_fused<FACE, M_FIRST | M_EIG><<<grid, block, smem, s>>>(P); break;
    case M_EIG: k_cheb_sgs_fused<FACE, M_EIG><<<grid, block, smem, s>>>(P); break;
    default: return cudaErrorInvalidValue;  // x_in = 0 needs the first step; the basis step needs x_in
  }
  return cudaGetLastError();
}

}  // namespace

bool fused_smoother_eligible(const Grid3& g) {
  return g.nx >= 32 && g.nx % 2 == 0 && g.ny >= 16 && g.nz >= 8 &&
         (size_t)(g.nz + 4) * (g.plane() / 2) < ((size_t)1 << 31);  // 32-bit pair offsets
}

cudaError_t launch_cheb_sgs_fused(const Grid3& g, const float* a, const float* b, const float* xin, float* xout,
                                    float* d, double c1, double c2, double ce, int flags, int* tma_status,
                                    cudaStream_t s) {
  if (tma_status && tma_smoother_eligible(g, a, b, xin, xout, d, flags)) {
    // cudaErrorNotSupported: no tensor map could be made and nothing was
    // launched; the step runs on this kernel (the same arithmetic)
    const cudaError_t e = launch_cheb_sgs_tma(g, a, b, xin, xout, d, c1, c2, flags, tma_status, s);
    if (e != cudaErrorNotSupported) return e;
  }
  if (!pair_aligned(a) || !pair_aligned(b) || (xin && !pair_aligned(xin)) || !pair_aligned(xout) || !pair_aligned(d))
    return cudaErrorMisalignedAddress;
  const int tx = (g.nx + FTX - 1) / FTX, ty = (g.ny + FTY - 1) / FTY;
  const long long units = (long long)tx * ty * g.nz;
  FusedArgs P{g, a, Faces<float>{}, b, xin, xout, d, (float)c1, (float)c2, (float)ce, flags, tx, units};
  return launch_fused<false>(P, units, s);
}

cudaError_t launch_cheb_sgs_fused_faces(const Grid3& g, const Faces<float>& F, const float* b, const float* xin,
                                        float* xout, float* d, double c1, double c2, double ce, int flags,
                                        cudaStream_t s) {
  if (!pair_aligned(F.kx) || !pair_aligned(F.ky) || !pair_aligned(F.kz) || !pair_aligned(F.ktop) ||
      !pair_aligned(b) || (xin && !pair_aligned(xin)) || !pair_aligned(xout) || !pair_aligned(d))
    return cudaErrorMisalignedAddress;
  const int tx = (g.nx + FTX - 1) / FTX, ty = (g.ny + FTY - 1) / FTY;
  const long long units = (long long)tx * ty * g.nz;
  FusedArgs P{g, nullptr, F, b, xin, xout, d, (float)c1, (float)c2, (float)ce, flags, tx, units};
  return launch_fused<true>(P, units, s);
}

}  // namespace gmg
