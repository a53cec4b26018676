// The fused Chebyshev + red-black SSOR step (eqs. (smootheq), (e19), Sec. 3.2)
// on the cell-coefficient level, with its planes brought into shared memory by
// the Tensor Memory Accelerator:
//
//   r = b - A x_in                         (x_in = 0 on the first pre-smoothing step)
//   z = B^{-1} r:  red  z = r / D,  black z = (r + N z)/D,  red z = (r + N z)/D
//   d = c1 d + c2 z   (d = c2 z on the first step),   x_out = x_in + d
//
// It computes what the step of k_smooth_fused.cu computes, cell by cell in the
// same order of operations, with the same z-pipeline: with plane t committed,
// the residual stage (r, 1/D, red z) runs on plane t - 1 over the tile + 2
// halo, the black stage on plane t - 2 over the tile + 1 halo, the final red z
// and the update on plane t - 3 over the tile.  What differs is how the planes
// arrive:
//
// - One elected thread issues, per plane step, tiled bulk-tensor copies of the
//   region planes of a and x_in (64 x 26 cells: the tile, a 4-cell x halo and
//   3 rows of y halo around the 24 computing rows), of b (64 x 24) and of d
//   (the 56 x 20 tile), PF - 1 plane steps ahead, into rings of shared-memory
//   slots; one transaction-count mbarrier per step's group of copies.  Cells
//   beyond the x/y edges of the domain arrive as zeros.
// - The x/y neighbours read those slots directly, so no thread stores a or x
//   into shared memory and no thread computes a global address for a load.
// - With the halo rows of a and x loaded by the copy engine, every one of the
//   24 thread rows computes: the tile grows from 56 x 18 to 56 x 20 cells on
//   the same 768 threads.
//
// The kernel runs the smoothing steps of the V-cycle (6-10% faster than on
// k_smooth_fused.cu at 512^3).  The eigen estimate's basis steps stay on
// k_smooth_fused.cu: on an earlier form of this kernel they measured 10%
// slower (0.97 against 0.88 ms at 512^3).
//
// Every wait on an mbarrier is bounded (about a second of the global timer);
// a thread whose wait runs out counts it in *status, stops waiting and runs
// to the end of its work on what its shared memory holds (all its accesses
// stay in bounds).  The host reads *status after the set-up and each solve.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <type_traits>

#include "gmg_internal.cuh"

namespace gmg {

namespace {

constexpr int RP = 32;             // cell pairs per region row: one warp
constexpr int RW = 2 * RP;         // 64 region columns
constexpr int HX = 4;              // x halo (keeps every copy's x origin 16-byte aligned)
constexpr int FTX = RW - 2 * HX;   // 56 tile columns
constexpr int TR = 24;             // thread rows: region rows 1 .. 24
constexpr int DR = TR + 2;         // data rows of a and x: region rows 0 .. 25
constexpr int FTY = TR - 4;        // 20 tile rows: region rows 3 .. 22
constexpr int NT = RP * TR;        // 768 threads
constexpr int PF = 3;              // the copies of step c are issued at step c - PF + 1
constexpr int SA = 8, SX = 8, SB = 4, SD = 4;  // ring slots (powers of two: slot = plane & (S - 1))
constexpr int NMB = 4;             // mbarriers: one per step group
// Slots a step's copies overwrite were last read at the step before the one
// that issues them (after its barrier); NMB >= PF for the same reason.
static_assert(SA >= PF + 4 && SX >= PF + 2 && SB >= PF && SD >= PF && NMB >= PF, "ring sizes for PF");
constexpr int NZS = 2;             // shared planes of the red and of the black z
constexpr int A_SLOT = RP * DR;          // float2 per a or x plane (832)
constexpr int B_SLOT = RP * TR;          // float2 per b plane (768)
constexpr int D_SLOT = (FTX / 2) * FTY;  // float2 per d plane (560)
constexpr uint32_t A_BYTES = A_SLOT * 8, B_BYTES = B_SLOT * 8, D_BYTES = D_SLOT * 8;
// shared-memory layout, in bytes from a 128-byte aligned base
constexpr uint32_t OFF_A = 0;
constexpr uint32_t OFF_X = OFF_A + SA * A_BYTES;
constexpr uint32_t OFF_B = OFF_X + SX * A_BYTES;
constexpr uint32_t OFF_D = OFF_B + SB * B_BYTES;
constexpr uint32_t OFF_Z = OFF_D + SD * D_BYTES;
constexpr uint32_t OFF_MB = OFF_Z + 2 * NZS * NT * sizeof(float);
constexpr uint32_t OFF_SEG = OFF_MB + NMB * 8;  // the issuing thread's copy origins of the segment
constexpr size_t TMA_SMEM = OFF_SEG + 16 + 128;  // + room to align the base
static_assert(A_BYTES % 128 == 0 && B_BYTES % 128 == 0 && D_BYTES % 128 == 0, "copy destinations 128-byte aligned");
static_assert(OFF_MB % 8 == 0, "mbarriers 8-byte aligned");
static_assert(TMA_SMEM <= 227 * 1024, "one block per SM");
constexpr unsigned long long kWaitLimitNs = 1000000000ull;

struct TmaArgs {
  CUtensorMap ma, mx, mb, md;  // a and x_in (64 x 26 boxes), b (64 x 24), d (56 x 20)
  Grid3 g;
  float* xout;
  float* d;
  float c1, c2;
  int tiles_x;      // tiles along x
  long long units;  // tiles x nz (one unit = one z-plane of one tile)
  int* status;      // count of waits that ran out
};

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sc2(float s) { return make_float2(s, s); }
__device__ __forceinline__ float lane(float2 v, int i) { return i ? v.y : v.x; }

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
// The elected thread's arrival, announcing the bytes the group's copies bring.
__device__ __forceinline__ void mbar_expect(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __noinline__ bool mbar_wait_slow(uint32_t a, uint32_t parity) {
  const unsigned long long t0 = global_ns();
  while (!mbar_try(a, parity))
    if (global_ns() - t0 > kWaitLimitNs) return false;
  return true;
}
// One tiled copy of a box of a 3-D tensor into shared memory; its bytes
// complete the transaction count of mbarrier mb.
__device__ __forceinline__ void tma_load(uint32_t dst, const CUtensorMap* m, int x, int y, int z, uint32_t mb) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(m)), "r"(x), "r"(y), "r"(z), "r"(mb)
      : "memory");
}

// Kind of step, fixed at compile time (as in k_smooth_fused.cu): the first
// step (d = c2 z, d not read), x_in = 0 (not read), the last step (d not
// written).
enum StepMode : int { M_FIRST = 1, M_XZERO = 2, M_LAST = 4 };

// The pipeline state a block carries across its segments: the parity each
// mbarrier's next phase completes with (bit i for mbarrier i), and whether one
// of this thread's waits has run out.
struct Pipe {
  uint32_t phase = 0;
  bool dead = false;
};

// Planes [k0, k1) of tile (bx, by).  INNER: the region lies inside the domain
// in x and y, so no computing cell is outside it or on a wall.
template <int MODE, bool INNER>
__device__ __forceinline__ void tma_segment(const TmaArgs& P, unsigned char* sm, const uint32_t sbase, Pipe& pipe,
                                            const int bx, const int by, const int k0, const int k1) {
  const float2* const Ar = reinterpret_cast<const float2*>(sm + OFF_A);
  const float2* const Xr = reinterpret_cast<const float2*>(sm + OFF_X);
  const float2* const Br = reinterpret_cast<const float2*>(sm + OFF_B);
  const float2* const Dr = reinterpret_cast<const float2*>(sm + OFF_D);
  float* const Z1s = reinterpret_cast<float*>(sm + OFF_Z);  // red z of the residual stage
  float* const ZBs = Z1s + NZS * NT;                          // black z
  const uint32_t mb0 = sbase + OFF_MB;
  const Grid3& g = P.g;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const size_t pl = g.plane();
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int me = ty * RP + tx;   // this pair in a b plane and in the z planes
  const int ma = me + RP;        // this pair in an a or x plane (region row ty + 1)
  const int gx0 = bx * FTX - HX + 2 * tx;  // region column 0 is x = bx FTX - HX
  const int gy = by * FTY - 3 + 1 + ty;     // region row 0 is y = by FTY - 3
  // The issuing thread keeps the copies' origins in shared memory (volatile:
  // read back at each issue), so no thread holds them in registers through
  // the plane loop.
  volatile int* const seg = reinterpret_cast<volatile int*>(sm + OFF_SEG);
  if (me == 0) {
    seg[0] = bx * FTX - HX;
    seg[1] = by * FTY - 3;
  }
  constexpr bool xzero = (MODE & M_XZERO) != 0;
  constexpr bool first = (MODE & M_FIRST) != 0;
  constexpr bool keep_d = (MODE & M_LAST) == 0;
  const bool in = INNER || (gx0 >= 0 && gx0 < nx && gy >= 0 && gy < ny);  // nx even: both cells or neither
  const bool rst = in && tx >= 1 && tx <= RP - 2;                          // residual: tile + 2
  const bool bst = in && ty >= 1 && ty <= TR - 2;                          // black: tile + 1
  const bool fst = in && tx >= HX / 2 && tx < RP - HX / 2 && ty >= 2 && ty < TR - 2;  // final: tile
  const int mdp = fst ? (ty - 2) * (FTX / 2) + (tx - HX / 2) : 0;                    // this pair in a d plane
  // the black stage covers the tile + 1 halo: cells of region columns HX - 1 .. RW - HX
  const bool bcol0 = 2 * tx >= HX - 1 && 2 * tx <= RW - HX, bcol1 = 2 * tx + 1 >= HX - 1 && 2 * tx + 1 <= RW - HX;
  const float mxl = gx0 > 0 ? 1.f : 0.f;       // face left of the first cell
  const float mxr = gx0 + 2 < nx ? 1.f : 0.f;  // face right of the second cell
  const float my0 = gy > 0 ? 1.f : 0.f, my1 = gy < ny - 1 ? 1.f : 0.f;
  auto wall = [](float v, float m) { return INNER ? v : v * m; };
  auto wall2 = [](float2 v, float2 m) { return INNER ? v : mul2(v, m); };
  const float2 fx2 = sc2(g.fx), fy2 = sc2(g.fy), fz2 = sc2(g.fz), fp2 = sc2(g.fp);
  const float2 zero2 = make_float2(0.f, 0.f);
  const int rlo = max(0, k0 - 2), rhi = min(nz, k1 + 2);
  const int blo = max(0, k0 - 1), bhi = min(nz, k1 + 1);
  // pair offsets in 32 bits for the stores (fused_smoother_eligible keeps (nz + 4) planes of pairs below 2^31)
  const int qo = in ? (gy * nx + gx0) >> 1 : 0;
  const int pl2 = (int)(pl >> 1);
  const int tstart = k0 - 3, tend = k1 + 2;

  // The copies consumed at plane step c: a and x_in of plane c + 1 (this
  // pair's values for the next step, the neighbours' two steps later), b of
  // plane c - 1 (residual stage) and d of plane c - 3 (final stage).  Planes a
  // step never reads are not copied.  Issued by thread 0 only, after the
  // block barrier that retires every read of the slots they overwrite (for
  // the first groups of a segment, the barrier that ends the previous one).
  auto issue = [&](const int c, const bool ax_only) {
    const int x0 = seg[0], y0 = seg[1];
    const uint32_t mb = mb0 + 8u * (uint32_t)(c & (NMB - 1));
    const int pa = c + 1, pb = c - 1, pd = c - 3;
    const bool lax = pa >= 0 && pa < nz && pa <= k1 + 2;
    const bool lb = !ax_only && pb >= rlo && pb < rhi;
    const bool ld = !ax_only && !first && pd >= k0 && pd < k1;
    const uint32_t bytes = (lax ? (xzero ? A_BYTES : 2 * A_BYTES) : 0u) + (lb ? B_BYTES : 0u) + (ld ? D_BYTES : 0u);
    mbar_expect(mb, bytes);
    if (lax) {
      tma_load(sbase + OFF_A + (uint32_t)(pa & (SA - 1)) * A_BYTES, &P.ma, x0, y0, pa, mb);
      if (!xzero) tma_load(sbase + OFF_X + (uint32_t)(pa & (SX - 1)) * A_BYTES, &P.mx, x0, y0, pa, mb);
    }
    if (lb) tma_load(sbase + OFF_B + (uint32_t)(pb & (SB - 1)) * B_BYTES, &P.mb, x0, y0 + 1, pb, mb);
    if (ld) tma_load(sbase + OFF_D + (uint32_t)(pd & (SD - 1)) * D_BYTES, &P.md, x0 + HX, y0 + 3, pd, mb);
  };
  // Every thread waits for the group of step c (each group once, in order).
  auto wait_group = [&](const int c) {
    const int i = c & (NMB - 1);
    const uint32_t mb = mb0 + 8u * (uint32_t)i;
    const uint32_t par = (pipe.phase >> i) & 1u;
    if (!pipe.dead && !mbar_try(mb, par) && !mbar_wait_slow(mb, par)) {
      pipe.dead = true;
      atomicAdd(P.status, 1);
    }
    pipe.phase ^= 1u << i;
  };

  if (me == 0) {
    issue(tstart - 1, true);
    for (int c = tstart; c < tstart + PF - 1; ++c) issue(c, false);  // tend - tstart = k1 - k0 + 5 >= PF
  }
  for (int s = 0; s < NZS; ++s) Z1s[s * NT + me] = ZBs[s * NT + me] = 0.f;

  // register windows along z (plane t = current iteration)
  float2 aw0 = zero2, aw1 = zero2, aw2 = zero2, aw3 = zero2, aw4 = zero2;  // a: t-4 .. t
  float2 xw0 = zero2, xw1 = zero2, xw2 = zero2, xw3 = zero2;              // x_in: t-3 .. t
  float2 rw0 = zero2, rw1 = zero2, rw2 = zero2;                           // r: t-3 .. t-1
  float2 dw0 = zero2, dw1 = zero2, dw2 = zero2;                           // 1/D: t-3 .. t-1
  float z1w0 = 0.f, z1w1 = 0.f, z1w2 = 0.f;                               // red z: t-3 .. t-1
  float zbw0 = 0.f, zbw1 = 0.f, zbw2 = 0.f;                               // black z: t-4 .. t-2
  wait_group(tstart - 1);
  float2 pa = Ar[(tstart & (SA - 1)) * A_SLOT + ma];
  float2 px = xzero ? zero2 : Xr[(tstart & (SX - 1)) * A_SLOT + ma];

  // One plane step; LM and ST as in k_smooth_fused.cu (the lane of the cell
  // each stage updates at compile time or computed; steady: every plane index
  // of the step inside the segment and off the plates).
  auto body = [&](auto LMT, auto STT, const int t) {
    constexpr int LM = decltype(LMT)::value;
    constexpr bool ST = decltype(STT)::value;
    const int L = LM < 2 ? LM : (((gy + t) & 1) ^ 1);
    // ---- commit plane t (read from its slot during the previous step) ----
    aw0 = aw1; aw1 = aw2; aw2 = aw3; aw3 = aw4; aw4 = pa;
    xw0 = xw1; xw1 = xw2; xw2 = xw3; xw3 = px;
    // ---- the copies for step t + PF - 1, then this step's copies ----
    if (me == 0 && t + PF - 1 <= tend) issue(t + PF - 1, false);
    wait_group(t);
    pa = Ar[((t + 1) & (SA - 1)) * A_SLOT + ma];
    if (!xzero) px = Xr[((t + 1) & (SX - 1)) * A_SLOT + ma];

    // ---- residual stage, plane kr = t - 1: r, 1/D (both cells), red z ----
    const int kr = t - 1;
    {
      float2 r = zero2, di = zero2;
      float z1 = 0.f;
      if (rst && (ST || (kr >= rlo && kr < rhi))) {
        const bool zlo = ST || kr > 0, zhi = ST || kr < nz - 1;
        const float2* ac = Ar + (kr & (SA - 1)) * A_SLOT;
        const float2* xc = Xr + (kr & (SX - 1)) * A_SLOT;
        const float2 a2 = aw3;  // plane kr
        const float2 al = ac[ma - 1], ar = ac[ma + 1];
        const float2 aL = make_float2(al.y, a2.x), aR = make_float2(a2.y, ar.x);
        const float2 fxm = wall2(add2(a2, aL), make_float2(mxl, 1.f));
        const float2 fxp = wall2(add2(a2, aR), make_float2(1.f, mxr));
        const float2 fym = wall2(add2(a2, ac[ma - RP]), sc2(my0)), fyp = wall2(add2(a2, ac[ma + RP]), sc2(my1));
        const float2 fzm = zlo ? add2(a2, aw2) : zero2, fzp = zhi ? add2(a2, aw4) : zero2;
        float2 D;
        if constexpr (ST) {
          D = fma2(fx2, add2(fxm, fxp), fma2(fy2, add2(fym, fyp), mul2(fz2, add2(fzm, fzp))));
        } else {
          const float2 plate = add2(zlo ? zero2 : a2, zhi ? zero2 : a2);
          D = fma2(fx2, add2(fxm, fxp), fma2(fy2, add2(fym, fyp), fma2(fz2, add2(fzm, fzp), mul2(fp2, plate))));
        }
        r = Br[(kr & (SB - 1)) * B_SLOT + me];
        if (!xzero) {
          const float2 x2 = xw2;  // plane kr
          const float2 xl = xc[ma - 1], xr = xc[ma + 1];
          const float2 xL = make_float2(xl.y, x2.x), xR = make_float2(x2.y, xr.x);
          float2 sx = mul2(fxm, sub2(x2, xL));
          sx = fma2(fxp, sub2(x2, xR), sx);
          float2 sy = mul2(fym, sub2(x2, xc[ma - RP]));
          sy = fma2(fyp, sub2(x2, xc[ma + RP]), sy);
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
      Z1s[(kr & 1) * NT + me] = z1;
    }
    // ---- black stage, plane kb = t - 2: z_B = (r + N z1) / D ----
    const int kb = t - 2;
    {
      float zb = 0.f;
      const bool colok = L ? bcol1 : bcol0;
      if (bst && colok && (ST || (kb >= blo && kb < bhi))) {
        const bool zlo = ST || kb > 0, zhi = ST || kb < nz - 1;
        const float2* ac = Ar + (kb & (SA - 1)) * A_SLOT;
        const float* zc = Z1s + (kb & 1) * NT;
        const float a0 = lane(aw2, L);       // plane kb
        const float ain = lane(aw2, L ^ 1);  // the red cell of the pair
        const float aout = L ? ac[ma + 1].x : ac[ma - 1].y;
        const float mout = L ? mxr : mxl;
        float sx = (a0 + ain) * z1w1;  // z1w1: red z of this pair, plane kb
        sx = fmaf(wall(a0 + aout, mout), L ? zc[me + 1] : zc[me - 1], sx);
        float sy = wall(a0 + lane(ac[ma - RP], L), my0) * zc[me - RP];
        sy = fmaf(wall(a0 + lane(ac[ma + RP], L), my1), zc[me + RP], sy);
        float sz = 0.f;
        if (zlo) sz = (a0 + lane(aw1, L)) * z1w0;
        if (zhi) sz = fmaf(a0 + lane(aw3, L), z1w2, sz);
        const float N = fmaf(g.fx, sx, fmaf(g.fy, sy, g.fz * sz));
        zb = (lane(rw1, L) + N) * lane(dw1, L);
      }
      zbw0 = zbw1; zbw1 = zbw2; zbw2 = zb;
      ZBs[(kb & 1) * NT + me] = zb;
    }
    // ---- final stage, plane kf = t - 3: red z and the Chebyshev update ----
    const int kf = t - 3;
    if (fst && (ST || (kf >= k0 && kf < k1))) {
      const bool zlo = ST || kf > 0, zhi = ST || kf < nz - 1;
      const float2* ac = Ar + (kf & (SA - 1)) * A_SLOT;
      const float* zc = ZBs + (kf & 1) * NT;
      const float a0 = lane(aw1, L);  // plane kf
      const float ain = lane(aw1, L ^ 1);
      const float aout = L ? ac[ma + 1].x : ac[ma - 1].y;
      const float mout = L ? mxr : mxl;
      float sx = (a0 + ain) * zbw1;  // zbw1: black z of this pair, plane kf
      sx = fmaf(wall(a0 + aout, mout), L ? zc[me + 1] : zc[me - 1], sx);
      float sy = wall(a0 + lane(ac[ma - RP], L), my0) * zc[me - RP];
      sy = fmaf(wall(a0 + lane(ac[ma + RP], L), my1), zc[me + RP], sy);
      float sz = 0.f;
      if (zlo) sz = (a0 + lane(aw0, L)) * zbw0;
      if (zhi) sz = fmaf(a0 + lane(aw2, L), zbw2, sz);
      const float N = fmaf(g.fx, sx, fmaf(g.fy, sy, g.fz * sz));
      const float zr = (lane(rw0, L) + N) * lane(dw0, L);
      const float2 z = L ? make_float2(zbw1, zr) : make_float2(zr, zbw1);
      const float2 c2 = sc2(P.c2);
      float2 dv = mul2(c2, z);
      if constexpr (!first) dv = fma2(sc2(P.c1), Dr[(kf & (SD - 1)) * D_SLOT + mdp], dv);
      const int q = kf * pl2 + qo;
      if constexpr (keep_d) reinterpret_cast<float2*>(P.d)[q] = dv;
      reinterpret_cast<float2*>(P.xout)[q] = xzero ? dv : add2(xw0, dv);
    }
  };

  // One barrier per plane, at a block-uniform point before each step.  Every
  // shared slot a step writes (red z of t - 1, black z of t - 2; the copies it
  // issues) is read by no one in the same step, and every slot it reads was
  // written before the barrier or waited for.  Steady steps run in pairs.
  using I0 = std::integral_constant<int, 0>;
  using I1 = std::integral_constant<int, 1>;
  using IR = std::integral_constant<int, 2>;
  using TS = std::integral_constant<bool, true>;
  using TG = std::integral_constant<bool, false>;
  const int s0 = max(k0 + 3, 4), s1 = min(k1, nz - 2);  // steady steps
  const bool godd = (gy & 1) != 0;
  int t = tstart;
  while (t <= tend) {
    if (!(t & 1) && t >= s0 && t + 1 <= s1) {
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

// Tile (bx, by)'s region (x from bx FTX - HX, 64 columns; y from by FTY - 3,
// 26 rows) lies inside the domain with no computing cell on a wall.
__device__ __forceinline__ bool inner_tile(const Grid3& g, int bx, int by) {
  return bx >= 1 && by >= 1 && bx * FTX - HX + RW < g.nx && by * FTY - 3 + DR < g.ny;
}

template <int MODE>
__global__ void __launch_bounds__(NT, 1) k_cheb_sgs_tma(const __grid_constant__ TmaArgs P) {
  extern __shared__ unsigned char smraw[];
  const uint32_t raw = (uint32_t)__cvta_generic_to_shared(smraw);
  const uint32_t sbase = (raw + 127u) & ~127u;
  unsigned char* const sm = smraw + (sbase - raw);
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    for (int i = 0; i < NMB; ++i) mbar_init(sbase + OFF_MB + 8u * i, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  Pipe pipe;
  const int nz = P.g.nz;
  const long long G = gridDim.x, b = blockIdx.x;
  // whole columns first (tile r G + b in round r < full), then an equal
  // contiguous share of the leftover columns' (tile, plane) units
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
    if (inner_tile(P.g, bx, by))
      tma_segment<MODE, true>(P, sm, sbase, pipe, bx, by, k0, k1);
    else
      tma_segment<MODE, false>(P, sm, sbase, pipe, bx, by, k0, k1);
    __syncthreads();
  }
}

constexpr int kModes[] = {M_FIRST | M_XZERO, M_FIRST | M_XZERO | M_LAST, 0, M_LAST};

template <int MODE>
cudaError_t set_smem() {
  return cudaFuncSetAttribute(k_cheb_sgs_tma<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TMA_SMEM);
}

constexpr int kMaxDevices = 64;
int g_slots[kMaxDevices] = {};
std::mutex g_mutex;
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
bool g_encode_tried = false;

// Per device: the shared-memory attribute of every step kind set and the
// resident block count known; the tensor-map encoder looked up once.
cudaError_t tma_slots(int* out, PFN_cuTensorMapEncodeTiled_v12000* enc) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_encode_tried) {
    g_encode_tried = true;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  *enc = g_encode;
  int& slots = g_slots[dev];
  if (slots == 0) {
    const cudaError_t es[] = {set_smem<kModes[0]>(), set_smem<kModes[1]>(), set_smem<kModes[2]>(),
                              set_smem<kModes[3]>()};
    for (cudaError_t q : es)
      if (q != cudaSuccess) return q;
    int sms = 0, per = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cheb_sgs_tma<0>, NT, TMA_SMEM);
    if (e != cudaSuccess) return e;
    slots = std::max(1, sms * std::max(1, per));
  }
  *out = slots;
  return cudaSuccess;
}

// A [nz][ny][nx] FP32 array as a 3-D tensor with a box of bw x bh x 1 cells.
bool encode(PFN_cuTensorMapEncodeTiled_v12000 enc, CUtensorMap* m, const float* base, const Grid3& g, int bw, int bh) {
  const cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
  const cuuint64_t strides[2] = {(cuuint64_t)g.nx * sizeof(float), (cuuint64_t)g.plane() * sizeof(float)};
  const cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

}  // namespace

bool tma_smoother_eligible(const Grid3& g, const float* a, const float* b, const float* xin, const float* xout,
                           const float* d, int flags) {
  return (flags & CHEB_EIG) == 0 && g.nx % 4 == 0 && g.nx >= RW && g.ny >= DR && fused_smoother_eligible(g) &&
         aligned16(a) && aligned16(b) && (!xin || aligned16(xin)) && ((uintptr_t)xout & 7) == 0 && aligned16(d);
}

cudaError_t launch_cheb_sgs_tma(const Grid3& g, const float* a, const float* b, const float* xin, float* xout,
                                float* d, double c1, double c2, int flags, int* status, cudaStream_t s) {
  if (!tma_smoother_eligible(g, a, b, xin, xout, d, flags) || !status) return cudaErrorInvalidValue;
  int slots = 0;
  PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
  const cudaError_t e = tma_slots(&slots, &enc);
  if (e != cudaSuccess) return e;
  if (!enc) return cudaErrorNotSupported;  // no tensor-map encoder in this driver
  const int tx = (g.nx + FTX - 1) / FTX, ty = (g.ny + FTY - 1) / FTY;
  const long long units = (long long)tx * ty * g.nz;
  int mode = ((flags & CHEB_FIRST) ? M_FIRST : 0) | (xin ? 0 : M_XZERO) | ((flags & CHEB_LAST) ? M_LAST : 0);
  TmaArgs P;
  memset(&P, 0, sizeof(P));
  P.g = g;
  P.xout = xout;
  P.d = d;
  P.c1 = (float)c1;
  P.c2 = (float)c2;
  P.tiles_x = tx;
  P.units = units;
  P.status = status;
  // the first step with x_in runs as a middle step with c1 = 0 (d is kept finite)
  if ((mode & (M_FIRST | M_XZERO)) == M_FIRST) {
    mode &= ~M_FIRST;
    P.c1 = 0.f;
  }
  const bool rd_x = (mode & M_XZERO) == 0, rd_d = (mode & M_FIRST) == 0;
  if (!encode(enc, &P.ma, a, g, RW, DR) || (rd_x && !encode(enc, &P.mx, xin, g, RW, DR)) ||
      !encode(enc, &P.mb, b, g, RW, TR) || (rd_d && !encode(enc, &P.md, d, g, FTX, FTY)))
    return cudaErrorNotSupported;  // nothing launched: the caller runs the plain kernel
  // one block per resident slot, but at least 4 planes per block on small grids
  const long long blocks = std::max(1LL, std::min((long long)slots, units / 4));
  const dim3 grid((unsigned)blocks), block(RP, TR);
  switch (mode) {
    case M_FIRST | M_XZERO: k_cheb_sgs_tma<M_FIRST | M_XZERO><<<grid, block, TMA_SMEM, s>>>(P); break;
    case M_FIRST | M_XZERO | M_LAST: k_cheb_sgs_tma<M_FIRST | M_XZERO | M_LAST><<<grid, block, TMA_SMEM, s>>>(P); break;
    case 0: k_cheb_sgs_tma<0><<<grid, block, TMA_SMEM, s>>>(P); break;
    case M_LAST: k_cheb_sgs_tma<M_LAST><<<grid, block, TMA_SMEM, s>>>(P); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace gmg
