// One explicit stage of the transport equations of eq. (eM) for a given
// potential, as the second-order semi-implicit step eqs. (e1)-(e2) uses it
// twice (predictor with tau/2, corrector with tau):
//
//   out_e = base_e + c [ div(mu_e E n_e) + div(D_e grad n_e) + S ]
//   out_p = base_p + c [ -div(mu_p E n_p) + S ],   S = alpha(|E|) mu_e |E| n_e,
//
// with n_e, n_p and E taken at the "eval" state.  Finite volumes (Sec. 2.2):
// on each face the upwind cell's density extrapolated with the Koren-limited
// MUSCL slope times the face velocity (-mu_e E_f for electrons, +mu_p E_f for
// ions); E_f = -(phi_q - phi_p)/h with the solve's ghosts (mirror on the side
// walls, 2 g - phi on the plates); densities take two layers of zero-flux
// ghosts; |E| of the source comes from the cell-centred central differences.
//
// FP64 throughout.  GB300 runs FP64 at a small fraction of its FP32 rate, so
// the kernel is bound by the FP64 pipe, not by HBM, and the design removes FP64
// work: every face flux is computed once (a block of 32 x 8 columns marches
// along z; x and y faces of a plane go through shared memory, the z face is
// carried in registers to the next plane), the limiter's sign and min logic runs
// on the integer pipe, and 1/|E| comes from one reciprocal square root.
#include <algorithm>
#include <mutex>

#include "gmg_internal.cuh"

namespace gmg {

namespace {

__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }

// 2 x for finite x >= 0, exactly, on the integer pipe: one more in the exponent
// field for a normal number, the bit pattern doubled for a subnormal one (which
// carries into the exponent exactly when 2 x is normal).
__device__ __forceinline__ double twice(double x) {
  const long long b = dbits(x);
  return __longlong_as_double(b >= (1LL << 52) ? b + (1LL << 52) : b + b);
}

// Koren-limited slope phi(r) b, r = a / b, phi(r) = max(0, min(2r, (1 + 2r)/3, 2)),
// without the division: 0 unless a and b are nonzero with one sign, else
// sign(b) min(2|a|, (|b| + 2|a|)/3, 2|b|).  Only the middle candidate needs FP64
// arithmetic; the sign test, |a|, |b|, the doublings, the minimum of the three
// non-negative candidates (non-negative IEEE doubles order like their 64-bit
// patterns) and the sign of the result are exact integer operations.
__device__ __forceinline__ double koren(double a, double b) {
  const long long ia = dbits(a), ib = dbits(b);
  const long long ma = ia & 0x7fffffffffffffffLL, mb = ib & 0x7fffffffffffffffLL;
  if (ma == 0 || mb == 0 || ((ia ^ ib) < 0)) return 0.0;  // r <= 0 (NaN inputs do not occur)
  const double c1 = twice(__longlong_as_double(ma));
  const double c2 = (__longlong_as_double(mb) + c1) * (1.0 / 3.0);
  long long m = dbits(twice(__longlong_as_double(ma < mb ? ma : mb)));  // min(2|a|, 2|b|)
  const long long m2 = dbits(c2);
  m = m2 < m ? m2 : m;
  return __longlong_as_double(m | (ib & (long long)0x8000000000000000ULL));  // sign of b
}

// Index of a density ghost: two mirrored layers on each side (i in [-2, m+1]).
__device__ __forceinline__ int mirror2(int i, int m) {
  const int r = i < 0 ? -1 - i : (i >= m ? 2 * m - 1 - i : i);
  return r < 0 ? 0 : (r >= m ? m - 1 : r);
}

// Upwind MUSCL value on the face between cells q-1 and q (u0..u3 = cells q-2 ..
// q+1); fwd: the flow crosses the face from q-1 to q.  Forward flow extrapolates
// cell q-1 with the slope of (u2 - u1, u1 - u0); backward flow cell q with that
// of (u1 - u2, u2 - u3), which is minus the slope of (u2 - u1, u3 - u2) (the
// limiter is odd under a joint sign change), so both share one evaluation.
// d1 = u2 - u1, the difference across the face.
__device__ __forceinline__ double face_value(bool fwd, double u0, double u1, double u2, double u3, double d1) {
  const double b = (fwd ? u1 : u3) - (fwd ? u0 : u2);
  const double k = koren(d1, b);
  return (fwd ? u1 : u2) + (fwd ? 0.5 : -0.5) * k;
}

// Scaled drift fluxes through one face.  dphi = phi_{q-1} - phi_q, so the face
// field is E_f = dphi / h; the kernel carries g = dphi n_face per species and
// the physical fluxes are -mu_e g_e / h (electrons drift against E) and
// mu_p g_p / h (ions along it), the mobility and 1/h being applied once per
// cell in the divergence.  Ions cross from q-1 to q when dphi > 0, electrons
// when dphi < 0; at dphi = 0 the flux is zero whichever side is taken.
// FOLD (mu_e > 0): the electron value also carries the diffusion flux,
// g_e += (D / mu_e) (n_q - n_{q-1}) with dk = D / mu_e for the face's axis, so
// that mu_e times its divergence is drift plus diffusion and the cell needs no
// second differences of n_e.
struct FaceFlux {
  double e, p;
};
template <bool FOLD>
__device__ __forceinline__ FaceFlux face_flux(double dphi, double dk, double e0, double e1, double e2, double e3,
                                              double p0, double p1, double p2, double p3) {
  const bool ion_fwd = dbits(dphi) > 0;
  const double d1e = e2 - e1;
  const double ge = dphi * face_value(!ion_fwd, e0, e1, e2, e3, d1e);
  return {FOLD ? fma(dk, d1e, ge) : ge, dphi * face_value(ion_fwd, p0, p1, p2, p3, p2 - p1)};
}

constexpr int TBX = 32, TBY = 8;           // columns per block (one thread each)
constexpr int NT = TBX * TBY;
constexpr int DX = TBX + 4, DY = TBY + 4;  // density tile of one plane: two ghost layers
constexpr int PX = TBX + 2, PY = TBY + 2;  // potential tile: one ghost layer
static_assert(DX * DY <= 2 * NT && PX * PY <= 2 * NT, "two staging loads per thread");

// The ionization rate nu = alpha(|E|) mu_e |E| (S = nu n_e) depends on phi
// only, so the two stages of a step share it: RM = 0 computes it, RM = 1
// computes it and stores it in rate[], RM = 2 reads it from rate[].
//
// Block (bx, by, bz) owns columns [i0, i0+32) x [j0, j0+8) and planes
// [bz kc, min(nz, bz kc + kc)).  Per plane: stage the density and potential
// tiles in shared memory (loaded into registers during the previous plane),
// compute each x face [i0, i0+32] and y face [j0, j0+8] once, the z face above
// the own cell from the column's register windows, then difference the fluxes.
// base_e / base_p may be out_e / out_p (each cell reads its own base value before
// writing).
template <int RM, bool FOLD>
__global__ void __launch_bounds__(NT, 2) k_transport(Grid3 g, TransportCoef tc, const double* base_e,
                                                    const double* base_p, const double* __restrict__ ev_e,
                                                    const double* __restrict__ ev_p,
                                                    const double* __restrict__ phi, double c, double* out_e,
                                                    double* out_p, double* __restrict__ rate, int kc) {
  __shared__ double se[DY][DX], sp[DY][DX], sf[PY][PX];
  __shared__ double xe[TBY][TBX + 1], xp[TBY][TBX + 1], ye[TBY + 1][TBX], yp[TBY + 1][TBX];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TBX + tx;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int i0 = blockIdx.x * TBX, j0 = blockIdx.y * TBY;
  const int i = i0 + tx, j = j0 + ty;
  const bool inside = i < nx && j < ny;
  const int k0 = blockIdx.z * kc, k1 = min(nz, k0 + kc);
  const size_t pl = g.plane();
  const size_t col = (size_t)min(j, ny - 1) * nx + min(i, nx - 1);  // clamped: idle columns load valid data

  // staging: this thread's (up to) two entries of each tile
  unsigned qd[2], qf[2];  // offsets within a plane
  bool hd[2], hf[2];
#pragma unroll
  for (int s2 = 0; s2 < 2; ++s2) {
    const int e = tid + s2 * NT;
    hd[s2] = e < DX * DY;
    hf[s2] = e < PX * PY;
    const int rd = hd[s2] ? e / DX : 0, cd = hd[s2] ? e - rd * DX : 0;
    const int rf = hf[s2] ? e / PX : 0, cf = hf[s2] ? e - rf * PX : 0;
    qd[s2] = (unsigned)(mirror2(j0 - 2 + rd, ny) * nx + mirror2(i0 - 2 + cd, nx));
    qf[s2] = (unsigned)(mirror2(j0 - 1 + rf, ny) * nx + mirror2(i0 - 1 + cf, nx));
  }
  double le[2], lp[2], lf[2];
  auto stage_load = [&](int k) {
    const size_t o = (size_t)k * pl;
#pragma unroll
    for (int s2 = 0; s2 < 2; ++s2) {
      if (hd[s2]) {
        le[s2] = ev_e[o + qd[s2]];
        lp[s2] = ev_p[o + qd[s2]];
      }
      if (hf[s2]) lf[s2] = phi[o + qf[s2]];
    }
  };
  auto stage_store = [&]() {
#pragma unroll
    for (int s2 = 0; s2 < 2; ++s2) {
      const int e = tid + s2 * NT;
      if (hd[s2]) {
        (&se[0][0])[e] = le[s2];
        (&sp[0][0])[e] = lp[s2];
      }
      if (hf[s2]) (&sf[0][0])[e] = lf[s2];
    }
  };
  if (k0 >= k1) return;  // block-uniform
  stage_load(k0);
  stage_store();

  // the column's windows: densities at k-1 .. k+2, potential at k-1 .. k+1
  double ze[4], zp[4];
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    const size_t q = col + (size_t)mirror2(k0 - 2 + d, nz) * pl;
    ze[d] = ev_e[q];
    zp[d] = ev_p[q];
  }
  double pc = phi[col + (size_t)k0 * pl];
  double pm = k0 > 0 ? phi[col + (size_t)(k0 - 1) * pl] : 2.0 * tc.g_bottom - pc;
  double pp = k0 < nz - 1 ? phi[col + (size_t)(k0 + 1) * pl] : 2.0 * tc.g_top - pc;
  // z face below plane k0 (cells k0-2 .. k0+1), then the window moves to k0-1 .. k0+2
  FaceFlux fz_lo = face_flux<FOLD>(pm - pc, tc.dmz, ze[0], ze[1], ze[2], ze[3], zp[0], zp[1], zp[2], zp[3]);
  {
    const size_t q = col + (size_t)mirror2(k0 + 2, nz) * pl;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      ze[d] = ze[d + 1];
      zp[d] = zp[d + 1];
    }
    ze[3] = ev_e[q];
    zp[3] = ev_p[q];
  }

  for (int k = k0; k < k1; ++k) {
    __syncthreads();  // plane k staged; the fluxes of plane k-1 consumed
    const bool more = k + 1 < k1;
    if (more) stage_load(k + 1);
    // next plane's column values and this plane's bases, loaded early
    const size_t qn = col + (size_t)mirror2(k + 3, nz) * pl;
    const double nze = ev_e[qn], nzp = ev_p[qn];
    const double npp = k + 2 < nz ? phi[col + (size_t)(k + 2) * pl] : 0.0;
    const size_t p = col + (size_t)k * pl;
    const double be = inside ? base_e[p] : 0.0, bp = inside ? base_p[p] : 0.0;
    const double nu_in = RM == 2 && inside ? rate[p] : 0.0;

    {  // x face between i-1 and i; y face between j-1 and j
      const FaceFlux fx = face_flux<FOLD>(sf[ty + 1][tx] - sf[ty + 1][tx + 1], tc.dmx, se[ty + 2][tx],
                                    se[ty + 2][tx + 1], se[ty + 2][tx + 2], se[ty + 2][tx + 3], sp[ty + 2][tx],
                                    sp[ty + 2][tx + 1], sp[ty + 2][tx + 2], sp[ty + 2][tx + 3]);
      xe[ty][tx] = fx.e;
      xp[ty][tx] = fx.p;
      const FaceFlux fy = face_flux<FOLD>(sf[ty][tx + 1] - sf[ty + 1][tx + 1], tc.dmy, se[ty][tx + 2],
                                    se[ty + 1][tx + 2], se[ty + 2][tx + 2], se[ty + 3][tx + 2], sp[ty][tx + 2],
                                    sp[ty + 1][tx + 2], sp[ty + 2][tx + 2], sp[ty + 3][tx + 2]);
      ye[ty][tx] = fy.e;
      yp[ty][tx] = fy.p;
    }
    if (ty == 0) {  // the tile's far y faces (between rows j0+TBY-1 and j0+TBY), one per column
      const FaceFlux f = face_flux<FOLD>(sf[TBY][tx + 1] - sf[TBY + 1][tx + 1], tc.dmy, se[TBY][tx + 2],
                                   se[TBY + 1][tx + 2], se[TBY + 2][tx + 2], se[TBY + 3][tx + 2], sp[TBY][tx + 2],
                                   sp[TBY + 1][tx + 2], sp[TBY + 2][tx + 2], sp[TBY + 3][tx + 2]);
      ye[TBY][tx] = f.e;
      yp[TBY][tx] = f.p;
    } else if (ty == 1 && tx < TBY) {  // the far x faces (between i0+TBX-1 and i0+TBX), one per row
      const int r = tx;
      const FaceFlux f = face_flux<FOLD>(sf[r + 1][TBX] - sf[r + 1][TBX + 1], tc.dmx, se[r + 2][TBX],
                                   se[r + 2][TBX + 1], se[r + 2][TBX + 2], se[r + 2][TBX + 3], sp[r + 2][TBX],
                                   sp[r + 2][TBX + 1], sp[r + 2][TBX + 2], sp[r + 2][TBX + 3]);
      xe[r][TBX] = f.e;
      xp[r][TBX] = f.p;
    }
    // z face between k and k+1 (cells k-1 .. k+2)
    const FaceFlux fz_hi = face_flux<FOLD>(pc - pp, tc.dmz, ze[0], ze[1], ze[2], ze[3], zp[0], zp[1], zp[2], zp[3]);

    const double ce = ze[1];
    double nu = nu_in;
    if (RM != 2) {  // |E| at the centre (central differences) and the ionization rate
      const double ex = (sf[ty + 1][tx] - sf[ty + 1][tx + 2]) * tc.ih2x;
      const double ey = (sf[ty][tx + 1] - sf[ty + 2][tx + 1]) * tc.ih2y;
      const double ez = (pm - pp) * tc.ih2z;
      const double e2 = ex * ex + ey * ey + ez * ez;
      const bool field = dbits(e2) > 0;
      const double rinv = rsqrt(e2);  // 1/|E|
      const double eabs = field ? e2 * rinv : 0.0;
      const double alpha = field ? tc.ion_ap * exp(-tc.ion_bp * rinv) : 0.0;
      nu = alpha * tc.mu_e * eabs;
      if (RM == 1 && inside) rate[p] = nu;
    }
    const double src = nu * ce;
    // electron diffusion with one mirrored layer (folded into the face values when FOLD)
    double diff = 0.0;
    if (!FOLD) {
      diff += tc.dih2x * ((se[ty + 2][tx + 3] - 2.0 * ce) + se[ty + 2][tx + 1]);
      diff += tc.dih2y * ((se[ty + 3][tx + 2] - 2.0 * ce) + se[ty + 1][tx + 2]);
      diff += tc.dih2z * ((ze[2] - 2.0 * ce) + ze[0]);
    }
    __syncthreads();  // all faces of plane k written; the tiles of plane k no longer read

    if (inside) {  // div of the scaled fluxes: sum over axes of (g_hi - g_lo) / h^2
      double de = (xe[ty][tx + 1] - xe[ty][tx]) * tc.kx;
      double dp = (xp[ty][tx + 1] - xp[ty][tx]) * tc.kx;
      de += (ye[ty + 1][tx] - ye[ty][tx]) * tc.ky;
      dp += (yp[ty + 1][tx] - yp[ty][tx]) * tc.ky;
      de += (fz_hi.e - fz_lo.e) * tc.kz;
      dp += (fz_hi.p - fz_lo.p) * tc.kz;
      out_e[p] = FOLD ? be + c * (tc.mu_e * de + src) : be + c * ((tc.mu_e * de + diff) + src);
      out_p[p] = bp + c * (src - tc.mu_p * dp);
    }
    if (more) stage_store();
    fz_lo = fz_hi;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      ze[d] = ze[d + 1];
      zp[d] = zp[d + 1];
    }
    ze[3] = nze;
    zp[3] = nzp;
    pm = pc;
    pc = pp;
    pp = k + 2 < nz ? npp : 2.0 * tc.g_top - pc;
  }
}

// Resident blocks of k_transport on the current device (0 = not yet known).
constexpr int kMaxDevices = 64;
int g_transport_slots[kMaxDevices] = {};
std::mutex g_transport_mutex;

cudaError_t transport_slots(int* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_transport_mutex);
  if (g_transport_slots[dev] == 0) {
    int sms = 0, per = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_transport<0, true>, NT, 0);
    if (e != cudaSuccess) return e;
    g_transport_slots[dev] = std::max(1, sms * std::max(1, per));
  }
  *out = g_transport_slots[dev];
  return cudaSuccess;
}

}  // namespace

// Planes per block: the chunk length kc that minimises (waves of blocks) x
// (kc + 1), the 1 standing for a chunk's start-up (its first z face and tile).
static int transport_chunk(int tiles, int nz, int slots) {
  int best = 1;
  long long best_cost = -1;
  for (int kc = 1; kc <= std::min(nz, 64); ++kc) {
    const long long blocks = (long long)tiles * ((nz + kc - 1) / kc);
    const long long waves = (blocks + slots - 1) / slots;
    const long long cost = waves * (kc + 1);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = kc;
    }
  }
  return best;
}

cudaError_t launch_transport(const Grid3& g, const TransportCoef& tc, const double* base_e, const double* base_p,
                             const double* ev_e, const double* ev_p, const double* phi, double c, double* out_e,
                             double* out_p, double* rate, int rate_mode, cudaStream_t s) {
  if ((size_t)g.nx * (size_t)g.ny >= (size_t)1 << 31) return cudaErrorInvalidValue;  // 32-bit plane offsets
  if (rate_mode < 0 || rate_mode > 2 || (rate_mode != 0 && !rate)) return cudaErrorInvalidValue;
  int slots = 0;
  const cudaError_t e = transport_slots(&slots);
  if (e != cudaSuccess) return e;
  const int bx = (g.nx + TBX - 1) / TBX, by = (g.ny + TBY - 1) / TBY;
  const int kc = transport_chunk(bx * by, g.nz, slots);
  dim3 grid((unsigned)bx, (unsigned)by, (unsigned)((g.nz + kc - 1) / kc));
  const dim3 block(TBX, TBY);
#define GMG_TRANSPORT(RM, FOLD) \
  k_transport<RM, FOLD><<<grid, block, 0, s>>>(g, tc, base_e, base_p, ev_e, ev_p, phi, c, out_e, out_p, rate, kc)
  const bool fold = tc.mu_e > 0.0;
  if (rate_mode == 0) {
    if (fold) GMG_TRANSPORT(0, true); else GMG_TRANSPORT(0, false);
  } else if (rate_mode == 1) {
    if (fold) GMG_TRANSPORT(1, true); else GMG_TRANSPORT(1, false);
  } else {
    if (fold) GMG_TRANSPORT(2, true); else GMG_TRANSPORT(2, false);
  }
#undef GMG_TRANSPORT
  return cudaGetLastError();
}

}  // namespace gmg
