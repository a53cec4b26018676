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
// FP64 throughout, one thread per cell.
#include "gmg_internal.cuh"

namespace gmg {

namespace {

// Koren-limited slope phi(r) b, r = a / b, without the division (GB300 runs an
// FP64 divide as a multi-instruction sequence; 1/3 is a multiplication).
__device__ __forceinline__ double koren(double a, double b) {
  if (!(a * b > 0.0)) return 0.0;
  const double aa = fabs(a), ab = fabs(b);
  const double s = fmin(fmin(2.0 * aa, (ab + 2.0 * aa) * (1.0 / 3.0)), 2.0 * ab);
  return copysign(s, b);
}

// Index of a density ghost: two mirrored layers on each side (i in [-2, m+1]).
__device__ __forceinline__ int mirror2(int i, int m) {
  const int r = i < 0 ? -1 - i : (i >= m ? 2 * m - 1 - i : i);
  return r < 0 ? 0 : (r >= m ? m - 1 : r);
}

// Upwind face value on the face between cells q-1 and q; u[0..3] = cells q-2 .. q+1 along the axis.
__device__ __forceinline__ double face_value(double v, const double* u) {
  return v > 0.0 ? u[1] + 0.5 * koren(u[2] - u[1], u[1] - u[0]) : u[2] + 0.5 * koren(u[1] - u[2], u[2] - u[3]);
}

// base_e / base_p may be out_e / out_p (each cell reads its own base value before writing).
__global__ void __launch_bounds__(256) k_transport(Grid3 g, TransportCoef tc, const double* base_e,
                                                   const double* base_p,
                                                   const double* __restrict__ ev_e, const double* __restrict__ ev_p,
                                                   const double* __restrict__ phi, double c, double* out_e,
                                                   double* out_p) {
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y * 8 + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const size_t pl = g.plane();
  const size_t p = ((size_t)k * ny + j) * nx + i;
  const double fc = phi[p];
  // phi of the six neighbours with the solve's ghosts
  const double fxm = i > 0 ? phi[p - 1] : fc, fxp = i < nx - 1 ? phi[p + 1] : fc;
  const double fym = j > 0 ? phi[p - nx] : fc, fyp = j < ny - 1 ? phi[p + nx] : fc;
  const double fzm = k > 0 ? phi[p - pl] : 2.0 * tc.g_bottom - fc;
  const double fzp = k < nz - 1 ? phi[p + pl] : 2.0 * tc.g_top - fc;
  // |E| at the centre (central differences) and the ionization source rate
  const double ex = (fxm - fxp) * tc.ih2x, ey = (fym - fyp) * tc.ih2y, ez = (fzm - fzp) * tc.ih2z;
  const double eabs = sqrt(ex * ex + ey * ey + ez * ez);
  const double alpha = eabs > 0.0 ? tc.ion_ap * exp(-tc.ion_bp / eabs) : 0.0;
  const double src = alpha * tc.mu_e * eabs * ev_e[p];
  // face fields: low and high face along each axis
  const double E[3][2] = {{(fxm - fc) * tc.ihx, (fc - fxp) * tc.ihx},
                          {(fym - fc) * tc.ihy, (fc - fyp) * tc.ihy},
                          {(fzm - fc) * tc.ihz, (fc - fzp) * tc.ihz}};
  const int pos[3] = {i, j, k}, len[3] = {nx, ny, nz};
  const size_t stride[3] = {1, (size_t)nx, pl};
  const double ih[3] = {tc.ihx, tc.ihy, tc.ihz};
  const double dd[3] = {tc.dih2x, tc.dih2y, tc.dih2z};  // D_alpha / h_alpha^2
  double div_e = 0.0, div_p = 0.0, diff = 0.0;
  const double ce = ev_e[p];
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const size_t base = p - (size_t)pos[ax] * stride[ax];  // the cell with index 0 on this line
    double ue[5], up[5];                                     // cells pos-2 .. pos+2
#pragma unroll
    for (int d = 0; d < 5; ++d) {
      const size_t q = base + (size_t)mirror2(pos[ax] + d - 2, len[ax]) * stride[ax];
      ue[d] = ev_e[q];
      up[d] = ev_p[q];
    }
    // low face (between pos-1 and pos): cells pos-2 .. pos+1; high face: pos-1 .. pos+2
    const double vlo_e = -tc.mu_e * E[ax][0], vhi_e = -tc.mu_e * E[ax][1];
    const double vlo_p = tc.mu_p * E[ax][0], vhi_p = tc.mu_p * E[ax][1];
    const double flo_e = vlo_e * face_value(vlo_e, ue), fhi_e = vhi_e * face_value(vhi_e, ue + 1);
    const double flo_p = vlo_p * face_value(vlo_p, up), fhi_p = vhi_p * face_value(vhi_p, up + 1);
    div_e += (fhi_e - flo_e) * ih[ax];
    div_p += (fhi_p - flo_p) * ih[ax];
    // electron diffusion with one mirrored layer (ue[1], ue[3] are the neighbours)
    diff += dd[ax] * ((ue[3] - 2.0 * ce) + ue[1]);
  }
  out_e[p] = base_e[p] + c * ((-div_e + diff) + src);
  out_p[p] = base_p[p] + c * (-div_p + src);
}

}  // namespace

cudaError_t launch_transport(const Grid3& g, const TransportCoef& tc, const double* base_e, const double* base_p,
                             const double* ev_e, const double* ev_p, const double* phi, double c, double* out_e,
                             double* out_p, cudaStream_t s) {
  dim3 grid((unsigned)((g.nx + 31) / 32), (unsigned)((g.ny + 7) / 8), (unsigned)g.nz);
  k_transport<<<grid, dim3(32, 8), 0, s>>>(g, tc, base_e, base_p, ev_e, ev_p, phi, c, out_e, out_p);
  return cudaGetLastError();
}

}  // namespace gmg
