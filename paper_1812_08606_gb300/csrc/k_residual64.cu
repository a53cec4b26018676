// The FP64 true residual r = b - A x of the outer FGMRES (Algorithm 1: the
// check after each cycle and the restart vector), A the 7-point operator of
// eq. (e18) with face coefficient (a_p + a_q)/2, mirror (zero-flux) x/y walls
// and the Dirichlet plates' diagonal term.
//
// GB300 runs FP64 at 1/64 of its FP32 rate, so this pass is bound by the FP64
// pipe, and every face product is formed once: a block of 32 x 8 columns
// marches along z; per plane the x and y faces of the tile go through shared
// memory, the z face above a cell is carried in registers to the next plane.
// With G = (a_q + a_p)(x_p - x_q) on the face from cell q to cell p (q below p
// along the axis), (A x)_p = sum over axes c_axis (G_low - G_high), plus
// c_plate a_p x_p on a plate; a wall face (mirror ghost) has G = 0 exactly.
#include <algorithm>
#include <mutex>

#include "gmg_internal.cuh"

namespace gmg {

namespace {

constexpr int QX = 32, QY = 8, QN = QX * QY;
constexpr int SXW = QX + 2, SYH = QY + 2;  // plane tile of x and a with one ghost layer
static_assert(SXW * SYH <= 2 * QN, "two staging loads per thread");

__device__ __forceinline__ int clamp_index(int i, int m) { return i < 0 ? 0 : (i >= m ? m - 1 : i); }

// Block (bx, by, bz): columns [i0, i0+32) x [j0, j0+8), planes [bz kc, min(nz, bz kc + kc)).
__global__ void __launch_bounds__(QN) k_residual64_tiled(Grid3 g, const double* __restrict__ a,
                                                          const double* __restrict__ b,
                                                          const double* __restrict__ x, double* __restrict__ r,
                                                          int kc) {
  __shared__ double sa[SYH][SXW], sx[SYH][SXW];
  __shared__ double gx[QY][QX + 1], gy[QY + 1][QX];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * QX + tx;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int i0 = blockIdx.x * QX, j0 = blockIdx.y * QY;
  const int i = i0 + tx, j = j0 + ty;
  const bool inside = i < nx && j < ny;
  const int k0 = blockIdx.z * kc, k1 = min(nz, k0 + kc);
  if (k0 >= k1) return;  // block-uniform
  const size_t pl = g.plane();
  const size_t col = (size_t)min(j, ny - 1) * nx + min(i, nx - 1);  // clamped: idle columns load valid data
  // this thread's (up to) two staging entries; ghosts copy the wall cell
  size_t qs[2];
  bool hs[2];
#pragma unroll
  for (int s2 = 0; s2 < 2; ++s2) {
    const int e = tid + s2 * QN;
    hs[s2] = e < SXW * SYH;
    const int rr = hs[s2] ? e / SXW : 0, cc = hs[s2] ? e - rr * SXW : 0;
    qs[s2] = (size_t)clamp_index(j0 - 1 + rr, ny) * nx + clamp_index(i0 - 1 + cc, nx);
  }
  // the column's values at plane k and the z face below plane k0
  double xc = x[col + (size_t)k0 * pl], ac = a[col + (size_t)k0 * pl];
  double gz_lo = 0.0;
  if (k0 > 0) {
    const double xm = x[col + (size_t)(k0 - 1) * pl], am = a[col + (size_t)(k0 - 1) * pl];
    gz_lo = (am + ac) * (xc - xm);
  }
  for (int k = k0; k < k1; ++k) {
    const size_t o = (size_t)k * pl;
    __syncthreads();  // the previous plane's faces consumed
#pragma unroll
    for (int s2 = 0; s2 < 2; ++s2) {
      if (hs[s2]) {
        const int e = tid + s2 * QN;
        (&sx[0][0])[e] = x[o + qs[s2]];
        (&sa[0][0])[e] = a[o + qs[s2]];
      }
    }
    const size_t p = col + o;
    const double bp = inside ? b[p] : 0.0;
    double xn = 0.0, an = 0.0;
    if (k + 1 < nz) {
      xn = x[p + pl];
      an = a[p + pl];
    }
    __syncthreads();
    // low x face (i-1, i) and low y face (j-1, j) of the own cell; tile column / row offset 1
    gx[ty][tx] = (sa[ty + 1][tx] + sa[ty + 1][tx + 1]) * (sx[ty + 1][tx + 1] - sx[ty + 1][tx]);
    gy[ty][tx] = (sa[ty][tx + 1] + sa[ty + 1][tx + 1]) * (sx[ty + 1][tx + 1] - sx[ty][tx + 1]);
    if (ty == 0)  // the tile's far y faces (rows j0+7, j0+8)
      gy[QY][tx] = (sa[QY][tx + 1] + sa[QY + 1][tx + 1]) * (sx[QY + 1][tx + 1] - sx[QY][tx + 1]);
    else if (ty == 1 && tx < QY)  // the far x faces (columns i0+31, i0+32)
      gx[tx][QX] = (sa[tx + 1][QX] + sa[tx + 1][QX + 1]) * (sx[tx + 1][QX + 1] - sx[tx + 1][QX]);
    // z face (k, k+1); zero above the top plate (its term is the plate's)
    const double gz_hi = k + 1 < nz ? (ac + an) * (xn - xc) : 0.0;
    __syncthreads();
    if (inside) {
      double ax = g.cx * (gx[ty][tx] - gx[ty][tx + 1]);
      ax = fma(g.cy, gy[ty][tx] - gy[ty + 1][tx], ax);
      ax = fma(g.cz, gz_lo - gz_hi, ax);
      if (k == 0 || k == nz - 1) {  // plate faces (both when nz = 1)
        const double pt = ac * g.cp * xc;
        ax += pt;
        if (nz == 1) ax += pt;
      }
      r[p] = bp - ax;
    }
    gz_lo = gz_hi;
    xc = xn;
    ac = an;
  }
}

constexpr int kMaxDevices = 64;
int g_res_slots[kMaxDevices] = {};
std::mutex g_res_mutex;

cudaError_t residual64_slots(int* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_res_mutex);
  if (g_res_slots[dev] == 0) {
    int sms = 0, per = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_residual64_tiled, QN, 0);
    if (e != cudaSuccess) return e;
    g_res_slots[dev] = std::max(1, sms * std::max(1, per));
  }
  *out = g_res_slots[dev];
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_residual64_tiled(const Grid3& g, const double* a, const double* b, const double* x, double* r,
                                   cudaStream_t s) {
  int slots = 0;
  const cudaError_t e = residual64_slots(&slots);
  if (e != cudaSuccess) return e;
  const int bx = (g.nx + QX - 1) / QX, by = (g.ny + QY - 1) / QY;
  // planes per block: the chunk that minimises (waves of blocks) x (chunk + 1)
  int best = 1;
  long long best_cost = -1;
  for (int c = 1; c <= std::min(g.nz, 64); ++c) {
    const long long blocks = (long long)bx * by * ((g.nz + c - 1) / c);
    const long long cost = ((blocks + slots - 1) / slots) * (c + 1);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = c;
    }
  }
  dim3 grid((unsigned)bx, (unsigned)by, (unsigned)((g.nz + best - 1) / best));
  k_residual64_tiled<<<grid, dim3(QX, QY), 0, s>>>(g, a, b, x, r, best);
  return cudaGetLastError();
}

}  // namespace gmg
