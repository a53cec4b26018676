// Levels whose operator carries one coefficient per face (the coarse levels
// of the series-parallel coarsening), and the operator-dependent
// prolongation.
//
// Face form of a level (see gmg_level_faces): matrix entries, i.e. the face
// coefficient divided by h^2, of the low faces of every cell
//   kx[k][j][i]  couples cells i-1 and i (0 at i = 0, the side wall),
//   ky[k][j][i]  couples rows  j-1 and j (0 at j = 0),
//   kz[k][j][i]  couples planes k-1 and k; at k = 0 the bottom plate's entry,
//   ktop[j][i]   the top plate's entry,
// so (A x)_p = sum over the six faces of k_f (x_p - x_q), with x_q = 0 beyond
// a plate (the homogeneous Dirichlet ghost; the plate data enter the
// right-hand side only on the finest level).
//
// Coarsening (from a cell-form level, eq. (e18), or a face-form level): with
// fine entries k1, k2, k3 of the three fine links between the centres of
// coarse cells I-1 and I (half of each coarse cell's inner link in series
// with the link they share), a coarse column carries 1 / (1/k1 + 2/k2 + 1/k3);
// the four fine columns crossing the coarse face add in parallel (their
// mean).  A coarse plate face: 1 / (1/k_inner + 2/k_plate).  With a constant
// coefficient this is the re-discretised operator on the coarse grid.
//
// Operator-dependent prolongation: per axis the fine child mixes its parent
// and the coarse neighbour on its side with weights from the series
// resistances between them, R_parent = 1/(2 k_inner) and R_neighbour =
// 1/k_shared + 1/(2 k_neighbour_inner) (in units of h^2); the parent's weight
// is R_n / (R_n + R_p).  At a side wall the parent's weight is 1; at a plate
// the neighbour is the plate (value 0) with R_n = 1/k_plate.  The three axes
// combine as a tensor product.
#include <algorithm>
#include <type_traits>

#include "gmg_internal.cuh"

namespace gmg {

namespace {

constexpr int BX = 32, BY = 8;

inline dim3 grid_cells(const Grid3& g) {
  return dim3((unsigned)((g.nx + BX - 1) / BX), (unsigned)((g.ny + BY - 1) / BY), (unsigned)g.nz);
}

template <typename C>
struct Six {
  C xm, xp, ym, yp, zm, zp;  // zm / zp are the plate entries on the first / last plane
};

template <typename C, typename T>
__device__ __forceinline__ Six<C> load_six(const Grid3& g, const Faces<T>& F, int i, int j, int k, size_t p) {
  const size_t pl = g.plane();
  Six<C> s;
  s.xm = i > 0 ? (C)ldg(F.kx + p) : (C)0;
  s.xp = i < g.nx - 1 ? (C)ldg(F.kx + p + 1) : (C)0;
  s.ym = j > 0 ? (C)ldg(F.ky + p) : (C)0;
  s.yp = j < g.ny - 1 ? (C)ldg(F.ky + p + g.nx) : (C)0;
  s.zm = (C)ldg(F.kz + p);
  s.zp = k < g.nz - 1 ? (C)ldg(F.kz + p + pl) : (C)ldg(F.ktop + (p - (size_t)k * pl));
  return s;
}

// (A x)_p in the difference form.
template <typename C, typename T, typename TX>
__device__ __forceinline__ C face_diff(const Grid3& g, const Faces<T>& F, const TX* __restrict__ x, int i, int j,
                                       int k, size_t p) {
  const Six<C> s = load_six<C>(g, F, i, j, k, p);
  const size_t pl = g.plane();
  const C xp = (C)ldg(x + p);
  C acc = (C)0;
  if (i > 0) acc += s.xm * (xp - (C)ldg(x + p - 1));
  if (i < g.nx - 1) acc += s.xp * (xp - (C)ldg(x + p + 1));
  if (j > 0) acc += s.ym * (xp - (C)ldg(x + p - g.nx));
  if (j < g.ny - 1) acc += s.yp * (xp - (C)ldg(x + p + g.nx));
  acc += k > 0 ? s.zm * (xp - (C)ldg(x + p - pl)) : s.zm * xp;
  acc += k < g.nz - 1 ? s.zp * (xp - (C)ldg(x + p + pl)) : s.zp * xp;
  return acc;
}

// Diagonal D_p and neighbour sum (N z)_p (z may be null: zero).
template <typename C, typename T>
__device__ __forceinline__ void face_split(const Grid3& g, const Faces<T>& F, const T* z, int i, int j, int k,
                                           size_t p, C& diag, C& nsum) {
  const Six<C> s = load_six<C>(g, F, i, j, k, p);
  const size_t pl = g.plane();
  diag = ((s.xm + s.xp) + (s.ym + s.yp)) + (s.zm + s.zp);
  C t = (C)0;
  if (z) {
    if (i > 0) t += s.xm * (C)z[p - 1];
    if (i < g.nx - 1) t += s.xp * (C)z[p + 1];
    if (j > 0) t += s.ym * (C)z[p - g.nx];
    if (j < g.ny - 1) t += s.yp * (C)z[p + g.nx];
    if (k > 0) t += s.zm * (C)z[p - pl];
    if (k < g.nz - 1) t += s.zp * (C)z[p + pl];
  }
  nsum = t;
}

template <typename C, typename T, typename TX, typename TY>
__global__ void __launch_bounds__(BX* BY) k_apply_faces(Grid3 g, Faces<T> F, const TX* __restrict__ x,
                                                        TY* __restrict__ y) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  const size_t p = ((size_t)k * g.ny + j) * g.nx + i;
  y[p] = (TY)face_diff<C>(g, F, x, i, j, k, p);
}

template <typename T>
__global__ void __launch_bounds__(BX* BY) k_residual_faces(Grid3 g, Faces<T> F, const T* __restrict__ b,
                                                           const T* __restrict__ x, T* __restrict__ r,
                                                           T* __restrict__ z, int pc) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  const size_t p = ((size_t)k * g.ny + j) * g.nx + i;
  T res = ldg(b + p);
  if (x) res -= face_diff<T>(g, F, x, i, j, k, p);
  if (r) r[p] = res;
  if (pc == PC_IDENTITY) {
    z[p] = res;
  } else if (pc == PC_JACOBI || (pc == PC_SGS && ((i + j + k) & 1) == 0)) {
    T diag, nsum;
    face_split<T>(g, F, (const T*)nullptr, i, j, k, p, diag, nsum);
    z[p] = res / diag;
  }
}

template <typename T>
__global__ void __launch_bounds__(BX* BY) k_sgs_half_faces(Grid3 g, Faces<T> F, const T* __restrict__ r, T* z,
                                                           int color, T* __restrict__ d, T* __restrict__ x, T c1,
                                                           T c2, int flags) {
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  const int i = 2 * (int)(blockIdx.x * BX + threadIdx.x) + ((j + k + color) & 1);
  if (i >= g.nx || j >= g.ny) return;
  const size_t p = ((size_t)k * g.ny + j) * g.nx + i;
  T diag, nsum;
  face_split<T>(g, F, (const T*)z, i, j, k, p, diag, nsum);
  const T zp = (ldg(r + p) + nsum) / diag;
  z[p] = zp;
  if (flags & CHEB_UPDATE) {
    const T dp = (flags & CHEB_FIRST) ? c2 * zp : c1 * d[p] + c2 * zp;
    d[p] = dp;
    x[p] = (flags & CHEB_XZERO) ? dp : x[p] + dp;
  }
}

// coarse = mean over the 8 children of (b - A x); one thread per coarse cell.
template <typename T>
__global__ void __launch_bounds__(BX* BY) k_residual_restrict_faces(Grid3 g, Faces<T> F, const T* __restrict__ b,
                                                                    const T* __restrict__ x, T* __restrict__ coarse) {
  const int nxc = g.nx / 2, nyc = g.ny / 2;
  const int ic = blockIdx.x * BX + threadIdx.x;
  const int jc = blockIdx.y * BY + threadIdx.y;
  const int kc = blockIdx.z;
  if (ic >= nxc || jc >= nyc) return;
  T sum = (T)0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int i = 2 * ic + (c & 1), j = 2 * jc + ((c >> 1) & 1), k = 2 * kc + (c >> 2);
    const size_t p = ((size_t)k * g.ny + j) * g.nx + i;
    sum += ldg(b + p) - face_diff<T>(g, F, x, i, j, k, p);
  }
  coarse[((size_t)kc * nyc + jc) * nxc + ic] = sum * (T)0.125;
}

// The fine level's link entries, from a cell coefficient (eq. (e18): face
// means, plate faces 2 a_p / hz^2) or from stored faces.
template <typename T, bool CELL>
struct Links {
  Grid3 g;
  const T* a;
  Faces<T> F;
  // entry of the x link between cells i-1 and i of row (j, k), 1 <= i < nx
  __device__ __forceinline__ T x(int i, int j, int k) const {
    const size_t p = ((size_t)k * g.ny + j) * g.nx + i;
    if constexpr (CELL) return (ldg(a + p - 1) + ldg(a + p)) * GridCoef<T>::x(g);
    else return ldg(F.kx + p);
  }
  __device__ __forceinline__ T y(int i, int j, int k) const {
    const size_t p = ((size_t)k * g.ny + j) * g.nx + i;
    if constexpr (CELL) return (ldg(a + p - g.nx) + ldg(a + p)) * GridCoef<T>::y(g);
    else return ldg(F.ky + p);
  }
  // z link between planes k-1 and k (1 <= k < nz); k = 0: bottom plate; k = nz: top plate
  __device__ __forceinline__ T z(int i, int j, int k) const {
    const size_t pl = g.plane(), q = (size_t)j * g.nx + i;
    if constexpr (CELL) {
      if (k == 0) return ldg(a + q) * GridCoef<T>::p(g);
      if (k == g.nz) return ldg(a + (size_t)(g.nz - 1) * pl + q) * GridCoef<T>::p(g);
      return (ldg(a + (size_t)(k - 1) * pl + q) + ldg(a + (size_t)k * pl + q)) * GridCoef<T>::z(g);
    } else {
      if (k == g.nz) return ldg(F.ktop + q);
      return ldg(F.kz + (size_t)k * pl + q);
    }
  }
};

// Quotients of the set-up: in FP32 the fast hardware reciprocal (about 2 ulp;
// the coarse operators and the weights only shape the FP32 preconditioner),
// in FP64 the correctly rounded division.
__device__ __forceinline__ float quot(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double quot(double a, double b) { return a / b; }

// 1 / (1/k1 + 2/k2 + 1/k3) as k1 k3 / (k1 + k3 + 2 k1 k3 / k2): two quotients
// instead of four, and no product of more than two entries (no overflow).
template <typename T>
__device__ __forceinline__ T series3(T k1, T k2, T k3) {
  const T p = k1 * k3;
  return quot(p, k1 + k3 + (T)2 * quot(p, k2));
}
template <typename T>
__device__ __forceinline__ T series_plate(T kin, T kplate) {
  return quot(kin * kplate, kplate + (T)2 * kin);  // 1 / (1/kin + 2/kplate)
}

// One thread per coarse column (I, J) of a 32 x 8 block, marching through
// kchunk coarse planes: per coarse cell its low faces and, on the last coarse
// plane, its top plate face.  g is the fine grid.
template <typename T, bool CELL>
__global__ void __launch_bounds__(256) k_coarsen_faces(Links<T, CELL> L, T* __restrict__ kx, T* __restrict__ ky,
                                                       T* __restrict__ kz, T* __restrict__ ktop, int kchunk) {
  const Grid3& g = L.g;
  const int nxc = g.nx / 2, nyc = g.ny / 2, nzc = g.nz / 2;
  const int I = blockIdx.x * 32 + threadIdx.x, J = blockIdx.y * 8 + threadIdx.y;
  if (I >= nxc || J >= nyc) return;
  const int K0 = blockIdx.z * kchunk, K1 = min(nzc, K0 + kchunk);
  const size_t plc = (size_t)nxc * nyc;
  size_t q = (size_t)K0 * plc + (size_t)J * nxc + I;
  for (int K = K0; K < K1; ++K, q += plc) {
    T sx = (T)0, sy = (T)0, sz = (T)0, st = (T)0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int u = c & 1, v = c >> 1;
      if (I > 0) sx += series3(L.x(2 * I - 1, 2 * J + u, 2 * K + v), L.x(2 * I, 2 * J + u, 2 * K + v),
                               L.x(2 * I + 1, 2 * J + u, 2 * K + v));
      if (J > 0) sy += series3(L.y(2 * I + u, 2 * J - 1, 2 * K + v), L.y(2 * I + u, 2 * J, 2 * K + v),
                               L.y(2 * I + u, 2 * J + 1, 2 * K + v));
      if (K > 0)
        sz += series3(L.z(2 * I + u, 2 * J + v, 2 * K - 1), L.z(2 * I + u, 2 * J + v, 2 * K),
                      L.z(2 * I + u, 2 * J + v, 2 * K + 1));
      else
        sz += series_plate(L.z(2 * I + u, 2 * J + v, 1), L.z(2 * I + u, 2 * J + v, 0));
      if (K == nzc - 1) st += series_plate(L.z(2 * I + u, 2 * J + v, g.nz - 1), L.z(2 * I + u, 2 * J + v, g.nz));
    }
    kx[q] = (T)0.25 * sx;
    ky[q] = (T)0.25 * sy;
    kz[q] = (T)0.25 * sz;
    if (K == nzc - 1) ktop[(size_t)J * nxc + I] = (T)0.25 * st;
  }
}

// Face form of a cell-coefficient level (for gmg_level_faces), FP64 out.
template <typename T>
__global__ void k_faces_of_cells(Links<T, true> L, double* __restrict__ kx, double* __restrict__ ky,
                                 double* __restrict__ kz, double* __restrict__ ktop) {
  const Grid3& g = L.g;
  const size_t n = g.n();
  for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(p % g.nx), j = (int)((p / g.nx) % g.ny), k = (int)(p / g.plane());
    kx[p] = i > 0 ? (double)L.x(i, j, k) : 0.0;
    ky[p] = j > 0 ? (double)L.y(i, j, k) : 0.0;
    kz[p] = (double)L.z(i, j, k);
    if (k == g.nz - 1) ktop[(size_t)j * g.nx + i] = (double)L.z(i, j, g.nz);
  }
}

// Parent weight R_n / (R_n + R_p) along one axis for fine index c of n (n
// even) with link entries lk(m) (m = 1..n-1 interior; lk(0), lk(n) the plates
// when `plates`), with the denominators cleared: one quotient instead of four,
// the same value up to rounding.  Low child (c even), links k0 = lk(c-1),
// k1 = lk(c), k2 = lk(c+1) (to its sibling):
//   R_n = 1/k1 + 1/(2 k0), R_p = 1/(2 k2)  =>  w = (2 k0 + k1) k2 / ((2 k0 + k1) k2 + k0 k1);
// the high child mirrors it (k0 = lk(c) to its sibling, k1 = lk(c+1), k2 = lk(c+2));
// next to a plate (R_n = 1/k_plate, R_p = 1/(2 k_in)): w = 2 k_in / (2 k_in + k_plate).
// Products of two entries stay far inside the FP32 range.
template <typename T, typename F>
__device__ __forceinline__ T parent_weight(int c, int n, bool plates, F lk) {
  const int m = n / 2, I = c >> 1;
  if ((c & 1) == 0) {
    const T k2 = lk(c + 1);
    if (I > 0) {
      const T k0 = lk(c - 1), k1 = lk(c);
      const T s = ((T)2 * k0 + k1) * k2;
      return quot(s, s + k0 * k1);
    }
    if (plates) return quot((T)2 * k2, (T)2 * k2 + lk(0));
    return (T)1;
  }
  const T k0 = lk(c);
  if (I < m - 1) {
    const T k1 = lk(c + 1), k2 = lk(c + 2);
    const T s = ((T)2 * k2 + k1) * k0;
    return quot(s, s + k1 * k2);
  }
  if (plates) return quot((T)2 * k0, (T)2 * k0 + lk(n));
  return (T)1;
}

// One thread per (i, j) column of a 32 x 8 block, marching through kchunk
// planes: cell indices come from the grid, with no division per cell.
template <typename T, bool CELL>
__global__ void __launch_bounds__(256) k_prolong_weights(Links<T, CELL> L, T* __restrict__ w, int kchunk) {
  const Grid3& g = L.g;
  const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y;
  if (i >= g.nx || j >= g.ny) return;
  const int k0 = blockIdx.z * kchunk, k1 = min(g.nz, k0 + kchunk);
  const size_t n = g.n(), pl = g.plane();
  size_t p = (size_t)k0 * pl + (size_t)j * g.nx + i;
  for (int k = k0; k < k1; ++k, p += pl) {
    w[p] = parent_weight<T>(i, g.nx, false, [&](int m) { return L.x(m, j, k); });
    w[n + p] = parent_weight<T>(j, g.ny, false, [&](int m) { return L.y(i, m, k); });
    w[2 * n + p] = parent_weight<T>(k, g.nz, true, [&](int m) { return L.z(i, j, m); });
  }
}

// x_fine += P e with per-cell parent weights w (wx | wy | wz).
template <typename T>
__global__ void __launch_bounds__(BX* BY) k_prolong_opdep(Grid3 g, const T* __restrict__ e, T* __restrict__ x,
                                                          const T* __restrict__ w) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  const int nxc = g.nx / 2, nyc = g.ny / 2, nzc = g.nz / 2;
  const int ic = i >> 1, jc = j >> 1, kc = k >> 1;
  const size_t n = g.n(), p = ((size_t)k * g.ny + j) * g.nx + i;
  const int in = (i & 1) ? ic + 1 : ic - 1;
  const int jn = (j & 1) ? jc + 1 : jc - 1;
  const int kn = (k & 1) ? kc + 1 : kc - 1;
  const bool kin = kn >= 0 && kn < nzc;
  const int ii[2] = {ic, (in >= 0 && in < nxc) ? in : ic};  // a wall neighbour has weight 0
  const int jj[2] = {jc, (jn >= 0 && jn < nyc) ? jn : jc};
  const int kk[2] = {kc, kin ? kn : kc};
  const T wx = ldg(w + p), wy = ldg(w + n + p), wz = ldg(w + 2 * n + p);
  const T Wx[2] = {wx, (T)1 - wx}, Wy[2] = {wy, (T)1 - wy}, Wz[2] = {wz, (T)1 - wz};
  auto at = [&](int a, int b2, int c) { return ldg(e + ((size_t)a * nyc + b2) * nxc + c); };
  T v = (T)0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int sx = c & 1, sy = (c >> 1) & 1, sz = c >> 2;
    if (sz && !kin) continue;  // beyond a plate: the homogeneous Dirichlet value 0
    v += Wz[sz] * (Wy[sy] * (Wx[sx] * at(kk[sz], jj[sy], ii[sx])));
  }
  x[p] += v;
}

// The same prolongation in FP32 with one thread per fine cell pair (2 ic,
// 2 ic + 1) of one fine row j, marching through coarse planes [kc0, kc1)
// (fine planes 2 kc, 2 kc + 1).  The thread keeps its coarse column ic (rows jc
// and the y-neighbour row jn, planes kc - 1 .. kc + 1) in registers; the
// columns ic - 1 and ic + 1 come from the neighbouring lanes by shuffle (the
// first and last lane of a warp load theirs).  Each fine cell interpolates the
// two columns it needs in y and z with its own weights, then combines them in
// x.  Weights, x and e are read as float2 pairs: 8-byte aligned arrays, nx even.
constexpr int PTP = 32;  // pairs per row = lanes
constexpr int PTR = 8;   // fine rows per block
constexpr unsigned FULLMASK = 0xffffffffu;

__global__ void __launch_bounds__(PTP* PTR) k_prolong_opdep_pairs(Grid3 g, const float* __restrict__ e,
                                                                float* __restrict__ x, const float* __restrict__ w,
                                                                int kchunk) {
  const int nx = g.nx, ny = g.ny;
  const int nxc = nx / 2, nyc = ny / 2, nzc = g.nz / 2;
  const int tx = threadIdx.x;
  const int ip = blockIdx.x * PTP + tx;
  const int j = blockIdx.y * PTR + threadIdx.y;
  const int kc0 = blockIdx.z * kchunk, kc1 = min(nzc, kc0 + kchunk);
  const bool act = ip < nxc && j < ny;
  const int jc = j >> 1;
  int jn = (j & 1) ? jc + 1 : jc - 1;
  if (jn < 0 || jn >= nyc) jn = jc;  // side wall: the weight array gives this neighbour weight 0
  const int ih = tx == 0 ? ip - 1 : (tx == PTP - 1 ? ip + 1 : -1);  // the edge lanes' extra column
  const bool hact = act && ih >= 0 && ih < nxc;
  // 32-bit offsets: the launcher keeps nz + 4 planes of fine cells below 2^31
  const int pc = nyc * nxc;
  const int rc = act ? jc * nxc : 0, rn = act ? jn * nxc : 0;
  auto ld = [&](bool on, int kc, int row, int col) {
    return (on && kc >= 0 && kc < nzc) ? __ldg(e + (kc * pc + row + col)) : 0.f;
  };
  // coarse planes kc - 1, kc, kc + 1 of rows (jc, jn): own column (c*, n*) and extra column (h*, q*)
  float cm = ld(act, kc0 - 1, rc, ip), nm = ld(act, kc0 - 1, rn, ip);
  float c0 = ld(act, kc0, rc, ip), n0 = ld(act, kc0, rn, ip);
  float cp = ld(act, kc0 + 1, rc, ip), np = ld(act, kc0 + 1, rn, ip);
  float hm = ld(hact, kc0 - 1, rc, ih), qm = ld(hact, kc0 - 1, rn, ih);
  float h0 = ld(hact, kc0, rc, ih), q0 = ld(hact, kc0, rn, ih);
  float hp = ld(hact, kc0 + 1, rc, ih), qp = ld(hact, kc0 + 1, rn, ih);
  const int n = (int)g.n();
  const int pl2 = (int)(g.plane() >> 1);
  const int q = act ? (j * nx + 2 * ip) >> 1 : 0;
  float2* X2 = reinterpret_cast<float2*>(x);
  const float2* WX = reinterpret_cast<const float2*>(w);
  const float2* WY = reinterpret_cast<const float2*>(w + n);
  const float2* WZ = reinterpret_cast<const float2*>(w + 2 * n);
  for (int kc = kc0; kc < kc1; ++kc) {
    const float c1 = ld(act, kc + 2, rc, ip), n1 = ld(act, kc + 2, rn, ip);
    const float h1 = ld(hact, kc + 2, rc, ih), q1 = ld(hact, kc + 2, rn, ih);
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int k = 2 * kc + half;
      // the plane beyond the parent's on this child's side; zero beyond a plate
      const bool kin = half ? kc + 1 < nzc : kc > 0;
      const float oc = half ? cp : cm, on = half ? np : nm;   // own column, neighbour plane
      const float ho = half ? hp : hm, qo = half ? qp : qm;   // extra column, neighbour plane
      const float oz = kin ? oc : 0.f, ozn = kin ? on : 0.f, hz = kin ? ho : 0.f, qz = kin ? qo : 0.f;
      // columns ic - 1 (from the lane on the left) and ic + 1 (on the right): rows jc, jn at kc and beyond
      float lc = __shfl_up_sync(FULLMASK, c0, 1), ln = __shfl_up_sync(FULLMASK, n0, 1);
      float lz = __shfl_up_sync(FULLMASK, oz, 1), lzn = __shfl_up_sync(FULLMASK, ozn, 1);
      float uc = __shfl_down_sync(FULLMASK, c0, 1), un = __shfl_down_sync(FULLMASK, n0, 1);
      float uz = __shfl_down_sync(FULLMASK, oz, 1), uzn = __shfl_down_sync(FULLMASK, ozn, 1);
      if (tx == 0) { lc = h0; ln = q0; lz = hz; lzn = qz; }
      if (tx == PTP - 1) { uc = h0; un = q0; uz = hz; uzn = qz; }
      if (act) {
        const int o = k * pl2 + q;
        // this cell's weights and x two planes ahead into L2: the loads below have
        // no lead, and with them the kernel ran at 5.0 TB/s instead of 6.8
        if (k + 2 < g.nz) {
          asm volatile("prefetch.global.L2 [%0];" ::"l"(WX + o + 2 * pl2));
          asm volatile("prefetch.global.L2 [%0];" ::"l"(WY + o + 2 * pl2));
          asm volatile("prefetch.global.L2 [%0];" ::"l"(WZ + o + 2 * pl2));
          asm volatile("prefetch.global.L2 [%0];" ::"l"(X2 + o + 2 * pl2));
        }
        const float2 wx = __ldg(WX + o), wy = __ldg(WY + o), wz = __ldg(WZ + o);
        // y then z for one column with a cell's weights
        auto yz = [](float wyv, float wzv, float e00, float e01, float e10, float e11) {
          const float a0 = fmaf(wyv, e00 - e01, e01);  // wy e(jc) + (1 - wy) e(jn), plane kc
          const float a1 = fmaf(wyv, e10 - e11, e11);  // the same on the neighbour plane
          return fmaf(wzv, a0 - a1, a1);
        };
        const float own0 = yz(wy.x, wz.x, c0, n0, oz, ozn), left = yz(wy.x, wz.x, lc, ln, lz, lzn);
        const float own1 = yz(wy.y, wz.y, c0, n0, oz, ozn), right = yz(wy.y, wz.y, uc, un, uz, uzn);
        const float v0 = fmaf(wx.x, own0 - left, left), v1 = fmaf(wx.y, own1 - right, right);
        float2 xv = X2[o];
        xv.x += v0;
        xv.y += v1;
        X2[o] = xv;
      }
    }
    cm = c0; nm = n0; c0 = cp; n0 = np; cp = c1; np = n1;
    hm = h0; qm = q0; h0 = hp; q0 = qp; hp = h1; qp = q1;
  }
}

// Dense coarsest operator from faces, one thread per row.
template <typename T>
__global__ void k_coarse_assemble_faces(Grid3 g, Faces<T> F, double* __restrict__ A) {
  const int n = (int)g.n();
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n) return;
  const int i = row % g.nx, j = (row / g.nx) % g.ny, k = row / (g.nx * g.ny);
  const int pl = g.nx * g.ny;
  double* Ar = A + (size_t)row * n;
  for (int c = 0; c < n; ++c) Ar[c] = 0.0;
  const Six<double> s = load_six<double>(g, F, i, j, k, (size_t)row);
  if (i > 0) Ar[row - 1] = -s.xm;
  if (i < g.nx - 1) Ar[row + 1] = -s.xp;
  if (j > 0) Ar[row - g.nx] = -s.ym;
  if (j < g.ny - 1) Ar[row + g.nx] = -s.yp;
  if (k > 0) Ar[row - pl] = -s.zm;
  if (k < g.nz - 1) Ar[row + pl] = -s.zp;
  Ar[row] = ((s.xm + s.xp) + (s.ym + s.yp)) + (s.zm + s.zp);
}

inline unsigned flat_blocks(size_t n, int threads) {
  size_t b = (n + threads - 1) / threads;
  if (b > 152 * 32) b = 152 * 32;
  if (b == 0) b = 1;
  return (unsigned)b;
}

template <typename A, typename B>
using wider_t = typename std::conditional<std::is_same<A, double>::value || std::is_same<B, double>::value,
                                          double, float>::type;

}  // namespace

template <typename T, typename TX, typename TY>
cudaError_t launch_apply_faces(const Grid3& g, const Faces<T>& F, const TX* x, TY* y, cudaStream_t s) {
  using C = wider_t<wider_t<T, TX>, TY>;
  k_apply_faces<C, T, TX, TY><<<grid_cells(g), dim3(BX, BY), 0, s>>>(g, F, x, y);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_residual_faces(const Grid3& g, const Faces<T>& F, const T* b, const T* x, T* r, T* z, int pc,
                                  cudaStream_t s) {
  k_residual_faces<T><<<grid_cells(g), dim3(BX, BY), 0, s>>>(g, F, b, x, r, z, pc);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sgs_half_faces(const Grid3& g, const Faces<T>& F, const T* r, T* z, int color, T* d, T* x,
                                  double c1, double c2, int flags, cudaStream_t s) {
  dim3 grid((unsigned)(((g.nx + 1) / 2 + BX - 1) / BX), (unsigned)((g.ny + BY - 1) / BY), (unsigned)g.nz);
  k_sgs_half_faces<T><<<grid, dim3(BX, BY), 0, s>>>(g, F, r, z, color, d, x, (T)c1, (T)c2, flags);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_residual_restrict_faces(const Grid3& g, const Faces<T>& F, const T* b, const T* x, T* coarse,
                                           cudaStream_t s) {
  dim3 grid((unsigned)((g.nx / 2 + BX - 1) / BX), (unsigned)((g.ny / 2 + BY - 1) / BY), (unsigned)(g.nz / 2));
  k_residual_restrict_faces<T><<<grid, dim3(BX, BY), 0, s>>>(g, F, b, x, coarse);
  return cudaGetLastError();
}

namespace {
// Grid of 32 x 8 column blocks over an nx x ny x nz box, with z cut into chunks
// for about two waves of 8 blocks per SM (at least 4 planes per chunk).
struct ColumnLaunch {
  dim3 grid;
  int kchunk;
};
ColumnLaunch column_launch(int nx, int ny, int nz) {
  const int gx = (nx + 31) / 32, gy = (ny + 7) / 8;
  const long long target = 152LL * 8 * 2, xy = (long long)gx * gy;
  const int zc = (int)std::max(1LL, std::min((target + xy - 1) / xy, (long long)std::max(1, nz / 4)));
  const int kchunk = (nz + zc - 1) / zc;
  return {dim3((unsigned)gx, (unsigned)gy, (unsigned)((nz + kchunk - 1) / kchunk)), kchunk};
}
}  // namespace

template <typename T>
cudaError_t launch_coarsen_faces(const Grid3& g, const T* a, const Faces<T>& F, T* kx, T* ky, T* kz, T* ktop,
                                 cudaStream_t s) {
  const ColumnLaunch cl = column_launch(g.nx / 2, g.ny / 2, g.nz / 2);
  const dim3 block(32, 8);
  if (a) k_coarsen_faces<T, true><<<cl.grid, block, 0, s>>>(Links<T, true>{g, a, F}, kx, ky, kz, ktop, cl.kchunk);
  else k_coarsen_faces<T, false><<<cl.grid, block, 0, s>>>(Links<T, false>{g, a, F}, kx, ky, kz, ktop, cl.kchunk);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prolong_weights(const Grid3& g, const T* a, const Faces<T>& F, T* w, cudaStream_t s) {
  const ColumnLaunch cl = column_launch(g.nx, g.ny, g.nz);
  const dim3 block(32, 8);
  if (a) k_prolong_weights<T, true><<<cl.grid, block, 0, s>>>(Links<T, true>{g, a, F}, w, cl.kchunk);
  else k_prolong_weights<T, false><<<cl.grid, block, 0, s>>>(Links<T, false>{g, a, F}, w, cl.kchunk);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prolong_opdep(const Grid3& g, const T* e, T* x, const T* w, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) {
    if (pair_aligned(x) && pair_aligned(w) && g.nx % 2 == 0 && cells_fit_int32(g) && g.n() % 2 == 0) {
      const int gx = (g.nx / 2 + PTP - 1) / PTP, gy = (g.ny + PTR - 1) / PTR;
      const int nzc = g.nz / 2;
      // about two waves of 8 blocks per SM, at least 4 coarse planes per block
      const long long target = 152LL * 8 * 2, xy = (long long)gx * gy;
      const int zc = (int)std::max(1LL, std::min((target + xy - 1) / xy, (long long)std::max(1, nzc / 4)));
      const int kchunk = (nzc + zc - 1) / zc;
      const int gz = (nzc + kchunk - 1) / kchunk;
      k_prolong_opdep_pairs<<<dim3((unsigned)gx, (unsigned)gy, (unsigned)gz), dim3(PTP, PTR), 0, s>>>(g, e, x, w,
                                                                                                kchunk);
      return cudaGetLastError();
    }
  }
  k_prolong_opdep<T><<<grid_cells(g), dim3(BX, BY), 0, s>>>(g, e, x, w);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_faces_of_cells(const Grid3& g, const T* a, double* kx, double* ky, double* kz, double* ktop,
                                  cudaStream_t s) {
  k_faces_of_cells<T><<<flat_blocks(g.n(), 256), 256, 0, s>>>(Links<T, true>{g, a, Faces<T>{}}, kx, ky, kz, ktop);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_coarse_assemble_faces(const Grid3& g, const Faces<T>& F, double* A, cudaStream_t s) {
  const int n = (int)g.n();
  k_coarse_assemble_faces<T><<<(n + 127) / 128, 128, 0, s>>>(g, F, A);
  return cudaGetLastError();
}

#define GMG_INST(T)                                                                                                \
  template cudaError_t launch_apply_faces<T, T, T>(const Grid3&, const Faces<T>&, const T*, T*, cudaStream_t);      \
  template cudaError_t launch_residual_faces<T>(const Grid3&, const Faces<T>&, const T*, const T*, T*, T*, int,    \
                                                cudaStream_t);                                                     \
  template cudaError_t launch_sgs_half_faces<T>(const Grid3&, const Faces<T>&, const T*, T*, int, T*, T*, double,  \
                                                double, int, cudaStream_t);                                        \
  template cudaError_t launch_residual_restrict_faces<T>(const Grid3&, const Faces<T>&, const T*, const T*, T*,    \
                                                         cudaStream_t);                                            \
  template cudaError_t launch_coarsen_faces<T>(const Grid3&, const T*, const Faces<T>&, T*, T*, T*, T*,            \
                                               cudaStream_t);                                                      \
  template cudaError_t launch_prolong_weights<T>(const Grid3&, const T*, const Faces<T>&, T*, cudaStream_t);       \
  template cudaError_t launch_prolong_opdep<T>(const Grid3&, const T*, T*, const T*, cudaStream_t);                \
  template cudaError_t launch_faces_of_cells<T>(const Grid3&, const T*, double*, double*, double*, double*,        \
                                                cudaStream_t);                                                     \
  template cudaError_t launch_coarse_assemble_faces<T>(const Grid3&, const Faces<T>&, double*, cudaStream_t);
GMG_INST(float)
GMG_INST(double)
#undef GMG_INST

}  // namespace gmg
