// Host side of libgmg: the C ABI of include/gmg.h.
//
// Set-up (renewed every time step, Sec. 3): coefficient check, 8-child
// coefficient coarsening, Chebyshev eigen bounds per level from a 10-step
// Arnoldi run on B^{-1} A_l (Sec. 3.2), dense Cholesky of the coarsest
// operator (Sec. 3.2).  Solve: FGMRES with right preconditioning (Algorithm
// 1, Sec. 3.1), one V-cycle from zero per iteration (Sec. 3.2, Appendix A),
// stopping on the least-squares residual and then on the true FP64 residual
// (eq. (criterion), Sec. 5.2).  Every vector operation runs in the kernels of
// k_*.cu; the host keeps only the (m+1) x m Hessenberg matrix, its Givens
// rotations and the 10 x 10 eigenvalue problem.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <vector>

#include "../../include/gmg.h"
#include "gmg_internal.cuh"

using namespace gmg;

namespace {

int g_fail_alloc_countdown = 0;

gmg_status map_err(cudaError_t e) {
  if (e == cudaSuccess) return GMG_OK;
  (void)cudaGetLastError();  // clear a non-sticky error so the context stays usable
  return e == cudaErrorMemoryAllocation ? GMG_ERR_ALLOC : GMG_ERR_CUDA;
}

#define CK(...)                                \
  do {                                         \
    cudaError_t e_ = (__VA_ARGS__);            \
    if (e_ != cudaSuccess) return map_err(e_); \
  } while (0)

#define CKS(...)                    \
  do {                              \
    gmg_status s_ = (__VA_ARGS__);  \
    if (s_ != GMG_OK) return s_;    \
  } while (0)

constexpr int MAX_COARSE = 1024;  // unknowns of the dense coarsest grid
constexpr int MAXV = 64;          // Krylov vectors
// device scalar slots
constexpr int SL_H1 = 0, SL_H2 = 64, SL_NORM = 128, SL_Y = 136, SL_CHECK = 200, N_SCAL = 256;
// one eigen-estimate column: h1[0..k), h2[0..k), ||w|| with k <= 32 (eig_steps <= 32)
constexpr int EIG_STRIDE = 65, EIG_MAX_STEPS = 32;

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// ---------------------------------------------------------------------------
// Largest real eigenvalue of a small upper Hessenberg matrix: Francis
// double-shift QR (Golub & Van Loan, Matrix Computations, Sec. 7.5) working
// on the active diagonal block only, since only eigenvalues are wanted.
// ---------------------------------------------------------------------------
int hessenberg_eigs(std::vector<double>& H, int n, std::vector<double>& wr, std::vector<double>& wi) {
  auto h = [&](int r, int c) -> double& { return H[(size_t)r * n + c]; };
  wr.assign(n, 0.0);
  wi.assign(n, 0.0);
  double anorm = 0.0;
  for (int r = 0; r < n; ++r)
    for (int c = std::max(0, r - 1); c < n; ++c) anorm += fabs(h(r, c));
  const double eps = 2.220446049250313e-16;
  int hi = n - 1, iter = 0, total = 0;
  while (hi >= 0) {
    int l = hi;
    while (l > 0) {
      double s = fabs(h(l - 1, l - 1)) + fabs(h(l, l));
      if (s == 0.0) s = anorm;
      if (fabs(h(l, l - 1)) <= eps * s) {
        h(l, l - 1) = 0.0;
        break;
      }
      --l;
    }
    if (l == hi) {
      wr[hi] = h(hi, hi);
      --hi;
      iter = 0;
      continue;
    }
    if (l == hi - 1) {
      const double a = h(hi - 1, hi - 1), b = h(hi - 1, hi), c = h(hi, hi - 1), d = h(hi, hi);
      const double m = 0.5 * (a + d), p = 0.5 * (a - d), disc = p * p + b * c;
      if (disc >= 0.0) {
        const double q = sqrt(disc);
        wr[hi - 1] = m + q;
        wr[hi] = m - q;
      } else {
        wr[hi - 1] = wr[hi] = m;
        wi[hi - 1] = sqrt(-disc);
        wi[hi] = -wi[hi - 1];
      }
      hi -= 2;
      iter = 0;
      continue;
    }
    if (++iter > 60 || ++total > 60 * n) return -1;
    double s, t;
    if (iter % 11 == 10) {  // exceptional shift to break a cycle
      const double w = fabs(h(hi, hi - 1)) + fabs(h(hi - 1, hi - 2));
      s = 1.5 * w;
      t = w * w;
    } else {
      s = h(hi - 1, hi - 1) + h(hi, hi);
      t = h(hi - 1, hi - 1) * h(hi, hi) - h(hi - 1, hi) * h(hi, hi - 1);
    }
    // first column of (H - mu1)(H - mu2) restricted to the active block
    double x = h(l, l) * h(l, l) + h(l, l + 1) * h(l + 1, l) - s * h(l, l) + t;
    double y = h(l + 1, l) * (h(l, l) + h(l + 1, l + 1) - s);
    double z = h(l + 1, l) * h(l + 2, l + 1);
    for (int k = l; k <= hi - 2; ++k) {
      double alpha = sqrt(x * x + y * y + z * z);
      if (x > 0) alpha = -alpha;
      const double u0 = x - alpha, u1 = y, u2 = z;
      const double uu = u0 * u0 + u1 * u1 + u2 * u2;
      if (uu != 0.0) {
        const double beta = 2.0 / uu;
        for (int c = std::max(l, k - 1); c <= hi; ++c) {
          const double dd = beta * (u0 * h(k, c) + u1 * h(k + 1, c) + u2 * h(k + 2, c));
          h(k, c) -= dd * u0;
          h(k + 1, c) -= dd * u1;
          h(k + 2, c) -= dd * u2;
        }
        for (int r = l; r <= std::min(k + 3, hi); ++r) {
          const double dd = beta * (h(r, k) * u0 + h(r, k + 1) * u1 + h(r, k + 2) * u2);
          h(r, k) -= dd * u0;
          h(r, k + 1) -= dd * u1;
          h(r, k + 2) -= dd * u2;
        }
      }
      if (k > l) {
        h(k + 1, k - 1) = 0.0;
        h(k + 2, k - 1) = 0.0;
      }
      x = h(k + 1, k);
      y = h(k + 2, k);
      z = (k < hi - 2) ? h(k + 3, k) : 0.0;
    }
    {
      const int k = hi - 1;
      double alpha = sqrt(x * x + y * y);
      if (x > 0) alpha = -alpha;
      const double u0 = x - alpha, u1 = y;
      const double uu = u0 * u0 + u1 * u1;
      if (uu != 0.0) {
        const double beta = 2.0 / uu;
        for (int c = std::max(l, k - 1); c <= hi; ++c) {
          const double dd = beta * (u0 * h(k, c) + u1 * h(k + 1, c));
          h(k, c) -= dd * u0;
          h(k + 1, c) -= dd * u1;
        }
        for (int r = l; r <= hi; ++r) {
          const double dd = beta * (h(r, k) * u0 + h(r, k + 1) * u1);
          h(r, k) -= dd * u0;
          h(r, k + 1) -= dd * u1;
        }
      }
      if (k > l) h(k + 1, k - 1) = 0.0;
    }
  }
  return 0;
}

}  // namespace

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------

// Kernel classes of the per-kernel profile (launch counts, CUDA-event time and
// algorithmic bytes: each array a kernel must touch, read or written once).
enum KernelClass : int {
  K_APPLY_F64, K_APPLY_OUTER, K_APPLY_F32, K_RESIDUAL_F64, K_RESIDUAL_F32, K_SGS_F64, K_SGS_F32,
  K_CHEB_F64, K_CHEB_F32, K_RESTRICT_F64, K_RESTRICT_F32, K_PROLONG_F64, K_PROLONG_F32, K_COARSE_F64,
  K_COARSE_F32, K_DOT, K_FINALIZE, K_AXPY, K_SCALE, K_UPDATE_X, K_CAST, K_COPY, K_RHS, K_FIELD, K_ADJOINT,
  K_COARSEN, K_COEF_CHECK, K_HASH, K_COARSE_ASSEMBLE, K_COARSE_FACTOR, K_DOT_F32, K_AXPY_F32, K_APPLY_DF64,
  K_SPLIT, K_CHEB_FUSED, K_CGS_DOTS, K_CGS_DOTS_F32, K_CGS_UPDATE, K_CGS_UPDATE_F32, K_LIN3, K_MGS, K_MGS_F32,
  K_SCALE_ROUND, K_COARSEN_FACES, K_PROLONG_WEIGHTS, K_GRAM, K_HOST_GAP, NK
};
static const char* const kKernelNames[NK] = {
    "apply_f64", "apply_outer_f64a_f32x", "apply_f32", "residual_f64", "residual_f32", "sgs_half_f64",
    "sgs_half_f32", "cheb_update_f64", "cheb_update_f32", "residual_restrict_f64", "residual_restrict_f32",
    "prolong_add_f64", "prolong_add_f32", "coarse_apply_f64", "coarse_apply_f32", "multi_dot", "finalize",
    "multi_axpy", "scale", "update_solution", "cast", "copy", "rhs", "field", "adjoint_grad", "coarsen_coef",
    "coef_check", "hash_vector", "coarse_assemble", "coarse_factor", "multi_dot_f32", "multi_axpy_f32",
    "apply_outer_df64", "split_coef", "cheb_sgs_fused_f32", "cgs_dots", "cgs_dots_f32", "cgs_update",
    "cgs_update_f32", "vector_lin3", "mgs_pass", "mgs_pass_f32", "scale_round", "coarsen_faces",
    "prolong_weights", "gram_f32", "host_round_trip"};

struct ProfPending {
  int cls;
  cudaEvent_t a, b;
  double bytes;
};

struct LevelData {
  int nx = 0, ny = 0, nz = 0;
  size_t n = 0;
  Grid3 g{};
  double* a64 = nullptr;
  float* a32 = nullptr;
  float2* a2 = nullptr;  // finest level, mixed + double-float outer product: (hi, lo) split of a64
  DfCoef dc{};
  void *x = nullptr, *b = nullptr, *r = nullptr, *z = nullptr, *d = nullptr;  // level precision
  float* x2 = nullptr;  // second x buffer of the fused smoother (ping-pong), when fused
  bool fused = false;
  // face form (coarse levels of GMG_COARSEN_SERIES): kx | ky | kz (n each) |
  // ktop (nx * ny), level precision; no cell coefficient then
  bool faces = false;
  void* kf = nullptr;
  // parent weights wx | wy | wz (3 n, level precision) of the prolongation into
  // this level (GMG_PROLONG_OPDEP, levels >= 1)
  void* wp = nullptr;
  double lam_max = 0, lam_min = 0, lam_hat = 0;
};

struct gmg_ctx {
  gmg_params p{};
  cudaStream_t s = nullptr;
  bool mixed = false;
  size_t esz = 8;
  std::vector<LevelData> lev;  // 0 = coarsest
  int nc = 0;
  double *cA = nullptr, *cW = nullptr, *cinv64 = nullptr;
  int* cstatus = nullptr;
  int nv = 0;
  double* V = nullptr;
  void* Z = nullptr;
  double* w = nullptr;
  double* bvec = nullptr;
  double* partial = nullptr;
  double* dscal = nullptr;
  double* hpin = nullptr;      // mapped pinned host scalars ...
  double* hpin_dev = nullptr;  // ... and their device address
  double* eigH = nullptr;      // the eigen estimate's Hessenberg columns (device) ...
  double* heig = nullptr;      // ... their mapped pinned host copy ...
  double* heig_dev = nullptr;  // ... and its device address
  int* hstat = nullptr;
  int* hstat_dev = nullptr;
  double *st_a = nullptr, *st_f = nullptr, *st_phi = nullptr;
  void *st_ex = nullptr, *st_ey = nullptr, *st_ez = nullptr;
  int st_fp32 = -1;  // element type of the field staging buffers (-1: none yet)
  bool fmg_now = false;  // the preconditioner of the current solve is full multigrid
  long long precond_calls = 0;  // preconditioner applications (reported per solve)
  // mixed precision: the finest level's FP32 right-hand side already holds the
  // rounding of this FP64 vector (written with it by prof_scale_round)
  const double* b32_of = nullptr;
  // copy stream of gmg_solve_host: input copies overlap the set-up, the
  // potential's copy-out overlaps the field kernel
  cudaStream_t cs = nullptr, cso = nullptr;  // input and copy-out streams
  cudaEvent_t ev_in = nullptr, ev_a = nullptr, ev_out = nullptr, ev_done = nullptr;
  // gmg_solve_host_async's copy-out of phi (and E), left for the next call to
  // enqueue once its upload of a is done, or for gmg_host_wait
  struct PendingOut {
    bool on = false;
    double* phi = nullptr;
    void *ex = nullptr, *ey = nullptr, *ez = nullptr;
    size_t bytes = 0, ebytes = 0;
  } pend_out;
  float setup_ms = 0.f;
  // per-kernel profile
  bool prof_on = false;
  double prof_min_bytes = 0.0;  // launches below this are counted, not timed
  std::vector<cudaEvent_t> ev_pool;
  std::vector<ProfPending> pend;
  double k_ms[NK] = {};
  double k_bytes[NK] = {};
  long long k_launch[NK] = {};
  long long k_timed[NK] = {};
  std::vector<void*> dev_allocs;
  std::vector<void*> host_allocs;

  size_t N() const { return lev.back().n; }
  const LevelData& fine() const { return lev.back(); }
};

namespace {

gmg_status dev_alloc(gmg_ctx* c, void** p, size_t bytes) {
  *p = nullptr;
  if (g_fail_alloc_countdown > 0 && --g_fail_alloc_countdown == 0) return GMG_ERR_ALLOC;
  cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
  if (e != cudaSuccess) {
    *p = nullptr;
    return map_err(e);
  }
  c->dev_allocs.push_back(*p);
  return GMG_OK;
}

template <typename P>
gmg_status dalloc(gmg_ctx* c, P** p, size_t count, size_t elem = sizeof(P)) {
  void* v = nullptr;
  gmg_status st = dev_alloc(c, &v, count * elem);
  *p = (P*)v;
  return st;
}

// ---- per-kernel profile ----
cudaEvent_t prof_event(gmg_ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Fold finished launches into the totals; the stream must be synchronised.
void prof_collect(gmg_ctx* c) {
  for (const ProfPending& q : c->pend) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, q.a, q.b) == cudaSuccess) {
      c->k_ms[q.cls] += ms;
      c->k_bytes[q.cls] += q.bytes;
      c->k_timed[q.cls] += 1;
    }
    c->ev_pool.push_back(q.a);
    c->ev_pool.push_back(q.b);
  }
  c->pend.clear();
}

template <typename F>
gmg_status run_kernel(gmg_ctx* c, int cls, double bytes, F&& launch) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c->prof_on && bytes >= c->prof_min_bytes && (e0 = prof_event(c)) != nullptr) cudaEventRecord(e0, c->s);
  const cudaError_t e = launch();
  c->k_launch[cls] += 1;
  if (e != cudaSuccess) {
    if (e0) c->ev_pool.push_back(e0);
    return map_err(e);
  }
  if (e0) {
    if ((e1 = prof_event(c)) != nullptr && cudaEventRecord(e1, c->s) == cudaSuccess)
      c->pend.push_back({cls, e0, e1, bytes});
    else
      c->ev_pool.push_back(e0);
  }
  return GMG_OK;
}

template <typename T>
constexpr bool is_f32() { return sizeof(T) == 4; }

#define GMG_RUN(cls, bytes, ...) return run_kernel(c, (cls), (double)(bytes), [&]() { return __VA_ARGS__; })

template <typename TA, typename TX, typename TY>
gmg_status prof_apply(gmg_ctx* c, const Grid3& g, const TA* a, const TX* x, TY* y, cudaStream_t s) {
  const int cls = is_f32<TA>() ? K_APPLY_F32 : (is_f32<TX>() ? K_APPLY_OUTER : K_APPLY_F64);
  GMG_RUN(cls, g.n() * (sizeof(TA) + sizeof(TX) + sizeof(TY)), launch_apply<TA, TX, TY>(g, a, x, y, s));
}
template <typename T>
gmg_status prof_residual(gmg_ctx* c, const Grid3& g, const T* a, const T* b, const T* x, T* r, T* z, int pc,
                         cudaStream_t s) {
  const double n = (double)g.n(), e = sizeof(T);
  const double zw = pc == PC_SGS ? 0.5 * n : (pc == PC_NONE ? 0.0 : n);
  const double bytes = n * e * (2 + (x ? 1 : 0) + (r ? 1 : 0)) + zw * e;
  GMG_RUN(is_f32<T>() ? K_RESIDUAL_F32 : K_RESIDUAL_F64, bytes, launch_residual<T>(g, a, b, x, r, z, pc, s));
}
template <typename T>
gmg_status prof_sgs_half(gmg_ctx* c, const Grid3& g, const T* a, const T* r, T* z, int color, T* d, T* x,
                         double c1, double c2, int flags, cudaStream_t s) {
  const double n = (double)g.n(), e = sizeof(T), h = 0.5 * n;
  double bytes = n * e + h * e * 3;
  if (flags & CHEB_UPDATE) bytes += h * e * (((flags & CHEB_FIRST) ? 1 : 2) + ((flags & CHEB_XZERO) ? 1 : 2));
  GMG_RUN(is_f32<T>() ? K_SGS_F32 : K_SGS_F64, bytes, launch_sgs_half<T>(g, a, r, z, color, d, x, c1, c2, flags, s));
}
template <typename T>
gmg_status prof_cheb_update(gmg_ctx* c, size_t n, const T* z, T* d, T* x, double c1, double c2, int flags,
                            cudaStream_t s) {
  const double bytes = (double)n * sizeof(T) * (1 + ((flags & CHEB_FIRST) ? 1 : 2) + ((flags & CHEB_XZERO) ? 1 : 2));
  GMG_RUN(is_f32<T>() ? K_CHEB_F32 : K_CHEB_F64, bytes, launch_cheb_update<T>(n, z, d, x, c1, c2, flags, s));
}
template <typename T>
gmg_status prof_residual_restrict(gmg_ctx* c, const Grid3& g, const T* a, const T* b, const T* x, T* coarse,
                                  cudaStream_t s) {
  GMG_RUN(is_f32<T>() ? K_RESTRICT_F32 : K_RESTRICT_F64, (double)g.n() * sizeof(T) * (3.0 + 0.125),
          launch_residual_restrict<T>(g, a, b, x, coarse, s));
}
template <typename T>
gmg_status prof_prolong_add(gmg_ctx* c, const Grid3& g, const T* e, T* x, int mode, cudaStream_t s) {
  GMG_RUN(is_f32<T>() ? K_PROLONG_F32 : K_PROLONG_F64, (double)g.n() * sizeof(T) * (2.0 + 0.125),
          launch_prolong_add<T>(g, e, x, mode, s));
}
template <typename T>
gmg_status prof_coarse_apply(gmg_ctx* c, int n, const double* Ainv, const T* b, T* x, cudaStream_t s) {
  GMG_RUN(is_f32<T>() ? K_COARSE_F32 : K_COARSE_F64, (double)n * n * 8.0 + 2.0 * n * sizeof(T),
          launch_coarse_apply<T>(n, Ainv, b, x, s));
}
template <typename T>
gmg_status prof_multi_dot(gmg_ctx* c, size_t n, const T* w, const T* V, size_t ldv, int k, double* partial,
                          cudaStream_t s) {
  const double bytes = (V == w && ldv == 0) ? (double)sizeof(T) * n : (double)sizeof(T) * n * (1 + k);
  GMG_RUN(is_f32<T>() ? K_DOT_F32 : K_DOT, bytes, launch_multi_dot<T>(n, w, V, ldv, k, partial, s));
}
gmg_status prof_finalize(gmg_ctx* c, const double* partial, int nblocks, int k, double* out, int acc, cudaStream_t s) {
  GMG_RUN(K_FINALIZE, 8.0 * nblocks * k, launch_finalize(partial, nblocks, k, out, acc, s));
}
gmg_status prof_finalize_norm(gmg_ctx* c, const double* partial, int nblocks, double* out, cudaStream_t s) {
  GMG_RUN(K_FINALIZE, 8.0 * nblocks, launch_finalize_norm(partial, nblocks, out, s));
}
gmg_status prof_finalize_check(gmg_ctx* c, const double* partial, int nblocks, double* out, cudaStream_t s) {
  GMG_RUN(K_FINALIZE, 16.0 * nblocks, launch_finalize_check(partial, nblocks, out, s));
}
template <typename T>
gmg_status prof_cgs_dots(gmg_ctx* c, size_t n, const T* w, const T* V, size_t ldv, int k, const double* h,
                         double* partial, cudaStream_t s) {
  GMG_RUN(is_f32<T>() ? K_CGS_DOTS_F32 : K_CGS_DOTS, (double)sizeof(T) * n * (1 + k),
          launch_cgs_dots<T>(n, w, V, ldv, k, h, partial, s));
}
template <typename T>
gmg_status prof_cgs_update(gmg_ctx* c, size_t n, T* w, const T* V, size_t ldv, int k, const double* h1,
                           const double* h2, double* partial, cudaStream_t s) {
  GMG_RUN(is_f32<T>() ? K_CGS_UPDATE_F32 : K_CGS_UPDATE, (double)sizeof(T) * n * (2 + k),
          launch_cgs_update<T>(n, w, V, ldv, k, h1, h2, partial, s));
}
template <typename T>
gmg_status prof_multi_axpy(gmg_ctx* c, size_t n, T* w, const T* V, size_t ldv, int k, const double* h,
                           cudaStream_t s) {
  GMG_RUN(is_f32<T>() ? K_AXPY_F32 : K_AXPY, (double)sizeof(T) * n * (k + 2),
          launch_multi_axpy<T>(n, w, V, ldv, k, h, s));
}
template <typename T>
gmg_status prof_scale(gmg_ctx* c, size_t n, const T* src, T* dst, const double* sc, cudaStream_t s) {
  GMG_RUN(K_SCALE, 2.0 * sizeof(T) * n, launch_scale<T>(n, src, dst, sc, s));
}
gmg_status prof_scale_value(gmg_ctx* c, size_t n, const double* src, double* dst, double alpha, cudaStream_t s) {
  GMG_RUN(K_SCALE, 16.0 * n, launch_scale_value(n, src, dst, alpha, s));
}
gmg_status prof_scale_round(gmg_ctx* c, size_t n, const double* src, double* dst, float* dst32, const double* sc,
                            double alpha, cudaStream_t s) {
  GMG_RUN(K_SCALE_ROUND, 20.0 * n, launch_scale_round(n, src, dst, dst32, sc, alpha, s));
}
template <typename TZ>
gmg_status prof_update_solution(gmg_ctx* c, size_t n, double* x, const TZ* Z, size_t ldz, int k, const double* y,
                                cudaStream_t s) {
  GMG_RUN(K_UPDATE_X, (double)n * (16.0 + k * sizeof(TZ)), launch_update_solution<TZ>(n, x, Z, ldz, k, y, s));
}
template <typename T>
gmg_status prof_mgs_step(gmg_ctx* c, size_t n, T* w, const T* vi, const T* vnext, const double* hi, double* partial) {
  const double bytes = (double)sizeof(T) * n * (1.0 + (vi ? 2.0 : 0.0) + (vnext ? 1.0 : 0.0));
  cudaStream_t s = c->s;
  GMG_RUN(is_f32<T>() ? K_MGS_F32 : K_MGS, bytes, launch_mgs_step<T>(n, w, vi, vnext, hi, partial, s));
}
template <typename T1, typename T2>
gmg_status prof_lin3(gmg_ctx* c, size_t n, double a1, const T1* v1, double a2, const T2* v2, double a3,
                     const double* v3, double* out) {
  const double bytes = (double)n * (8.0 + (v1 ? sizeof(T1) : 0) + (v2 ? sizeof(T2) : 0) + (v3 ? 8.0 : 0.0));
  cudaStream_t s = c->s;
  GMG_RUN(K_LIN3, bytes, launch_lin3<T1, T2>(n, a1, v1, a2, v2, a3, v3, out, s));
}
gmg_status prof_cast_d2f(gmg_ctx* c, size_t n, const double* src, float* dst, cudaStream_t s) {
  GMG_RUN(K_CAST, 12.0 * n, launch_cast_d2f(n, src, dst, s));
}
gmg_status prof_cast_f2d(gmg_ctx* c, size_t n, const float* src, double* dst, cudaStream_t s) {
  GMG_RUN(K_CAST, 12.0 * n, launch_cast_f2d(n, src, dst, s));
}
gmg_status prof_copy_d(gmg_ctx* c, size_t n, const double* src, double* dst, cudaStream_t s) {
  GMG_RUN(K_COPY, 16.0 * n, launch_copy_d(n, src, dst, s));
}
gmg_status prof_rhs(gmg_ctx* c, const Grid3& g, const double* a, const double* f, double* b, double gb, double gt,
                    int homogeneous, cudaStream_t s) {
  GMG_RUN(K_RHS, 16.0 * g.n() + 16.0 * g.plane(), launch_rhs(g, a, f, b, gb, gt, homogeneous, s));
}
gmg_status prof_field(gmg_ctx* c, const Grid3& g, double hx, double hy, double hz, const double* phi, void* ex,
                      void* ey, void* ez, int fp32, double gb, double gt, cudaStream_t s) {
  GMG_RUN(K_FIELD, (double)g.n() * (8.0 + 3.0 * (fp32 ? 4 : 8)),
          launch_field(g, hx, hy, hz, phi, ex, ey, ez, fp32, gb, gt, s));
}
gmg_status prof_adjoint_grad(gmg_ctx* c, const Grid3& g, const double* phi, const double* lam, double* out,
                             double gb, double gt, cudaStream_t s) {
  GMG_RUN(K_ADJOINT, 24.0 * g.n(), launch_adjoint_grad(g, phi, lam, out, gb, gt, s));
}
template <typename T>
gmg_status prof_hash_vector(gmg_ctx* c, size_t n, T* u, cudaStream_t s) {
  GMG_RUN(K_HASH, (double)sizeof(T) * n, launch_hash_vector(n, u, s));
}
gmg_status prof_coef_check(gmg_ctx* c, size_t n, const double* a, double* partial, cudaStream_t s) {
  GMG_RUN(K_COEF_CHECK, 8.0 * n, launch_coef_check(n, a, partial, s));
}
gmg_status prof_coarsen_coef(gmg_ctx* c, const Grid3& g, const double* a, double* ac, float* ac32, cudaStream_t s) {
  GMG_RUN(K_COARSEN, 8.0 * g.n() + g.n() / 8.0 * (8.0 + (ac32 ? 4.0 : 0.0)), launch_coarsen_coef(g, a, ac, ac32, s));
}
gmg_status prof_coarse_assemble(gmg_ctx* c, const Grid3& g, const double* a, double* A, cudaStream_t s) {
  GMG_RUN(K_COARSE_ASSEMBLE, 8.0 * g.n() * g.n(), launch_coarse_assemble(g, a, A, s));
}
gmg_status prof_coarse_factor(gmg_ctx* c, int n, double* A, double* work, double* Ainv, float* Ainv32, int* st,
                              cudaStream_t s) {
  GMG_RUN(K_COARSE_FACTOR, 36.0 * n * n, launch_coarse_factor(n, A, work, Ainv, Ainv32, st, s));
}
gmg_status prof_apply_df64(gmg_ctx* c, const Grid3& g, const DfCoef& dc, const float2* a2, const float* z, double* w,
                           cudaStream_t s) {
  GMG_RUN(K_APPLY_DF64, 20.0 * g.n(), launch_apply_df64(g, dc, a2, z, w, s));
}
// Words per cell a fused step moves: a, b (not for the eigen-estimate basis
// step), x_in (if any), d (unless the first step), x_out, d (unless the last
// step or the basis step).
double fused_words(bool xin, int flags) {
  const bool eig = (flags & CHEB_EIG) != 0;
  return 1.0 + (eig ? 0.0 : 1.0) + (xin ? 1.0 : 0.0) + ((flags & CHEB_FIRST) ? 0.0 : 1.0) + 1.0 +
         ((flags & CHEB_LAST) || eig ? 0.0 : 1.0);
}
gmg_status prof_cheb_sgs_fused(gmg_ctx* c, const Grid3& g, const float* a, const float* b, const float* xin,
                               float* xout, float* d, double c1, double c2, double ce, int flags, cudaStream_t s) {
  const double words = fused_words(xin != nullptr, flags);
  int* tma_status = c->p.smoother_kernel == 0 ? c->cstatus + 1 : nullptr;
  GMG_RUN(K_CHEB_FUSED, 4.0 * words * g.n(),
          launch_cheb_sgs_fused(g, a, b, xin, xout, d, c1, c2, ce, flags, tma_status, s));
}
gmg_status prof_gram(gmg_ctx* c, size_t n, const float* V, size_t ldv, int nv, double* partial, cudaStream_t s) {
  GMG_RUN(K_GRAM, 4.0 * n * nv, launch_gram(n, V, ldv, nv, partial, s));
}
template <typename T>
gmg_status prof_three_term(gmg_ctx* c, size_t n, const T* t, const T* v, const T* u, T* out, double alpha,
                           double beta, double gamma, cudaStream_t s) {
  GMG_RUN(K_LIN3, (double)sizeof(T) * n * (u ? 4 : 3), launch_three_term<T>(n, t, v, u, out, alpha, beta, gamma, s));
}
gmg_status prof_split(gmg_ctx* c, size_t n, const double* a, float2* a2, cudaStream_t s) {
  GMG_RUN(K_SPLIT, 16.0 * n, launch_split(n, a, a2, s));
}
#undef GMG_RUN

gmg_status validate(const gmg_params* p, int* nlevels) {
  if (!p) return GMG_ERR_ARG;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return GMG_ERR_ARG;
  if (!(p->lx > 0 && p->ly > 0 && p->lz > 0) || !isfinite(p->lx) || !isfinite(p->ly) || !isfinite(p->lz))
    return GMG_ERR_ARG;
  if (!isfinite(p->phi_bottom) || !isfinite(p->phi_top)) return GMG_ERR_ARG;
  if (p->coarse_min < 1 || p->cheb_steps < 1 || p->cheb_steps > 8) return GMG_ERR_ARG;
  if (p->restart < 1 || p->restart > MAXV - 1 || p->max_iters < 1) return GMG_ERR_ARG;
  if (!(p->rtol > 0) || !isfinite(p->rtol)) return GMG_ERR_ARG;
  if (p->eig_steps < 1 || p->eig_steps > EIG_MAX_STEPS) return GMG_ERR_ARG;
  if (!(p->eig_hi > p->eig_lo) || !(p->eig_lo > 0) || !isfinite(p->eig_hi)) return GMG_ERR_ARG;
  if (p->precision != GMG_PREC_FP64 && p->precision != GMG_PREC_MIXED) return GMG_ERR_ARG;
  if (p->prolongation < GMG_PROLONG_TRILINEAR || p->prolongation > GMG_PROLONG_OPDEP) return GMG_ERR_ARG;
  if (p->coarsening != GMG_COARSEN_MEAN && p->coarsening != GMG_COARSEN_SERIES) return GMG_ERR_ARG;
  if (p->smoother_pc < 0 || p->smoother_pc > 2) return GMG_ERR_ARG;
  if (p->orthogonalization != 0 && p->orthogonalization != 1) return GMG_ERR_ARG;
  if (p->outer_arith != GMG_OUTER_FP64 && p->outer_arith != GMG_OUTER_DOUBLE_FLOAT) return GMG_ERR_ARG;
  if (p->smoother_kernel < 0 || p->smoother_kernel > 2) return GMG_ERR_ARG;
  if (p->cycle < GMG_CYCLE_V || p->cycle > GMG_CYCLE_AUTO) return GMG_ERR_ARG;
  if ((double)p->nx * p->ny * p->nz > 4.0e9) return GMG_ERR_ARG;
  int nx = p->nx, ny = p->ny, nz = p->nz, L = 1;
  while (std::min(nx, std::min(ny, nz)) > p->coarse_min) {
    if ((nx | ny | nz) & 1) return GMG_ERR_ARG;
    nx /= 2;
    ny /= 2;
    nz /= 2;
    ++L;
  }
  if (std::min(nx, std::min(ny, nz)) != p->coarse_min) return GMG_ERR_ARG;
  if ((long long)nx * ny * nz > MAX_COARSE) return GMG_ERR_ARG;
  *nlevels = L;
  return GMG_OK;
}

// Read `count` device scalars from slot `slot` into ctx->hpin[slot...]; synchronises.
// With gap_start non-null (profiling on), an event is recorded on the stream
// just before the synchronisation: it completes when the GPU has finished the
// work the host waits for, and the interval from it to the next event the
// host records (host_gap_end) is the time the GPU waits for the host.
gmg_status read_scalars(gmg_ctx* c, int slot, int count, cudaEvent_t* gap_start = nullptr) {
  CK(launch_words_to_host(c->dscal + slot, c->hpin_dev + slot, sizeof(double) * count, c->s));
  if (gap_start && c->prof_on && (*gap_start = prof_event(c)) != nullptr) cudaEventRecord(*gap_start, c->s);
  CK(cudaStreamSynchronize(c->s));
  prof_collect(c);
  return GMG_OK;
}

// Close a host round trip opened by read_scalars: the GPU sat idle from
// gap_start until this event, enqueued once the host has done its part.
void host_gap_end(gmg_ctx* c, cudaEvent_t gap_start) {
  if (!gap_start) return;
  cudaEvent_t e1 = prof_event(c);
  if (e1 && cudaEventRecord(e1, c->s) == cudaSuccess) {
    c->pend.push_back({K_HOST_GAP, gap_start, e1, 0.0});
    c->k_launch[K_HOST_GAP] += 1;
  } else {
    c->ev_pool.push_back(gap_start);
    if (e1) c->ev_pool.push_back(e1);
  }
}

// Device: out slots [slot, slot+2) = (||w||, 1/||w||).
template <typename T>
gmg_status norm_dev(gmg_ctx* c, size_t n, const T* w, int slot) {
  CKS(prof_multi_dot<T>(c, n, w, w, 0, 1, c->partial, c->s));
  CKS(prof_finalize_norm(c, c->partial, reduce_blocks(n), c->dscal + slot, c->s));
  return GMG_OK;
}

// Orthogonalise w against the k vectors V[0..k) (row stride ld), leaving the
// coefficients in slots SL_H1 (+ SL_H2 for the second CGS pass) and the norm
// of the result and its reciprocal in SL_NORM.
template <typename T>
gmg_status orthogonalize(gmg_ctx* c, size_t n, const T* V, size_t ld, int k, T* w, bool one_pass = false) {
  const int nb = reduce_blocks(n);
  if (c->p.orthogonalization == GMG_ORTH_MGS && !one_pass) {
    // Algorithm 1's modified Gram-Schmidt, one fused pass per basis vector:
    // pass i applies h_{i} v_i to w and forms (w, v_{i+1}); the last forms ||w||.
    CKS(prof_mgs_step<T>(c, n, w, (const T*)nullptr, V, nullptr, c->partial));
    CKS(prof_finalize(c, c->partial, nb, 1, c->dscal + SL_H1, 0, c->s));
    for (int i = 0; i < k; ++i) {
      const T* vnext = i + 1 < k ? V + (size_t)(i + 1) * ld : nullptr;
      CKS(prof_mgs_step<T>(c, n, w, V + (size_t)i * ld, vnext, c->dscal + SL_H1 + i, c->partial));
      if (vnext)
        CKS(prof_finalize(c, c->partial, nb, 1, c->dscal + SL_H1 + i + 1, 0, c->s));
      else
        CKS(prof_finalize_norm(c, c->partial, nb, c->dscal + SL_NORM, c->s));
    }
    return GMG_OK;
  } else if (k <= kCgsMaxVectors) {
    // three fused passes: h1 = V^T w; h2 = V^T (w - V h1); w -= V (h1 + h2) with ||w||^2
    // (one_pass: h2 = 0, two passes)
    CKS(prof_cgs_dots<T>(c, n, w, V, ld, k, nullptr, c->partial, c->s));
    CKS(prof_finalize(c, c->partial, nb, k, c->dscal + SL_H1, 0, c->s));
    if (one_pass) {
      CK(cudaMemsetAsync(c->dscal + SL_H2, 0, sizeof(double) * k, c->s));
    } else {
      CKS(prof_cgs_dots<T>(c, n, w, V, ld, k, c->dscal + SL_H1, c->partial, c->s));
      CKS(prof_finalize(c, c->partial, nb, k, c->dscal + SL_H2, 0, c->s));
    }
    CKS(prof_cgs_update<T>(c, n, w, V, ld, k, c->dscal + SL_H1, c->dscal + SL_H2, c->partial, c->s));
    CKS(prof_finalize_norm(c, c->partial, nb, c->dscal + SL_NORM, c->s));
    return GMG_OK;
  } else {
    if (one_pass) CK(cudaMemsetAsync(c->dscal + SL_H2, 0, sizeof(double) * k, c->s));
    for (int pass = 0; pass < (one_pass ? 1 : 2); ++pass) {
      double* hslot = c->dscal + (pass == 0 ? SL_H1 : SL_H2);
      for (int c0 = 0; c0 < k; c0 += 8) {
        const int kc = std::min(8, k - c0);
        CKS(prof_multi_dot<T>(c, n, w, V + (size_t)c0 * ld, ld, kc, c->partial, c->s));
        CKS(prof_finalize(c, c->partial, nb, kc, hslot + c0, 0, c->s));
      }
      CKS(prof_multi_axpy<T>(c, n, w, V, ld, k, hslot, c->s));
    }
  }
  return norm_dev<T>(c, n, w, SL_NORM);
}

// Column of H after orthogonalize (host copy): h[0..k) and h[k] = ||w||.
void gather_column(gmg_ctx* c, int k, double* h) {
  for (int i = 0; i < k; ++i) {
    h[i] = c->hpin[SL_H1 + i];
    if (c->p.orthogonalization == GMG_ORTH_CGS2) h[i] += c->hpin[SL_H2 + i];
  }
  h[k] = c->hpin[SL_NORM];
}

gmg_status read_column(gmg_ctx* c, int k, double* h, cudaEvent_t* gap_start = nullptr) {
  CKS(read_scalars(c, 0, SL_NORM + 2, gap_start));
  gather_column(c, k, h);
  return GMG_OK;
}

template <typename T>
const T* level_a(const LevelData& L);
template <>
const float* level_a<float>(const LevelData& L) { return L.a32; }
template <>
const double* level_a<double>(const LevelData& L) { return L.a64; }

template <typename T>
Faces<T> level_faces(const LevelData& L) {
  const T* k = (const T*)L.kf;
  Faces<T> F;
  F.kx = k;
  F.ky = k + L.n;
  F.kz = k + 2 * L.n;
  F.ktop = k + 3 * L.n;
  return F;
}

// Level kernels in level precision T, on the level's cell coefficient or faces.
template <typename T>
gmg_status lv_apply(gmg_ctx* c, const LevelData& L, const T* x, T* y) {
  if (!L.faces) return prof_apply<T, T, T>(c, L.g, level_a<T>(L), x, y, c->s);
  const double bytes = ((double)L.n * 5.0 + (double)L.g.plane()) * sizeof(T);
  return run_kernel(c, is_f32<T>() ? K_APPLY_F32 : K_APPLY_F64, bytes,
                    [&]() { return launch_apply_faces<T, T, T>(L.g, level_faces<T>(L), x, y, c->s); });
}
template <typename T>
gmg_status lv_residual(gmg_ctx* c, const LevelData& L, const T* b, const T* x, T* r, T* z, int pc) {
  if (!L.faces) return prof_residual<T>(c, L.g, level_a<T>(L), b, x, r, z, pc, c->s);
  const double n = (double)L.n, e = sizeof(T);
  const double zw = pc == PC_SGS ? 0.5 * n : (pc == PC_NONE ? 0.0 : n);
  const double bytes = n * e * (4 + (x ? 1 : 0) + (r ? 1 : 0)) + zw * e;
  return run_kernel(c, is_f32<T>() ? K_RESIDUAL_F32 : K_RESIDUAL_F64, bytes,
                    [&]() { return launch_residual_faces<T>(L.g, level_faces<T>(L), b, x, r, z, pc, c->s); });
}
template <typename T>
gmg_status lv_sgs_half(gmg_ctx* c, const LevelData& L, const T* r, T* z, int color, T* d, T* x, double c1, double c2,
                       int flags) {
  if (!L.faces) return prof_sgs_half<T>(c, L.g, level_a<T>(L), r, z, color, d, x, c1, c2, flags, c->s);
  const double n = (double)L.n, e = sizeof(T), h = 0.5 * n;
  double bytes = 3.0 * n * e + h * e * 3;
  if (flags & CHEB_UPDATE) bytes += h * e * (((flags & CHEB_FIRST) ? 1 : 2) + ((flags & CHEB_XZERO) ? 1 : 2));
  return run_kernel(c, is_f32<T>() ? K_SGS_F32 : K_SGS_F64, bytes, [&]() {
    return launch_sgs_half_faces<T>(L.g, level_faces<T>(L), r, z, color, d, x, c1, c2, flags, c->s);
  });
}
template <typename T>
gmg_status lv_residual_restrict(gmg_ctx* c, const LevelData& L, const T* b, const T* x, T* coarse) {
  if (!L.faces || !x) return prof_residual_restrict<T>(c, L.g, level_a<T>(L), b, x, coarse, c->s);
  return run_kernel(c, is_f32<T>() ? K_RESTRICT_F32 : K_RESTRICT_F64, (double)L.n * sizeof(T) * (5.0 + 0.125), [&]() {
    return launch_residual_restrict_faces<T>(L.g, level_faces<T>(L), b, x, coarse, c->s);
  });
}
// One fused Chebyshev + SSOR step on an FP32 level (cell or face form).
gmg_status lv_cheb_fused(gmg_ctx* c, const LevelData& L, const float* b, const float* xin, float* xout,
                         double c1, double c2, int flags, double ce = 0.0) {
  if (!L.faces) return prof_cheb_sgs_fused(c, L.g, L.a32, b, xin, xout, (float*)L.d, c1, c2, ce, flags, c->s);
  const double words = fused_words(xin != nullptr, flags) + 2.0;  // three face arrays instead of a
  return run_kernel(c, K_CHEB_FUSED, 4.0 * words * L.n, [&]() {
    return launch_cheb_sgs_fused_faces(L.g, level_faces<float>(L), b, xin, xout, (float*)L.d, c1, c2, ce, flags,
                                       c->s);
  });
}

// x += P e into level L (e on the level below).
template <typename T>
gmg_status lv_prolong(gmg_ctx* c, const LevelData& L, const T* e, T* x) {
  if (c->p.prolongation != GMG_PROLONG_OPDEP) return prof_prolong_add<T>(c, L.g, e, x, c->p.prolongation, c->s);
  return run_kernel(c, is_f32<T>() ? K_PROLONG_F32 : K_PROLONG_F64, (double)L.n * sizeof(T) * (5.0 + 0.125),
                    [&]() { return launch_prolong_opdep<T>(L.g, e, x, (const T*)L.wp, c->s); });
}

// z = B^{-1} r on a level in precision T (the smoother's preconditioner).
template <typename T>
gmg_status smoother_pc(gmg_ctx* c, const LevelData& L, const T* r, T* z) {
  const int pc = c->p.smoother_pc;
  if (pc == GMG_PC_IDENTITY) return map_err(cudaMemcpyAsync(z, r, L.n * sizeof(T), cudaMemcpyDeviceToDevice, c->s));
  CKS(lv_residual<T>(c, L, r, (const T*)nullptr, (T*)nullptr, z, pc == GMG_PC_SGS ? PC_SGS : PC_JACOBI));
  if (pc == GMG_PC_SGS) {
    CKS(lv_sgs_half<T>(c, L, r, z, 1, (T*)nullptr, (T*)nullptr, 0, 0, 0));
    CKS(lv_sgs_half<T>(c, L, r, z, 0, (T*)nullptr, (T*)nullptr, 0, 0, 0));
  }
  return GMG_OK;
}

// Largest real Ritz value of the Krylov space of the eigen estimate, FP32
// levels with the SSOR preconditioner.  Arnoldi (Sec. 3.2) projects
// M = B^{-1} A_l on K_m(M, v_0) with an orthonormal basis; any basis of the
// same nested spaces gives the same projection up to a similarity, so the
// same Ritz values.  For symmetric Gauss-Seidel B - A_l = L D^{-1} L^T is
// positive semi-definite, so M has its spectrum in (0, 1], and the Chebyshev
// basis of 2M - I on it,
//   v_1 = (2M - I) v_0,  v_{j+1} = 2 (2M - I) v_j - v_{j-1},
// stays well conditioned.  Each basis vector is one fused smoother pass; one
// pass over v_0 .. v_m then forms the Gram matrix G = K^T K.  With G_m = R^T R
// (Cholesky), K_m R^{-1} is Arnoldi's orthonormal basis, and
// H_m = R^{-T} (K_m^T M K_m) R^{-1} its Hessenberg matrix, where
// M v_0 = (v_1 + v_0)/2 and M v_j = (v_{j+1} + 2 v_j + v_{j-1})/4 make
// K_m^T M K_m a combination of columns of G.  This replaces Gram-Schmidt's
// passes over all previous vectors at every step (about m^2 vector passes)
// by m + 1.  A Cholesky pivot below kGramPivotTol of its diagonal entry is
// what FP32 vectors cannot resolve: the space ends there (Arnoldi's
// breakdown) and the projection keeps the vectors before it.
constexpr double kGramPivotTol = 1e-6;

gmg_status ritz_chebyshev_basis(gmg_ctx* c, int l, double* lam_out) {
  LevelData& L = c->lev[l];
  const size_t n = L.n;
  const int m = c->p.eig_steps;
  float* V = (float*)c->Z;  // (m + 1) vectors of n, stride n
  // v_0: the hash start vector as it is (entries in [-1, 1)); the projection
  // does not depend on the basis' scale, so it is not normalised
  CKS(prof_hash_vector<float>(c, n, V, c->s));
  for (int j = 0; j < m; ++j) {
    // v_{j+1} = alpha M v_j + beta v_j + gamma v_{j-1}
    const double alpha = j == 0 ? 2.0 : 4.0, beta = j == 0 ? -1.0 : -2.0, gamma = j == 0 ? 0.0 : -1.0;
    const float* vj = V + (size_t)j * n;
    float* vprev = j == 0 ? nullptr : V + (size_t)(j - 1) * n;
    float* vnext = V + (size_t)(j + 1) * n;
    if (L.fused) {
      // the basis step reads v_{j-1} through d (never written) and forms
      // x_out = beta x_in + gamma d - (-alpha) B^{-1} A x_in with b = 0; for
      // j = 0, d = v_0 with gamma = 0 (the kind that reads d runs faster than
      // the one that does not: 0.88 against 0.99 ms at 512^3)
      LevelData Lt = L;
      Lt.d = j == 0 ? (float*)vj : vprev;
      CKS(lv_cheb_fused(c, Lt, (const float*)L.b, vj, vnext, gamma, -alpha, CHEB_UPDATE | CHEB_EIG, beta));
    } else {
      CKS(lv_apply<float>(c, L, vj, (float*)L.r));
      CKS(smoother_pc<float>(c, L, (const float*)L.r, (float*)L.z));
      CKS(prof_three_term<float>(c, n, (const float*)L.z, vj, vprev, vnext, alpha, beta, gamma, c->s));
    }
  }
  const int nv = m + 1, np = nv * (nv + 1) / 2;
  CKS(prof_gram(c, n, V, n, nv, c->partial, c->s));
  CKS(prof_finalize(c, c->partial, reduce_blocks(n), np, c->eigH, 0, c->s));
  CK(launch_words_to_host(c->eigH, c->heig_dev, sizeof(double) * (size_t)np, c->s));
  CK(cudaStreamSynchronize(c->s));
  prof_collect(c);
  std::vector<double> G((size_t)nv * nv);
  for (int i = 0, q = 0; i < nv; ++i)
    for (int j = i; j < nv; ++j, ++q) {
      const double gij = c->heig[q];
      if (!isfinite(gij)) return GMG_ERR_NONFINITE;
      G[(size_t)i * nv + j] = G[(size_t)j * nv + i] = gij;
    }
  // G_k = R^T R, R upper triangular (stride m)
  std::vector<double> R((size_t)m * m, 0.0);
  int k = m;
  for (int j = 0; j < m; ++j) {
    for (int i = 0; i < j; ++i) {
      double t = G[(size_t)i * nv + j];
      for (int p = 0; p < i; ++p) t -= R[(size_t)p * m + i] * R[(size_t)p * m + j];
      R[(size_t)i * m + j] = t / R[(size_t)i * m + i];
    }
    double dd = G[(size_t)j * nv + j];
    for (int p = 0; p < j; ++p) dd -= R[(size_t)p * m + j] * R[(size_t)p * m + j];
    if (!(dd > kGramPivotTol * G[(size_t)j * nv + j])) {
      k = j;
      break;
    }
    R[(size_t)j * m + j] = sqrt(dd);
  }
  if (k == 0) return GMG_ERR_BREAKDOWN;
  // Y = R^{-T} C with C = K_k^T M K_k (forward substitution by columns), then H = Y R^{-1}
  std::vector<double> Y((size_t)k * k), H((size_t)k * k);
  for (int j = 0; j < k; ++j)
    for (int i = 0; i < k; ++i) {
      const double* g = &G[(size_t)i * nv];
      double t = j == 0 ? 0.5 * (g[1] + g[0]) : 0.25 * (g[j + 1] + 2.0 * g[j] + g[j - 1]);
      for (int p = 0; p < i; ++p) t -= R[(size_t)p * m + i] * Y[(size_t)p * k + j];
      Y[(size_t)i * k + j] = t / R[(size_t)i * m + i];
    }
  for (int r = 0; r < k; ++r)
    for (int j = 0; j < k; ++j) {
      double t = Y[(size_t)r * k + j];
      for (int p = 0; p < j; ++p) t -= H[(size_t)r * k + p] * R[(size_t)p * m + j];
      H[(size_t)r * k + j] = t / R[(size_t)j * m + j];
    }
  // H is upper Hessenberg in exact arithmetic; below the subdiagonal there is only rounding
  for (int r = 2; r < k; ++r)
    for (int j = 0; j < r - 1; ++j) H[(size_t)r * k + j] = 0.0;
  std::vector<double> wr, wi;
  if (hessenberg_eigs(H, k, wr, wi) != 0) return GMG_ERR_BREAKDOWN;
  double lam = -1e300;
  for (int i = 0; i < k; ++i) lam = std::max(lam, wr[i]);
  *lam_out = lam;
  return GMG_OK;
}

// lambda_max, lambda* of level l: the largest Ritz value of B^{-1} A_l
// (Sec. 3.2) in the level precision T.  FP32 with the SSOR preconditioner and
// at most 11 steps (the mixed-precision set-up; the bounds only steer the FP32
// smoother): the Chebyshev basis and its Gram matrix (ritz_chebyshev_basis).
// Otherwise Arnoldi with Gram-Schmidt: FP64 basis in V, temporaries bvec / w;
// FP32 basis in Z, temporaries the level's r / z.
template <typename T>
gmg_status eig_bounds(gmg_ctx* c, int l) {
  LevelData& L = c->lev[l];
  const size_t n = L.n;
  const int steps = c->p.eig_steps;
  const bool f32 = sizeof(T) == 4;
  T* V = f32 ? (T*)c->Z : (T*)(void*)c->V;  // (steps+1) vectors of n, stride n
  T* t1 = f32 ? (T*)L.r : (T*)(void*)c->bvec;
  T* t2 = f32 ? (T*)L.z : (T*)(void*)c->w;
  if (f32 && c->p.smoother_pc == GMG_PC_SGS && steps + 1 <= kGramMaxVectors) {
    double lam = 0.0;
    CKS(ritz_chebyshev_basis(c, l, &lam));
    if (!(lam > 0) || !isfinite(lam)) return GMG_ERR_BREAKDOWN;
    L.lam_hat = lam;
    L.lam_max = c->p.eig_hi * lam;
    L.lam_min = c->p.eig_lo * lam;
    return GMG_OK;
  }
  CKS(prof_hash_vector<T>(c, n, V, c->s));
  CKS(norm_dev<T>(c, n, V, SL_NORM));
  CKS(prof_scale<T>(c, n, V, V, c->dscal + SL_NORM + 1, c->s));
  // The columns of H stay on the device (the normalisation reads 1/||w|| there)
  // and come to the host once, after the last step: one host sync per level.
  // After a breakdown (||w|| = 0) the later vectors are zero and their columns
  // are dropped on the host.
  const bool fused_mv = sizeof(T) == 4 && L.fused;
  // On levels with the fused smoother, one fused basis step forms the product:
  // with b = 0 (not read), x_in = v, c2 = -1 and ce = 0 its x_out is B^{-1}(A v).
  for (int j = 0; j < steps; ++j) {
    if (fused_mv) {
      // the basis step with ce = 0 and no d: t2 = B^{-1} A v; the level's d stays untouched
      CKS(lv_cheb_fused(c, L, (const float*)L.b, (const float*)(V + (size_t)j * n), (float*)t2, 0.0, -1.0,
                        CHEB_UPDATE | CHEB_FIRST | CHEB_EIG, 0.0));
    } else {
      CKS(lv_apply<T>(c, L, V + (size_t)j * n, t1));
      CKS(smoother_pc<T>(c, L, t1, t2));
    }
    // One classical Gram-Schmidt pass in FP32: the bounds only steer the FP32
    // smoother, and the second pass moves lambda-hat by less than 1e-7.
    CKS(orthogonalize<T>(c, n, V, n, j + 1, t2, f32));
    CK(launch_gather_column(c->dscal + SL_H1, c->dscal + SL_H2, c->dscal + SL_NORM, j + 1,
                            c->eigH + (size_t)j * EIG_STRIDE, c->s));
    if (j + 1 < steps)  // v_{j+1}; the last one is never used
      CKS(prof_scale<T>(c, n, t2, V + (size_t)(j + 1) * n, c->dscal + SL_NORM + 1, c->s));
  }
  CK(launch_words_to_host(c->eigH, c->heig_dev, sizeof(double) * (size_t)steps * EIG_STRIDE, c->s));
  CK(cudaStreamSynchronize(c->s));
  prof_collect(c);
  std::vector<double> H((size_t)(steps + 1) * steps, 0.0);
  int m = steps;
  const bool cgs2 = c->p.orthogonalization == GMG_ORTH_CGS2;
  for (int j = 0; j < steps; ++j) {
    const double* col = c->heig + (size_t)j * EIG_STRIDE;
    const int k = j + 1;
    for (int i = 0; i < k; ++i) {
      const double h = col[i] + (cgs2 ? col[k + i] : 0.0);
      if (!isfinite(h)) return GMG_ERR_NONFINITE;
      H[(size_t)i * steps + j] = h;
    }
    if (!isfinite(col[2 * k])) return GMG_ERR_NONFINITE;
    H[(size_t)k * steps + j] = col[2 * k];
    if (col[2 * k] == 0.0) {
      m = k;
      break;
    }
  }
  std::vector<double> Hm((size_t)m * m);
  for (int r = 0; r < m; ++r)
    for (int q = 0; q < m; ++q) Hm[(size_t)r * m + q] = H[(size_t)r * steps + q];
  std::vector<double> wr, wi;
  if (hessenberg_eigs(Hm, m, wr, wi) != 0) return GMG_ERR_BREAKDOWN;
  double lam = -1e300;
  for (int i = 0; i < m; ++i) lam = std::max(lam, wr[i]);
  if (!(lam > 0) || !isfinite(lam)) return GMG_ERR_BREAKDOWN;
  L.lam_hat = lam;
  L.lam_max = c->p.eig_hi * lam;
  L.lam_min = c->p.eig_lo * lam;
  return GMG_OK;
}

// Coarse operators (8-child means or series-parallel faces) and the
// prolongation weights, in level precision T from the finest level's
// coefficient (FP32 copy in mixed precision).
template <typename T>
gmg_status build_operators(gmg_ctx* c) {
  const int top = (int)c->lev.size() - 1;
  if (c->p.coarsening == GMG_COARSEN_SERIES) {
    for (int l = top; l >= 1; --l) {
      const LevelData& Fi = c->lev[l];
      LevelData& Co = c->lev[l - 1];
      T* k = (T*)Co.kf;
      const T* a = Fi.faces ? nullptr : level_a<T>(Fi);
      const Faces<T> FF = Fi.faces ? level_faces<T>(Fi) : Faces<T>{};
      const double bytes = (a ? 1.0 : 3.0) * Fi.n * sizeof(T) + (3.0 * Co.n + Co.g.plane()) * sizeof(T);
      CKS(run_kernel(c, K_COARSEN_FACES, bytes, [&]() {
        return launch_coarsen_faces<T>(Fi.g, a, FF, k, k + Co.n, k + 2 * Co.n, k + 3 * Co.n, c->s);
      }));
    }
  } else {
    for (int l = top; l >= 1; --l)
      CKS(prof_coarsen_coef(c, c->lev[l].g, c->lev[l].a64, c->lev[l - 1].a64,
                            c->mixed ? c->lev[l - 1].a32 : nullptr, c->s));
  }
  if (c->p.prolongation == GMG_PROLONG_OPDEP) {
    for (int l = 1; l <= top; ++l) {
      const LevelData& L = c->lev[l];
      const T* a = L.faces ? nullptr : level_a<T>(L);
      const Faces<T> FF = L.faces ? level_faces<T>(L) : Faces<T>{};
      const double bytes = ((a ? 1.0 : 3.0) + 3.0) * L.n * sizeof(T);
      CKS(run_kernel(c, K_PROLONG_WEIGHTS, bytes,
                     [&]() { return launch_prolong_weights<T>(L.g, a, FF, (T*)L.wp, c->s); }));
    }
  }
  return GMG_OK;
}

template <typename T>
gmg_status assemble_coarse_faces(gmg_ctx* c, const LevelData& C0) {
  return run_kernel(c, K_COARSE_ASSEMBLE, 8.0 * C0.n * C0.n, [&]() {
    return launch_coarse_assemble_faces<T>(C0.g, level_faces<T>(C0), c->cA, c->s);
  });
}

gmg_status build(gmg_ctx* c, const double* a_dev) {
  const double t0 = now_ms();
  LevelData& F = c->lev.back();
  // coefficient must be finite and positive
  CKS(prof_coef_check(c, F.n, a_dev, c->partial, c->s));
  CKS(prof_finalize_check(c, c->partial, reduce_blocks(F.n), c->dscal + SL_CHECK, c->s));
  CKS(read_scalars(c, SL_CHECK, 2));
  if (c->hpin[SL_CHECK + 1] != 0.0) return GMG_ERR_ARG;
  CKS(prof_copy_d(c, F.n, a_dev, F.a64, c->s));
  if (c->mixed) CKS(prof_cast_d2f(c, F.n, F.a64, F.a32, c->s));
  if (F.a2) CKS(prof_split(c, F.n, F.a64, F.a2, c->s));
  CKS(c->mixed ? build_operators<float>(c) : build_operators<double>(c));
  for (int l = 1; l < (int)c->lev.size(); ++l) CKS(c->mixed ? eig_bounds<float>(c, l) : eig_bounds<double>(c, l));
  // coarsest: dense Cholesky and explicit inverse
  const LevelData& C0 = c->lev[0];
  if (C0.faces)
    CKS(c->mixed ? assemble_coarse_faces<float>(c, C0) : assemble_coarse_faces<double>(c, C0));
  else
    CKS(prof_coarse_assemble(c, C0.g, C0.a64, c->cA, c->s));
  CKS(prof_coarse_factor(c, c->nc, c->cA, c->cW, c->cinv64, nullptr, c->cstatus, c->s));
  CK(launch_words_to_host(c->cstatus, c->hstat_dev, 2 * sizeof(int), c->s));
  CK(cudaStreamSynchronize(c->s));
  if (c->hstat[1] != 0) return GMG_ERR_CUDA;  // a smoother step's copies did not arrive
  if (c->hstat[0] != 0) return GMG_ERR_BREAKDOWN;
  c->setup_ms = (float)(now_ms() - t0);
  return GMG_OK;
}

// ---------------------------------------------------------------------------
// V-cycle (Sec. 3.2, Appendix A)
// ---------------------------------------------------------------------------

// cheb_steps Chebyshev steps with the smoother preconditioner; x_is_zero
// starts from x = 0 (then r = b and x's contents are ignored).
template <typename T>
gmg_status smooth(gmg_ctx* c, int l, const T* b, T* x, bool x_is_zero) {
  const LevelData& L = c->lev[l];
  T* r = (T*)L.r;
  T* z = (T*)L.z;
  T* d = (T*)L.d;
  const double theta = 0.5 * (L.lam_max + L.lam_min), delta = 0.5 * (L.lam_max - L.lam_min);
  const double sigma = theta / delta;
  double rho = 1.0 / sigma;
  const int pc = c->p.smoother_pc;
  for (int st = 0; st < c->p.cheb_steps; ++st) {
    double c1 = 0.0, c2 = 1.0 / theta;
    int flags = CHEB_UPDATE;
    if (st == 0) {
      flags |= CHEB_FIRST;
      if (x_is_zero) flags |= CHEB_XZERO;
    } else {
      const double rho_new = 1.0 / (2.0 * sigma - rho);
      c1 = rho_new * rho;
      c2 = 2.0 * rho_new / delta;
      rho = rho_new;
    }
    const T* rr;
    if (st == 0 && x_is_zero) {
      CKS(lv_residual<T>(c, L, b, (const T*)nullptr, (T*)nullptr, z, pc));
      rr = b;
    } else {
      CKS(lv_residual<T>(c, L, b, x, r, z, pc));
      rr = r;
    }
    if (pc == GMG_PC_SGS) {
      CKS(lv_sgs_half<T>(c, L, rr, z, 1, d, x, c1, c2, flags));
      CKS(lv_sgs_half<T>(c, L, rr, z, 0, d, x, c1, c2, flags));
    } else {
      CKS(prof_cheb_update<T>(c, L.n, z, d, x, c1, c2, flags, c->s));
    }
  }
  return GMG_OK;
}

// cheb_steps fused Chebyshev steps on an FP32 level, x_in = xin (null: 0).
// Step st writes `target` if (steps-1-st) is even, else `alt`, so the last
// step writes `target`; the first step's output buffer must differ from xin.
gmg_status smooth_fused(gmg_ctx* c, int l, const float* b, const float* xin, float* target, float* alt) {
  const LevelData& L = c->lev[l];
  const double theta = 0.5 * (L.lam_max + L.lam_min), delta = 0.5 * (L.lam_max - L.lam_min);
  const double sigma = theta / delta;
  double rho = 1.0 / sigma;
  const int s = c->p.cheb_steps;
  const float* cur = xin;
  for (int st = 0; st < s; ++st) {
    double c1 = 0.0, c2 = 1.0 / theta;
    int flags = CHEB_UPDATE;
    if (st == 0) {
      flags |= CHEB_FIRST;
    } else {
      const double rho_new = 1.0 / (2.0 * sigma - rho);
      c1 = rho_new * rho;
      c2 = 2.0 * rho_new / delta;
      rho = rho_new;
    }
    if (st == s - 1) flags |= CHEB_LAST;
    float* dst = ((s - 1 - st) % 2 == 0) ? target : alt;
    if (dst == cur) return GMG_ERR_ARG;
    CKS(lv_cheb_fused(c, L, b, cur, dst, c1, c2, flags));
    cur = dst;
  }
  return GMG_OK;
}

template <typename T>
gmg_status vcycle(gmg_ctx* c, int l, const T* b, T* x, bool from_guess = false) {
  if (l == 0) return (prof_coarse_apply<T>(c, c->nc, c->cinv64, b, x, c->s));
  const LevelData& L = c->lev[l];
  const LevelData& Lc = c->lev[l - 1];
  if constexpr (sizeof(T) == 4) {
    if (L.fused) {
      // pre-smoothing ends in the buffer that post-smoothing does not write first
      float* U = L.x2;
      float* pre = (c->p.cheb_steps % 2) ? U : x;
      float* pre_alt = (pre == U) ? x : U;
      CKS(smooth_fused(c, l, b, from_guess ? x : nullptr, pre, pre_alt));
      CKS(lv_residual_restrict<float>(c, L, b, pre, (float*)Lc.b));
      CKS(vcycle<float>(c, l - 1, (const float*)Lc.b, (float*)Lc.x));
      CKS(lv_prolong<float>(c, L, (const float*)Lc.x, pre));
      return smooth_fused(c, l, b, pre, x, U);
    }
  }
  CKS(smooth<T>(c, l, b, x, !from_guess));
  CKS(lv_residual_restrict<T>(c, L, b, x, (T*)Lc.b));
  CKS(vcycle<T>(c, l - 1, (const T*)Lc.b, (T*)Lc.x));
  CKS(lv_prolong<T>(c, L, (const T*)Lc.x, x));
  CKS(smooth<T>(c, l, b, x, false));
  return GMG_OK;
}

// z (level precision, finest size) = M v, v FP64.
// Full multigrid (Sec. 3.2): b is carried down by the 8-child mean, the
// coarsest grid is solved directly, and each finer level starts from the
// prolonged coarser result and takes one V-cycle.  Level l < top keeps its
// right-hand side in lev[l].b and its result in lev[l].x; the V-cycle of
// level l then reuses the buffers of the levels below, which are done.
template <typename T>
gmg_status fmg(gmg_ctx* c, int top, const T* b, T* z) {
  const T* bl = b;
  for (int l = top; l >= 1; --l) {
    CKS(lv_residual_restrict<T>(c, c->lev[l], bl, (const T*)nullptr, (T*)c->lev[l - 1].b));
    bl = (const T*)c->lev[l - 1].b;
  }
  CKS(prof_coarse_apply<T>(c, c->nc, c->cinv64, (const T*)c->lev[0].b, (T*)c->lev[0].x, c->s));
  for (int l = 1; l <= top; ++l) {
    const LevelData& L = c->lev[l];
    T* xl = l == top ? z : (T*)L.x;
    const T* blv = l == top ? b : (const T*)L.b;
    CK(cudaMemsetAsync(xl, 0, L.n * sizeof(T), c->s));
    CKS(lv_prolong<T>(c, L, (const T*)c->lev[l - 1].x, xl));
    CKS(vcycle<T>(c, l, blv, xl, true));
  }
  return GMG_OK;
}

gmg_status precondition(gmg_ctx* c, const double* v, void* z) {
  const int top = (int)c->lev.size() - 1;
  ++c->precond_calls;
  if (c->mixed) {
    float* bf = (float*)c->lev[top].b;
    if (c->b32_of != v) CKS(prof_cast_d2f(c, c->N(), v, bf, c->s));
    c->b32_of = nullptr;  // the cycle may overwrite it
    if (c->fmg_now && top > 0) return fmg<float>(c, top, bf, (float*)z);
    return vcycle<float>(c, top, bf, (float*)z);
  }
  if (c->fmg_now && top > 0) return fmg<double>(c, top, v, (double*)z);
  return vcycle<double>(c, top, v, (double*)z);
}

// w = A z (FP64 operator on a level-precision vector of the finest size).
gmg_status apply_outer(gmg_ctx* c, const void* z, double* w) {
  const LevelData& F = c->fine();
  if (c->mixed && F.a2) return prof_apply_df64(c, F.g, F.dc, F.a2, (const float*)z, w, c->s);
  if (c->mixed) return (prof_apply<double, float, double>(c, F.g, F.a64, (const float*)z, w, c->s));
  return (prof_apply<double, double, double>(c, F.g, F.a64, (const double*)z, w, c->s));
}

void* zvec(gmg_ctx* c, int j) { return (char*)c->Z + (size_t)j * c->N() * c->esz; }

// FGMRES (flexible = true, Algorithm 1) or right-preconditioned GMRES, which
// keeps only V and forms x += M (V y) at the end of each cycle.
gmg_status solve_impl(gmg_ctx* c, const double* f, double* x, int homogeneous, gmg_solve_info* info,
                      bool flexible = true) {
  const double t0 = now_ms();
  c->precond_calls = 0;
  c->b32_of = nullptr;
  const LevelData& F = c->fine();
  const size_t n = F.n;
  const int m = c->p.restart;
  gmg_solve_info loc;
  memset(&loc, 0, sizeof(loc));
  loc.setup_ms = c->setup_ms;
  gmg_status result = GMG_OK;

  CKS(prof_rhs(c, F.g, F.a64, f, c->bvec, c->p.phi_bottom, c->p.phi_top, homogeneous, c->s));
  CKS(norm_dev(c, n, c->bvec, SL_NORM));
  CKS(read_scalars(c, SL_NORM, 2));
  const double bnorm = c->hpin[SL_NORM];
  loc.bnorm = bnorm;
  if (!isfinite(bnorm)) {
    result = GMG_ERR_NONFINITE;
    goto done;
  }
  if (bnorm == 0.0) {
    CK(cudaMemsetAsync(x, 0, n * sizeof(double), c->s));
    loc.converged = 1;
    loc.true_rel_residual = 0.0;
    goto done;
  }
  {
    std::vector<double> R((size_t)(m + 1) * m, 0.0), cs(m), sn(m), g(m + 1), col(m + 2), y(m);
    // A zero initial guess (||x0|| = 0) gives r0 = b exactly: the first cycle
    // then starts from b and ||b|| without the FP64 operator pass.
    CKS(norm_dev(c, n, x, SL_NORM));
    CKS(read_scalars(c, SL_NORM, 2));
    bool r0_is_b = c->hpin[SL_NORM] == 0.0;
    // Sec. 3.2: full multigrid for a solve without a previous potential
    c->fmg_now = c->p.cycle == GMG_CYCLE_FMG || (c->p.cycle == GMG_CYCLE_AUTO && r0_is_b);
    loc.fmg = c->fmg_now ? 1 : 0;
    for (;;) {
      // r0 = b - A x0, beta = ||r0||, v1 = r0 / beta (start of an Arnoldi cycle)
      double beta = bnorm;
      if (!r0_is_b) {
        CKS(prof_residual<double>(c, F.g, F.a64, c->bvec, x, c->V, nullptr, PC_NONE, c->s));
        CKS(norm_dev(c, n, c->V, SL_NORM));
        CKS(read_scalars(c, SL_NORM, 2));
        beta = c->hpin[SL_NORM];
      }
      if (!isfinite(beta)) {
        result = GMG_ERR_NONFINITE;
        break;
      }
      loc.true_rel_residual = beta / bnorm;
      if (loc.true_rel_residual < c->p.rtol) {
        loc.converged = 1;
        break;
      }
      if (loc.iterations >= c->p.max_iters) {
        result = GMG_ERR_NOT_CONVERGED;
        break;
      }
      if (c->mixed) {  // v_1 and its FP32 rounding (the first preconditioner input) in one pass
        CKS(prof_scale_round(c, n, r0_is_b ? c->bvec : c->V, c->V, (float*)c->lev.back().b, nullptr, 1.0 / beta,
                             c->s));
        c->b32_of = c->V;
      } else {
        CKS(prof_scale_value(c, n, r0_is_b ? c->bvec : c->V, c->V, 1.0 / beta, c->s));
      }
      r0_is_b = false;  // later cycles restart from x_k != 0
      std::fill(g.begin(), g.end(), 0.0);
      g[0] = beta;
      int k = 0;
      bool fail = false;
      for (int j = 0; j < m; ++j) {
        double* vj = c->V + (size_t)j * n;
        void* zj = zvec(c, flexible ? j : 0);            // GMRES needs no stored z
        CKS(precondition(c, vj, zj));                    // z_j = M v_j (one V-cycle)
        CKS(apply_outer(c, zj, c->w));                   // w = A z_j
        CKS(orthogonalize(c, n, c->V, n, j + 1, c->w));   // Gram-Schmidt: h_{i,j}
        cudaEvent_t gap = nullptr;                       // the GPU's wait for the host's Givens step
        CKS(read_column(c, j + 1, col.data(), &gap));    // h_{j+1,j} = ||w||
        host_gap_end(c, gap);  // the Givens update below takes about a microsecond more
        for (int i = 0; i <= j + 1; ++i)
          if (!isfinite(col[i])) fail = true;
        if (fail) {
          result = GMG_ERR_NONFINITE;
          break;
        }
        const double hnext = col[j + 1];
        // least-squares residual min ||beta e_1 - Hbar_j y|| by Givens rotations
        for (int i = 0; i < j; ++i) {
          const double t = cs[i] * col[i] + sn[i] * col[i + 1];
          col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
          col[i] = t;
        }
        const double rr = hypot(col[j], col[j + 1]);
        if (rr == 0.0) {
          result = GMG_ERR_BREAKDOWN;
          fail = true;
          break;
        }
        cs[j] = col[j] / rr;
        sn[j] = col[j + 1] / rr;
        col[j] = rr;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        for (int i = 0; i <= j; ++i) R[(size_t)i * m + j] = col[i];
        k = j + 1;
        loc.iterations++;
        const double est = fabs(g[j + 1]) / bnorm;
        if (loc.n_history < GMG_MAX_HISTORY) loc.res_history[loc.n_history++] = est;
        if (hnext == 0.0) break;  // lucky breakdown: the solution is in K_j
        if (est < c->p.rtol || loc.iterations >= c->p.max_iters) break;  // stopping test
        double* vnext = c->V + (size_t)(j + 1) * n;
        if (c->mixed) {  // v_{j+1} = w / h_{j+1,j} and its FP32 rounding for the next V-cycle
          CKS(prof_scale_round(c, n, c->w, vnext, (float*)c->lev.back().b, c->dscal + SL_NORM + 1, 0.0, c->s));
          c->b32_of = vnext;
        } else {
          CKS(prof_scale(c, n, c->w, vnext, c->dscal + SL_NORM + 1, c->s));
        }
      }
      if (fail) break;
      // y_k from the triangular system, x_k = x_0 + Z_k y_k
      for (int i = k - 1; i >= 0; --i) {
        double t = g[i];
        for (int q = i + 1; q < k; ++q) t -= R[(size_t)i * m + q] * y[q];
        y[i] = t / R[(size_t)i * m + i];
      }
      for (int i = 0; i < k; ++i) c->hpin[SL_Y + i] = y[i];
      CK(cudaMemcpyAsync(c->dscal + SL_Y, c->hpin + SL_Y, sizeof(double) * k, cudaMemcpyHostToDevice, c->s));
      if (!flexible) {
        // GMRES: u = V y, then x += M u
        CK(cudaMemsetAsync(c->w, 0, n * sizeof(double), c->s));
        CKS(prof_update_solution<double>(c, n, c->w, c->V, n, k, c->dscal + SL_Y, c->s));
        CKS(precondition(c, c->w, zvec(c, 0)));
        if (c->mixed)
          CKS(prof_lin3<float, double>(c, n, 1.0, (const float*)zvec(c, 0), 0.0, nullptr, 1.0, x, x));
        else
          CKS(prof_lin3<double, double>(c, n, 1.0, (const double*)zvec(c, 0), 0.0, nullptr, 1.0, x, x));
      } else if (c->mixed) {
        CKS(prof_update_solution<float>(c, n, x, (const float*)c->Z, n, k, c->dscal + SL_Y, c->s));
      } else {
        CKS(prof_update_solution<double>(c, n, x, (const double*)c->Z, n, k, c->dscal + SL_Y, c->s));
      }
      loc.restarts++;  // restart from x_k (the true residual is checked at the loop top)
    }
  }
done:
  CK(launch_words_to_host(c->cstatus + 1, c->hstat_dev + 1, sizeof(int), c->s));
  CK(cudaStreamSynchronize(c->s));
  prof_collect(c);
  if (c->hstat[1] != 0) result = GMG_ERR_CUDA;  // a smoother step's copies did not arrive
  loc.solve_ms = (float)(now_ms() - t0);
  loc.precond_calls = (int)c->precond_calls;
  if (info) *info = loc;
  return result;
}

// ---------------------------------------------------------------------------
// Short-recurrence Krylov methods with the same preconditioner (the paper's
// comparison of elliptic solvers, Tables t1 and t2): preconditioned CG,
// flexible CG with one stored direction, CGS and BiCGSTAB, right-
// preconditioned.  FP64 vectors; the preconditioner output z is FP32 in mixed
// mode and A z takes the double-float Arnoldi product; A p for a combination
// p = z + beta p' is formed as A z + beta A p' so no FP64 stencil runs inside
// the iteration.  Each method stops when its recurrence residual falls below
// rtol ||b||; the true residual is then checked and the method starts again
// from x if needed (as for FGMRES).  Work vectors live in the Krylov basis
// storage: V[0] r, V[1] p, V[2] q, V[3] the shadow residual, V[4..6] method
// temporaries; Z[0], Z[1] hold preconditioner outputs.
// ---------------------------------------------------------------------------

gmg_status dot64(gmg_ctx* c, const double* x, const double* y, double* out) {
  const size_t n = c->N();
  CKS(prof_multi_dot<double>(c, n, x, y, 0, 1, c->partial, c->s));
  CKS(prof_finalize(c, c->partial, reduce_blocks(n), 1, c->dscal + SL_H1, 0, c->s));
  CKS(read_scalars(c, SL_H1, 1));
  *out = c->hpin[SL_H1];
  return GMG_OK;
}

gmg_status norm64(gmg_ctx* c, const double* x, double* out) {
  CKS(norm_dev<double>(c, c->N(), x, SL_NORM));
  CKS(read_scalars(c, SL_NORM, 2));
  *out = c->hpin[SL_NORM];
  return GMG_OK;
}

template <typename TZ>
gmg_status short_cycle(gmg_ctx* c, int method, double* x, double bnorm, gmg_solve_info& loc, bool& breakdown) {
  const size_t n = c->N();
  double* V = c->V;
  double *r = V, *p = V + n, *q = V + 2 * n, *rt = V + 3 * n, *t4 = V + 4 * n, *t5 = V + 5 * n, *t6 = V + 6 * n;
  TZ* z0 = (TZ*)zvec(c, 0);
  TZ* z1 = (TZ*)zvec(c, 1);
  double* w = c->w;
  const bool widen = sizeof(TZ) == 4;
  const int cap = c->p.max_iters;
  auto record = [&](double rnorm) {
    ++loc.iterations;
    if (loc.n_history < GMG_MAX_HISTORY) loc.res_history[loc.n_history++] = rnorm / bnorm;
    return rnorm / bnorm < c->p.rtol || loc.iterations >= cap || !isfinite(rnorm);
  };
  // z = M r, zd = z in FP64 (a copy only in mixed mode), w = A z
  auto pc_op = [&](const double* rv, TZ* z, const double** zd) -> gmg_status {
    CKS(precondition(c, rv, z));
    if (widen) {
      CKS(prof_lin3<TZ, double>(c, n, 1.0, z, 0.0, nullptr, 0.0, nullptr, t6));
      *zd = t6;
    } else {
      *zd = (const double*)z;
    }
    return apply_outer(c, z, w);
  };
  breakdown = false;
  double rnorm = 0.0;
  if (method == GMG_KRYLOV_CG || method == GMG_KRYLOV_FCG) {
    const bool flexible = method == GMG_KRYLOV_FCG;
    double rho = 0.0, pq_prev = 0.0;
    for (int it = 0;; ++it) {
      const double* zd = nullptr;
      CKS(pc_op(r, z0, &zd));
      if (it == 0) {
        CKS(prof_lin3<double, double>(c, n, 1.0, zd, 0.0, nullptr, 0.0, nullptr, p));
        CKS(prof_lin3<double, double>(c, n, 1.0, w, 0.0, nullptr, 0.0, nullptr, q));
        if (!flexible) CKS(dot64(c, r, zd, &rho));
      } else {
        double beta;
        if (flexible) {  // Notay: beta = -(z, q') / (p', q')
          double zq;
          CKS(dot64(c, zd, q, &zq));
          beta = -zq / pq_prev;
        } else {         // Fletcher-Reeves form of PCG
          double rho_new;
          CKS(dot64(c, r, zd, &rho_new));
          beta = rho_new / rho;
          rho = rho_new;
        }
        if (!isfinite(beta)) {
          breakdown = true;
          return GMG_OK;
        }
        CKS(prof_lin3<double, double>(c, n, 1.0, zd, 0.0, nullptr, beta, p, p));  // p = z + beta p
        CKS(prof_lin3<double, double>(c, n, 1.0, w, 0.0, nullptr, beta, q, q));   // q = A z + beta q
      }
      double pq, num;
      CKS(dot64(c, p, q, &pq));
      if (flexible) CKS(dot64(c, p, r, &num));
      else num = rho;
      const double alpha = num / pq;
      if (!isfinite(alpha) || pq == 0.0) {
        breakdown = true;
        return GMG_OK;
      }
      CKS(prof_lin3<double, double>(c, n, alpha, p, 0.0, nullptr, 1.0, x, x));    // x += alpha p
      CKS(prof_lin3<double, double>(c, n, -alpha, q, 0.0, nullptr, 1.0, r, r));   // r -= alpha q
      CKS(norm64(c, r, &rnorm));
      if (record(rnorm)) return GMG_OK;
      pq_prev = pq;
    }
  }
  if (method == GMG_KRYLOV_CGS) {
    CKS(prof_lin3<double, double>(c, n, 1.0, r, 0.0, nullptr, 0.0, nullptr, rt));
    CK(cudaMemsetAsync(p, 0, n * sizeof(double), c->s));
    CK(cudaMemsetAsync(q, 0, n * sizeof(double), c->s));
    double rho_old = 1.0;
    for (int it = 0;; ++it) {
      double rho;
      CKS(dot64(c, rt, r, &rho));
      const double beta = it == 0 ? 0.0 : rho / rho_old;
      if (!isfinite(beta) || rho == 0.0) {
        breakdown = true;
        return GMG_OK;
      }
      double* u = t4;
      CKS(prof_lin3<double, double>(c, n, 1.0, r, beta, q, 0.0, nullptr, u));           // u = r + beta q
      CKS(prof_lin3<double, double>(c, n, 1.0, u, beta, q, beta * beta, p, p));         // p = u + beta (q + beta p)
      CKS(precondition(c, p, z0));                                                      // p^ = M p
      CKS(apply_outer(c, z0, w));                                                       // v^ = A p^
      double rv;
      CKS(dot64(c, rt, w, &rv));
      const double alpha = rho / rv;
      if (!isfinite(alpha)) {
        breakdown = true;
        return GMG_OK;
      }
      CKS(prof_lin3<double, double>(c, n, 1.0, u, -alpha, w, 0.0, nullptr, q));         // q = u - alpha v^
      CKS(prof_lin3<double, double>(c, n, 1.0, u, 1.0, q, 0.0, nullptr, t5));           // u + q
      CKS(precondition(c, t5, z1));                                                     // u^ = M (u + q)
      CKS(prof_lin3<TZ, double>(c, n, alpha, z1, 0.0, nullptr, 1.0, x, x));              // x += alpha u^
      CKS(apply_outer(c, z1, w));                                                       // A u^
      CKS(prof_lin3<double, double>(c, n, -alpha, w, 0.0, nullptr, 1.0, r, r));          // r -= alpha A u^
      rho_old = rho;
      CKS(norm64(c, r, &rnorm));
      if (record(rnorm)) return GMG_OK;
    }
  }
  // BiCGSTAB
  CKS(prof_lin3<double, double>(c, n, 1.0, r, 0.0, nullptr, 0.0, nullptr, rt));
  CKS(prof_lin3<double, double>(c, n, 1.0, r, 0.0, nullptr, 0.0, nullptr, p));
  double rho;
  CKS(dot64(c, rt, r, &rho));
  double* v = t4;
  double* sv = t5;
  double* tv = t6;
  for (;;) {
    CKS(precondition(c, p, z0));                                                        // p^ = M p
    CKS(apply_outer(c, z0, v));                                                         // v = A p^
    double rv;
    CKS(dot64(c, rt, v, &rv));
    const double alpha = rho / rv;
    if (!isfinite(alpha)) {
      breakdown = true;
      return GMG_OK;
    }
    CKS(prof_lin3<double, double>(c, n, 1.0, r, -alpha, v, 0.0, nullptr, sv));           // s = r - alpha v
    CKS(precondition(c, sv, z1));                                                       // s^ = M s
    CKS(apply_outer(c, z1, tv));                                                        // t = A s^
    double tt, ts;
    CKS(dot64(c, tv, tv, &tt));
    CKS(dot64(c, tv, sv, &ts));
    const double omega = tt > 0.0 ? ts / tt : 0.0;
    CKS(prof_lin3<TZ, TZ>(c, n, alpha, z0, omega, z1, 1.0, x, x));                       // x += alpha p^ + omega s^
    CKS(prof_lin3<double, double>(c, n, 1.0, sv, -omega, tv, 0.0, nullptr, r));         // r = s - omega t
    CKS(norm64(c, r, &rnorm));
    if (record(rnorm)) return GMG_OK;
    double rho_new;
    CKS(dot64(c, rt, r, &rho_new));
    const double beta = (rho_new / rho) * (alpha / omega);
    if (!isfinite(beta) || rho_new == 0.0) {
      breakdown = true;
      return GMG_OK;
    }
    CKS(prof_lin3<double, double>(c, n, 1.0, r, -beta * omega, v, beta, p, p));          // p = r + beta (p - omega v)
    rho = rho_new;
  }
}

gmg_status solve_short(gmg_ctx* c, int method, const double* f, double* x, int homogeneous, gmg_solve_info* info) {
  const double t0 = now_ms();
  c->precond_calls = 0;
  c->b32_of = nullptr;
  const LevelData& F = c->fine();
  const size_t n = F.n;
  gmg_solve_info loc;
  memset(&loc, 0, sizeof(loc));
  loc.setup_ms = c->setup_ms;
  gmg_status result = GMG_OK;
  if (c->p.restart < 7) return GMG_ERR_ARG;  // the work vectors live in V[0..6]
  CKS(prof_rhs(c, F.g, F.a64, f, c->bvec, c->p.phi_bottom, c->p.phi_top, homogeneous, c->s));
  double bnorm;
  CKS(norm64(c, c->bvec, &bnorm));
  loc.bnorm = bnorm;
  double xnorm;
  CKS(norm64(c, x, &xnorm));
  c->fmg_now = c->p.cycle == GMG_CYCLE_FMG || (c->p.cycle == GMG_CYCLE_AUTO && xnorm == 0.0);
  loc.fmg = c->fmg_now ? 1 : 0;
  if (!isfinite(bnorm)) {
    result = GMG_ERR_NONFINITE;
  } else if (bnorm == 0.0) {
    CK(cudaMemsetAsync(x, 0, n * sizeof(double), c->s));
    loc.converged = 1;
  } else {
    bool r_is_b = xnorm == 0.0;  // zero guess: r = b exactly
    for (;;) {
      if (r_is_b)
        CKS(prof_lin3<double, double>(c, n, 1.0, c->bvec, 0.0, nullptr, 0.0, nullptr, c->V));
      else
        CKS(prof_residual<double>(c, F.g, F.a64, c->bvec, x, c->V, nullptr, PC_NONE, c->s));  // r = b - A x
      r_is_b = false;
      double rn;
      CKS(norm64(c, c->V, &rn));
      if (!isfinite(rn)) {
        result = GMG_ERR_NONFINITE;
        break;
      }
      loc.true_rel_residual = rn / bnorm;
      if (loc.true_rel_residual < c->p.rtol) {
        loc.converged = 1;
        break;
      }
      if (loc.iterations >= c->p.max_iters) {
        result = GMG_ERR_NOT_CONVERGED;
        break;
      }
      bool breakdown = false;
      const int before = loc.iterations;
      CKS(c->mixed ? short_cycle<float>(c, method, x, bnorm, loc, breakdown)
                   : short_cycle<double>(c, method, x, bnorm, loc, breakdown));
      if (breakdown && loc.iterations == before) {  // no progress: a breakdown at the first step
        result = GMG_ERR_BREAKDOWN;
        break;
      }
      loc.restarts++;
    }
  }
  CK(launch_words_to_host(c->cstatus + 1, c->hstat_dev + 1, sizeof(int), c->s));
  CK(cudaStreamSynchronize(c->s));
  prof_collect(c);
  if (c->hstat[1] != 0) result = GMG_ERR_CUDA;  // a smoother step's copies did not arrive
  loc.solve_ms = (float)(now_ms() - t0);
  loc.precond_calls = (int)c->precond_calls;
  if (info) *info = loc;
  return result;
}

LevelData* level_ptr(gmg_ctx* c, int level) {
  if (!c || level < 0 || level >= (int)c->lev.size()) return nullptr;
  return &c->lev[level];
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" {

void gmg_default_params(gmg_params* p, int nx, int ny, int nz) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->nx = nx;
  p->ny = ny;
  p->nz = nz;
  p->lx = p->ly = p->lz = 1.0;
  p->phi_bottom = 0.0;
  p->phi_top = 1.0;
  p->coarse_min = 4;
  p->cheb_steps = 3;
  p->restart = 20;
  p->max_iters = 200;
  p->rtol = 1e-8;
  p->eig_steps = 10;
  p->eig_hi = 1.1;
  p->eig_lo = 0.1;
  p->precision = GMG_PREC_MIXED;
  p->prolongation = GMG_PROLONG_OPDEP;
  p->smoother_pc = GMG_PC_SGS;
  p->orthogonalization = GMG_ORTH_MGS;
  p->outer_arith = GMG_OUTER_DOUBLE_FLOAT;
  p->smoother_kernel = 0;
  p->cycle = GMG_CYCLE_V;
  p->coarsening = GMG_COARSEN_SERIES;
}

const char* gmg_status_string(gmg_status s) {
  switch (s) {
    case GMG_OK: return "ok";
    case GMG_ERR_ARG: return "invalid argument";
    case GMG_ERR_CUDA: return "CUDA error";
    case GMG_ERR_ALLOC: return "device allocation failed";
    case GMG_ERR_NOT_CONVERGED: return "not converged within max_iters";
    case GMG_ERR_BREAKDOWN: return "breakdown";
    case GMG_ERR_NONFINITE: return "non-finite value";
  }
  return "unknown status";
}

void gmg_destroy(gmg_ctx* c) {
  if (!c) return;
  if (c->s) cudaStreamSynchronize(c->s);
  prof_collect(c);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  for (cudaStream_t q : {c->cs, c->cso})
    if (q) {
      cudaStreamSynchronize(q);
      cudaStreamDestroy(q);
    }
  for (cudaEvent_t e : {c->ev_in, c->ev_a, c->ev_out, c->ev_done})
    if (e) cudaEventDestroy(e);
  for (void* p : c->dev_allocs) cudaFree(p);
  for (void* p : c->host_allocs) cudaFreeHost(p);
  delete c;
}

gmg_status gmg_setup(const gmg_params* p, const double* a_dev, void* stream, gmg_ctx** out) {
  if (!out) return GMG_ERR_ARG;
  *out = nullptr;
  int L = 0;
  CKS(validate(p, &L));
  if (!a_dev) return GMG_ERR_ARG;
  gmg_ctx* c = new (std::nothrow) gmg_ctx();
  if (!c) return GMG_ERR_ALLOC;
  c->p = *p;
  c->s = (cudaStream_t)stream;
  c->mixed = p->precision == GMG_PREC_MIXED;
  c->esz = c->mixed ? sizeof(float) : sizeof(double);
  auto fail = [&](gmg_status st) {
    gmg_destroy(c);
    return st;
  };
  // level grids, finest last
  c->lev.resize(L);
  int nx = p->nx, ny = p->ny, nz = p->nz;
  for (int l = L - 1; l >= 0; --l) {
    LevelData& D = c->lev[l];
    D.nx = nx;
    D.ny = ny;
    D.nz = nz;
    D.n = (size_t)nx * ny * nz;
    D.g = make_grid(nx, ny, nz, p->lx, p->ly, p->lz);
    nx /= 2;
    ny /= 2;
    nz /= 2;
  }
  c->nc = (int)c->lev[0].n;
  gmg_status st;
  for (int l = 0; l < L; ++l) {
    LevelData& D = c->lev[l];
    const bool top = l == L - 1;
    D.faces = p->coarsening == GMG_COARSEN_SERIES && !top;
    if (D.faces) {
      if ((st = dev_alloc(c, &D.kf, (3 * D.n + D.g.plane()) * c->esz)) != GMG_OK) return fail(st);
    } else {
      if ((st = dalloc(c, &D.a64, D.n)) != GMG_OK) return fail(st);
      if (c->mixed && (st = dalloc(c, &D.a32, D.n)) != GMG_OK) return fail(st);
    }
    if (l > 0 && p->prolongation == GMG_PROLONG_OPDEP &&
        (st = dev_alloc(c, &D.wp, 3 * D.n * c->esz)) != GMG_OK)
      return fail(st);
    if (top && c->mixed && p->outer_arith == GMG_OUTER_DOUBLE_FLOAT) {
      if ((st = dalloc(c, &D.a2, D.n)) != GMG_OK) return fail(st);
      D.dc = make_df_coef(D.g);
    }
    if (!top && (st = dev_alloc(c, &D.x, D.n * c->esz)) != GMG_OK) return fail(st);
    if ((!top || c->mixed) && (st = dev_alloc(c, &D.b, D.n * c->esz)) != GMG_OK) return fail(st);
    D.fused = c->mixed && l > 0 && p->smoother_pc == GMG_PC_SGS && p->smoother_kernel != 1 &&
              fused_smoother_eligible(D.g);
    if (D.fused && (st = dalloc(c, &D.x2, D.n)) != GMG_OK) return fail(st);
    if (l > 0 || L == 1) {
      if ((st = dev_alloc(c, &D.r, D.n * c->esz)) != GMG_OK) return fail(st);
      if ((st = dev_alloc(c, &D.z, D.n * c->esz)) != GMG_OK) return fail(st);
      if ((st = dev_alloc(c, &D.d, D.n * c->esz)) != GMG_OK) return fail(st);
      // the fused smoother's first step with x_in reads d with weight 0: d must hold finite values
      if (D.fused && cudaMemset(D.d, 0, D.n * c->esz) != cudaSuccess) return fail(GMG_ERR_CUDA);
    }
  }
  const size_t N = c->lev.back().n;
  c->nv = std::max(p->restart, p->eig_steps) + 1;
  if ((st = dalloc(c, &c->V, (size_t)c->nv * N)) != GMG_OK) return fail(st);
  // Z also holds the FP32 eigen-estimate basis of the mixed set-up (eig_steps + 1 vectors)
  const size_t nz_vec = (size_t)std::max(p->restart, c->mixed ? p->eig_steps + 1 : 0);
  if ((st = dev_alloc(c, &c->Z, nz_vec * N * c->esz)) != GMG_OK) return fail(st);
  if ((st = dalloc(c, &c->w, N)) != GMG_OK) return fail(st);
  if ((st = dalloc(c, &c->bvec, N)) != GMG_OK) return fail(st);
  // 1024 blocks x up to 78 sums (the Gram matrix of 12 vectors)
  if ((st = dalloc(c, &c->partial, (size_t)1024 * 80)) != GMG_OK) return fail(st);
  if ((st = dalloc(c, &c->dscal, N_SCAL)) != GMG_OK) return fail(st);
  if ((st = dalloc(c, &c->cA, (size_t)c->nc * c->nc)) != GMG_OK) return fail(st);
  if ((st = dalloc(c, &c->cW, (size_t)c->nc * c->nc)) != GMG_OK) return fail(st);
  if ((st = dalloc(c, &c->cinv64, (size_t)c->nc * c->nc)) != GMG_OK) return fail(st);
  // cstatus[0]: the coarse factorisation's status; cstatus[1]: waits of the
  // copy-fed smoother that ran out (sticky)
  if ((st = dalloc(c, &c->cstatus, 4)) != GMG_OK) return fail(st);
  if (cudaMemset(c->cstatus, 0, 4 * sizeof(int)) != cudaSuccess) return fail(GMG_ERR_CUDA);
  if ((st = dalloc(c, &c->eigH, (size_t)EIG_STRIDE * EIG_MAX_STEPS)) != GMG_OK) return fail(st);
  {
    // mapped, so that kernels write the scalars the host reads (read_scalars)
    void *h = nullptr, *hd = nullptr;
    if (cudaHostAlloc(&h, sizeof(double) * N_SCAL, cudaHostAllocMapped) != cudaSuccess) return fail(GMG_ERR_ALLOC);
    c->host_allocs.push_back(h);
    if (cudaHostGetDevicePointer(&hd, h, 0) != cudaSuccess) return fail(GMG_ERR_CUDA);
    c->hpin = (double*)h;
    c->hpin_dev = (double*)hd;
    if (cudaHostAlloc(&h, sizeof(int) * 4, cudaHostAllocMapped) != cudaSuccess) return fail(GMG_ERR_ALLOC);
    c->host_allocs.push_back(h);
    if (cudaHostGetDevicePointer(&hd, h, 0) != cudaSuccess) return fail(GMG_ERR_CUDA);
    c->hstat = (int*)h;
    c->hstat_dev = (int*)hd;
    if (cudaHostAlloc(&h, sizeof(double) * EIG_STRIDE * EIG_MAX_STEPS, cudaHostAllocMapped) != cudaSuccess)
      return fail(GMG_ERR_ALLOC);
    c->host_allocs.push_back(h);
    if (cudaHostGetDevicePointer(&hd, h, 0) != cudaSuccess) return fail(GMG_ERR_CUDA);
    c->heig = (double*)h;
    c->heig_dev = (double*)hd;
  }
  if ((st = build(c, a_dev)) != GMG_OK) return fail(st);
  *out = c;
  return GMG_OK;
}

gmg_status gmg_update_coefficient(gmg_ctx* c, const double* a_dev) {
  if (!c || !a_dev) return GMG_ERR_ARG;
  return build(c, a_dev);
}

gmg_status fgmres_solve(gmg_ctx* c, const double* f_dev, double* phi_dev, int homogeneous_bc,
                        gmg_solve_info* info) {
  if (!c || !f_dev || !phi_dev) return GMG_ERR_ARG;
  return solve_impl(c, f_dev, phi_dev, homogeneous_bc, info);
}

gmg_status apply_operator(gmg_ctx* c, const double* x_dev, double* y_dev) {
  if (!c || !x_dev || !y_dev) return GMG_ERR_ARG;
  const LevelData& F = c->fine();
  return (prof_apply<double, double, double>(c, F.g, F.a64, x_dev, y_dev, c->s));
}

gmg_status assemble_rhs(gmg_ctx* c, const double* f_dev, double* b_dev) {
  if (!c || !f_dev || !b_dev) return GMG_ERR_ARG;
  const LevelData& F = c->fine();
  return (prof_rhs(c, F.g, F.a64, f_dev, b_dev, c->p.phi_bottom, c->p.phi_top, 0, c->s));
}

gmg_status field_from_potential(gmg_ctx* c, const double* phi_dev, void* ex, void* ey, void* ez, int out_fp32) {
  if (!c || !phi_dev || !ex || !ey || !ez) return GMG_ERR_ARG;
  const LevelData& F = c->fine();
  const gmg_params& p = c->p;
  return (prof_field(c, F.g, p.lx / p.nx, p.ly / p.ny, p.lz / p.nz, phi_dev, ex, ey, ez, out_fp32,
                              p.phi_bottom, p.phi_top, c->s));
}

gmg_status adjoint_coefficient_grad(gmg_ctx* c, const double* phi_dev, const double* lambda_dev,
                                    double* dlda_dev) {
  if (!c || !phi_dev || !lambda_dev || !dlda_dev) return GMG_ERR_ARG;
  const LevelData& F = c->fine();
  return (prof_adjoint_grad(c, F.g, phi_dev, lambda_dev, dlda_dev, c->p.phi_bottom, c->p.phi_top, c->s));
}

namespace {

// The host-array solve.  wait = true: returns with every copy done.  wait =
// false (pipelined): returns once the solve has finished and the field kernel
// is enqueued.  The copy-out of phi and E is held back: the next call enqueues
// it once its upload of a is done, so that the upload the set-up waits for does
// not share the link with the copy-out (both directions at once run at about
// 146 GB/s each instead of 210 and 193), and the copy-out then overlaps the
// set-up; gmg_host_wait enqueues it if no call came.  The staging arrays of phi
// and E are rewritten only after it, through the event ev_done.

// Enqueue the held-back copy-out on the copy-out stream, after the compute
// stream's work (ev_out) and, if given, after the event `after`.
gmg_status flush_pending_out(gmg_ctx* c, cudaEvent_t after) {
  auto& po = c->pend_out;
  if (!po.on) return GMG_OK;
  po.on = false;
  if (after) CK(cudaStreamWaitEvent(c->cso, after, 0));
  CK(cudaStreamWaitEvent(c->cso, c->ev_out, 0));
  CK(cudaMemcpyAsync(po.phi, c->st_phi, po.bytes, cudaMemcpyDeviceToHost, c->cso));
  if (po.ex) {
    CK(cudaMemcpyAsync(po.ex, c->st_ex, po.ebytes, cudaMemcpyDeviceToHost, c->cso));
    CK(cudaMemcpyAsync(po.ey, c->st_ey, po.ebytes, cudaMemcpyDeviceToHost, c->cso));
    CK(cudaMemcpyAsync(po.ez, c->st_ez, po.ebytes, cudaMemcpyDeviceToHost, c->cso));
  }
  CK(cudaEventRecord(c->ev_done, c->cso));
  return GMG_OK;
}

gmg_status solve_host_impl(gmg_ctx* c, const double* a_host, const double* f_host, const double* phi0_host,
                           double* phi_host, void* ex_host, void* ey_host, void* ez_host, int field_fp32,
                           gmg_solve_info* info, bool wait) {
  if (!c || !f_host || !phi_host) return GMG_ERR_ARG;
  const bool want_e = ex_host && ey_host && ez_host;
  if ((ex_host || ey_host || ez_host) && !want_e) return GMG_ERR_ARG;
  const size_t n = c->N(), bytes = n * sizeof(double);
  if (!c->st_f) {
    CKS(dalloc(c, &c->st_f, n));
    CKS(dalloc(c, &c->st_phi, n));
  }
  if (a_host && !c->st_a) CKS(dalloc(c, &c->st_a, n));
  const size_t esz = field_fp32 ? sizeof(float) : sizeof(double);
  if (want_e && c->st_fp32 != (field_fp32 ? 1 : 0)) {
    if (c->st_ex) return GMG_ERR_ARG;  // staging already sized for the other field type
    CKS(dev_alloc(c, &c->st_ex, n * esz));
    CKS(dev_alloc(c, &c->st_ey, n * esz));
    CKS(dev_alloc(c, &c->st_ez, n * esz));
    c->st_fp32 = field_fp32 ? 1 : 0;
  }
  if (!c->cs) {
    CK(cudaStreamCreateWithFlags(&c->cs, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&c->cso, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&c->ev_a, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&c->ev_done, cudaEventDisableTiming));
    CK(cudaEventRecord(c->ev_done, c->cso));
  }
  // The synchronous form and every error wait for all three streams, so no copy
  // touches the host arrays after the call.
  auto finish = [&](gmg_status st) {
    if (!wait && (st == GMG_OK || st == GMG_ERR_NOT_CONVERGED)) return st;
    const gmg_status ps = flush_pending_out(c, nullptr);  // an earlier call's copy-out, after an error
    if (st == GMG_OK) st = ps;
    const cudaError_t e1 = cudaStreamSynchronize(c->cs);
    const cudaError_t e2 = cudaStreamSynchronize(c->cso);
    const cudaError_t e3 = cudaStreamSynchronize(c->s);
    if (st == GMG_OK && (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess)) return GMG_ERR_CUDA;
    return st;
  };
#define CKF(...)                                       \
  do {                                                 \
    const cudaError_t e_ = (__VA_ARGS__);              \
    if (e_ != cudaSuccess) return finish(map_err(e_)); \
  } while (0)
  // Inputs on the input copy stream, after earlier work on the compute stream
  // that may still read them (ev_a): a first (the set-up needs it), then f and
  // phi0, which arrive while the set-up runs.  phi's staging array is rewritten
  // only after the previous call's copy-out of it (ev_done).
  CKF(cudaEventRecord(c->ev_a, c->s));
  CKF(cudaStreamWaitEvent(c->cs, c->ev_a, 0));
  if (a_host) {
    CKF(cudaMemcpyAsync(c->st_a, a_host, bytes, cudaMemcpyHostToDevice, c->cs));
    CKF(cudaEventRecord(c->ev_a, c->cs));
    CKF(cudaStreamWaitEvent(c->s, c->ev_a, 0));
  }
  // the previous pipelined call's copy-out, after this call's upload of a
  {
    const gmg_status ps = flush_pending_out(c, a_host ? c->ev_a : nullptr);
    if (ps != GMG_OK) return finish(ps);
  }
  CKF(cudaMemcpyAsync(c->st_f, f_host, bytes, cudaMemcpyHostToDevice, c->cs));
  CKF(cudaStreamWaitEvent(c->cs, c->ev_done, 0));
  if (phi0_host)
    CKF(cudaMemcpyAsync(c->st_phi, phi0_host, bytes, cudaMemcpyHostToDevice, c->cs));
  else
    CKF(cudaMemsetAsync(c->st_phi, 0, bytes, c->cs));
  CKF(cudaEventRecord(c->ev_in, c->cs));
  if (a_host) {
    const gmg_status bs = build(c, c->st_a);
    if (bs != GMG_OK) return finish(bs);
  }
  CKF(cudaStreamWaitEvent(c->s, c->ev_in, 0));
  gmg_status st = solve_impl(c, c->st_f, c->st_phi, 0, info);
  if (st != GMG_OK && st != GMG_ERR_NOT_CONVERGED) return finish(st);
  if (wait) {
    // phi leaves on the copy-out stream while the field kernel runs
    CKF(cudaEventRecord(c->ev_out, c->s));
    CKF(cudaStreamWaitEvent(c->cso, c->ev_out, 0));
    CKF(cudaMemcpyAsync(phi_host, c->st_phi, bytes, cudaMemcpyDeviceToHost, c->cso));
  }
  if (want_e) {
    const gmg_status fs = field_from_potential(c, c->st_phi, c->st_ex, c->st_ey, c->st_ez, field_fp32);
    if (fs != GMG_OK) return finish(fs);
    if (wait) {
      CKF(cudaEventRecord(c->ev_out, c->s));
      CKF(cudaStreamWaitEvent(c->cso, c->ev_out, 0));
      CKF(cudaMemcpyAsync(ex_host, c->st_ex, n * esz, cudaMemcpyDeviceToHost, c->cso));
      CKF(cudaMemcpyAsync(ey_host, c->st_ey, n * esz, cudaMemcpyDeviceToHost, c->cso));
      CKF(cudaMemcpyAsync(ez_host, c->st_ez, n * esz, cudaMemcpyDeviceToHost, c->cso));
    }
  }
  if (wait) {
    // the next call rewrites phi's staging array (and, after its solve, E's) only
    // once this copy-out is done: its input stream waits on ev_done
    CKF(cudaEventRecord(c->ev_done, c->cso));
  } else {
    CKF(cudaEventRecord(c->ev_out, c->s));
    c->pend_out.on = true;
    c->pend_out.phi = phi_host;
    c->pend_out.ex = want_e ? ex_host : nullptr;
    c->pend_out.ey = want_e ? ey_host : nullptr;
    c->pend_out.ez = want_e ? ez_host : nullptr;
    c->pend_out.bytes = bytes;
    c->pend_out.ebytes = n * esz;
  }
#undef CKF
  return finish(st);
}

}  // namespace

gmg_status gmg_solve_host(gmg_ctx* c, const double* a_host, const double* f_host, const double* phi0_host,
                          double* phi_host, void* ex_host, void* ey_host, void* ez_host, int field_fp32,
                          gmg_solve_info* info) {
  return solve_host_impl(c, a_host, f_host, phi0_host, phi_host, ex_host, ey_host, ez_host, field_fp32, info, true);
}

gmg_status gmg_solve_host_async(gmg_ctx* c, const double* a_host, const double* f_host, const double* phi0_host,
                                double* phi_host, void* ex_host, void* ey_host, void* ez_host, int field_fp32,
                                gmg_solve_info* info) {
  return solve_host_impl(c, a_host, f_host, phi0_host, phi_host, ex_host, ey_host, ez_host, field_fp32, info,
                         false);
}

gmg_status gmg_host_wait(gmg_ctx* c) {
  if (!c) return GMG_ERR_ARG;
  if (!c->cs) return GMG_OK;  // no host-array solve yet
  const gmg_status ps = flush_pending_out(c, nullptr);
  const cudaError_t e1 = cudaStreamSynchronize(c->cs);
  const cudaError_t e2 = cudaStreamSynchronize(c->cso);
  const cudaError_t e3 = cudaStreamSynchronize(c->s);
  if (ps != GMG_OK) return ps;
  if (e1 != cudaSuccess) return map_err(e1);
  if (e2 != cudaSuccess) return map_err(e2);
  return e3 == cudaSuccess ? GMG_OK : map_err(e3);
}

gmg_status assemble_coefficient_rhs(const gmg_params* p, const double* ne_dev, const double* np_dev,
                                    const gmg_density_coef* dc, double* a_dev, double* f_dev, void* stream) {
  if (!p || !ne_dev || !np_dev || !dc || !a_dev || !f_dev) return GMG_ERR_ARG;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1 || !(p->lx > 0) || !(p->ly > 0) || !(p->lz > 0)) return GMG_ERR_ARG;
  if (a_dev == ne_dev || a_dev == np_dev || f_dev == ne_dev || f_dev == np_dev || a_dev == f_dev)
    return GMG_ERR_ARG;
  const double k[] = {dc->tau, dc->mu_e, dc->mu_p, dc->diff_x, dc->diff_y, dc->diff_z, dc->e_over_eps0};
  for (double v : k)
    if (!std::isfinite(v)) return GMG_ERR_ARG;
  if (dc->tau < 0) return GMG_ERR_ARG;
  const Grid3 g = make_grid(p->nx, p->ny, p->nz, p->lx, p->ly, p->lz);
  const double hx = p->lx / p->nx, hy = p->ly / p->ny, hz = p->lz / p->nz;
  DensityCoef d;
  d.half_tau_e_eps0_mu_e = dc->e_over_eps0 * 0.5 * dc->tau * std::fabs(dc->mu_e);
  d.half_tau_e_eps0_mu_p = dc->e_over_eps0 * 0.5 * dc->tau * std::fabs(dc->mu_p);
  d.e_over_eps0 = dc->e_over_eps0;
  d.half_tau = 0.5 * dc->tau;
  d.dx_ih2 = dc->diff_x / (hx * hx);
  d.dy_ih2 = dc->diff_y / (hy * hy);
  d.dz_ih2 = dc->diff_z / (hz * hz);
  const cudaError_t e = launch_assemble(g, d, ne_dev, np_dev, a_dev, f_dev, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? GMG_OK : map_err(e);
}

namespace {

// Validates the grid and constants of a transport call and fills the kernel's
// coefficients (mobility magnitudes, alpha's constants times the pressure,
// 1/h^2, 1/(2h), D/h^2).
gmg_status transport_coef(const gmg_params* p, const gmg_transport_coef* tc, double cstage, Grid3* g,
                          TransportCoef* t) {
  if (p->nx < 1 || p->ny < 1 || p->nz < 1 || !(p->lx > 0) || !(p->ly > 0) || !(p->lz > 0)) return GMG_ERR_ARG;
  if ((size_t)p->nx * (size_t)p->ny >= (size_t)1 << 31) return GMG_ERR_ARG;  // one plane indexed in 32 bits
  const double k[] = {tc->mu_e, tc->mu_p, tc->diff_x, tc->diff_y, tc->diff_z, tc->ion_a, tc->ion_b, tc->pressure,
                      cstage, p->phi_bottom, p->phi_top};
  for (double v : k)
    if (!std::isfinite(v)) return GMG_ERR_ARG;
  *g = make_grid(p->nx, p->ny, p->nz, p->lx, p->ly, p->lz);
  const double hx = p->lx / p->nx, hy = p->ly / p->ny, hz = p->lz / p->nz;
  t->mu_e = std::fabs(tc->mu_e);
  t->mu_p = std::fabs(tc->mu_p);
  t->diff_x = tc->diff_x;
  t->diff_y = tc->diff_y;
  t->diff_z = tc->diff_z;
  t->ion_ap = tc->ion_a * tc->pressure;
  t->ion_bp = tc->ion_b * tc->pressure;
  t->g_bottom = p->phi_bottom;
  t->g_top = p->phi_top;
  t->kx = 1.0 / (hx * hx);
  t->ky = 1.0 / (hy * hy);
  t->kz = 1.0 / (hz * hz);
  t->ih2x = 0.5 / hx;
  t->ih2y = 0.5 / hy;
  t->ih2z = 0.5 / hz;
  t->dih2x = tc->diff_x / (hx * hx);
  t->dih2y = tc->diff_y / (hy * hy);
  t->dih2z = tc->diff_z / (hz * hz);
  t->dmx = t->mu_e > 0.0 ? tc->diff_x / t->mu_e : 0.0;
  t->dmy = t->mu_e > 0.0 ? tc->diff_y / t->mu_e : 0.0;
  t->dmz = t->mu_e > 0.0 ? tc->diff_z / t->mu_e : 0.0;
  return GMG_OK;
}

}  // namespace

gmg_status transport_stage(const gmg_params* p, const double* base_e, const double* base_p,
                           const double* eval_e, const double* eval_p, const double* phi,
                           const gmg_transport_coef* tc, double cstage, double* out_e, double* out_p, void* stream) {
  if (!p || !base_e || !base_p || !eval_e || !eval_p || !phi || !tc || !out_e || !out_p) return GMG_ERR_ARG;
  const void* ins[] = {eval_e, eval_p, phi};
  for (const void* q : ins)
    if (q == out_e || q == out_p) return GMG_ERR_ARG;
  if (out_e == out_p || base_e == out_p || base_p == out_e) return GMG_ERR_ARG;
  Grid3 g;
  TransportCoef t;
  const gmg_status st = transport_coef(p, tc, cstage, &g, &t);
  if (st != GMG_OK) return st;
  const cudaError_t e = launch_transport(g, t, base_e, base_p, eval_e, eval_p, phi, cstage, out_e, out_p, nullptr, 0,
                                         static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? GMG_OK : map_err(e);
}

gmg_status transport_step(const gmg_params* p, const double* n_e, const double* n_p, const double* phi,
                          const gmg_transport_coef* tc, double tau, double* half_e, double* half_p, double* out_e,
                          double* out_p, double* rate, void* stream) {
  if (!p || !n_e || !n_p || !phi || !tc || !half_e || !half_p || !out_e || !out_p || !rate) return GMG_ERR_ARG;
  // half_* and rate are written while n_*, phi (and half_* in the corrector) are read
  const void* w[] = {half_e, half_p, rate};
  const void* r[] = {n_e, n_p, phi, out_e, out_p};
  for (int a = 0; a < 3; ++a) {
    for (const void* q : r)
      if (q == w[a]) return GMG_ERR_ARG;
    for (int b = a + 1; b < 3; ++b)
      if (w[a] == w[b]) return GMG_ERR_ARG;
  }
  if (out_e == out_p || out_e == phi || out_p == phi || out_e == n_p || out_p == n_e) return GMG_ERR_ARG;
  Grid3 g;
  TransportCoef t;
  gmg_status st = transport_coef(p, tc, tau, &g, &t);
  if (st != GMG_OK) return st;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = launch_transport(g, t, n_e, n_p, n_e, n_p, phi, 0.5 * tau, half_e, half_p, rate, 1, s);
  if (e == cudaSuccess) e = launch_transport(g, t, n_e, n_p, half_e, half_p, phi, tau, out_e, out_p, rate, 2, s);
  return e == cudaSuccess ? GMG_OK : map_err(e);
}

gmg_status gmg_round_to_f32(const double* src, float* dst, size_t n, void* stream) {
  if (n == 0) return GMG_OK;
  if (!src || !dst || (const void*)src == (const void*)dst) return GMG_ERR_ARG;
  const cudaError_t e = launch_cast_d2f(n, src, dst, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? GMG_OK : map_err(e);
}

gmg_status gmg_set_stream(gmg_ctx* c, void* stream) {
  if (!c) return GMG_ERR_ARG;
  CK(cudaStreamSynchronize(c->s));
  c->s = (cudaStream_t)stream;
  return GMG_OK;
}

int gmg_num_levels(const gmg_ctx* c) { return c ? (int)c->lev.size() : 0; }

gmg_status gmg_level_info(const gmg_ctx* c, int level, int* nx, int* ny, int* nz, double* lam_max,
                          double* lam_min) {
  if (!c || level < 0 || level >= (int)c->lev.size()) return GMG_ERR_ARG;
  const LevelData& L = c->lev[level];
  if (nx) *nx = L.nx;
  if (ny) *ny = L.ny;
  if (nz) *nz = L.nz;
  if (lam_max) *lam_max = L.lam_max;
  if (lam_min) *lam_min = L.lam_min;
  return GMG_OK;
}

gmg_status gmg_level_set_bounds(gmg_ctx* c, int level, double lam_max, double lam_min) {
  if (!c || level < 1 || level >= (int)c->lev.size()) return GMG_ERR_ARG;
  if (!(lam_max > lam_min) || !(lam_min > 0) || !isfinite(lam_max)) return GMG_ERR_ARG;
  LevelData& L = c->lev[level];
  L.lam_max = lam_max;
  L.lam_min = lam_min;
  return GMG_OK;
}

gmg_status gmg_level_coefficient(gmg_ctx* c, int level, double* out_dev) {
  LevelData* L = level_ptr(c, level);
  if (!L || !out_dev || L->faces) return GMG_ERR_ARG;
  return (prof_copy_d(c, L->n, L->a64, out_dev, c->s));
}

gmg_status gmg_level_faces(gmg_ctx* c, int level, double* kx, double* ky, double* kz, double* ktop) {
  LevelData* L = level_ptr(c, level);
  if (!L || !kx || !ky || !kz || !ktop) return GMG_ERR_ARG;
  if (!L->faces) return map_err(launch_faces_of_cells<double>(L->g, L->a64, kx, ky, kz, ktop, c->s));
  double* outs[4] = {kx, ky, kz, ktop};
  const size_t cnt[4] = {L->n, L->n, L->n, L->g.plane()};
  for (int q = 0; q < 4; ++q) {
    if (c->mixed) CKS(prof_cast_f2d(c, cnt[q], (const float*)L->kf + q * L->n, outs[q], c->s));
    else CKS(prof_copy_d(c, cnt[q], (const double*)L->kf + q * L->n, outs[q], c->s));
  }
  return GMG_OK;
}

gmg_status gmg_apply_preconditioner(gmg_ctx* c, const double* v_dev, double* z_dev) {
  if (!c || !v_dev || !z_dev) return GMG_ERR_ARG;
  c->fmg_now = c->p.cycle == GMG_CYCLE_FMG;
  CKS(precondition(c, v_dev, c->Z));
  if (c->mixed) return (prof_cast_f2d(c, c->N(), (const float*)c->Z, z_dev, c->s));
  return (prof_copy_d(c, c->N(), (const double*)c->Z, z_dev, c->s));
}

gmg_status gmg_krylov_solve(gmg_ctx* c, int method, const double* f_dev, double* phi_dev, int homogeneous_bc,
                            gmg_solve_info* info) {
  if (!c || !f_dev || !phi_dev) return GMG_ERR_ARG;
  switch (method) {
    case GMG_KRYLOV_FGMRES: return solve_impl(c, f_dev, phi_dev, homogeneous_bc, info, true);
    case GMG_KRYLOV_GMRES: return solve_impl(c, f_dev, phi_dev, homogeneous_bc, info, false);
    case GMG_KRYLOV_CG:
    case GMG_KRYLOV_FCG:
    case GMG_KRYLOV_CGS:
    case GMG_KRYLOV_BICGSTAB: return solve_short(c, method, f_dev, phi_dev, homogeneous_bc, info);
    default: return GMG_ERR_ARG;
  }
}

gmg_status gmg_apply_outer(gmg_ctx* c, const float* z, double* w) {
  if (!c || !z || !w || !c->mixed) return GMG_ERR_ARG;
  return apply_outer(c, z, w);
}

gmg_status gmg_level_apply(gmg_ctx* c, int level, const void* x, void* y) {
  LevelData* L = level_ptr(c, level);
  if (!L || !x || !y) return GMG_ERR_ARG;
  if (c->mixed) return lv_apply<float>(c, *L, (const float*)x, (float*)y);
  return lv_apply<double>(c, *L, (const double*)x, (double*)y);
}

gmg_status gmg_level_smooth(gmg_ctx* c, int level, const void* b, void* x, int x_is_zero) {
  LevelData* L = level_ptr(c, level);
  if (!L || level == 0 || !b || !x || !L->r) return GMG_ERR_ARG;
  // the fused kernel reads b and x as float2: other alignments take the separate kernels
  if (c->mixed && L->fused && pair_aligned(b) && pair_aligned(x)) {
    float* X = (float*)x;
    if (x_is_zero) return smooth_fused(c, level, (const float*)b, nullptr, X, L->x2);
    if (c->p.cheb_steps % 2 == 0) return smooth_fused(c, level, (const float*)b, X, X, L->x2);
    CK(cudaMemcpyAsync(L->x2, X, L->n * sizeof(float), cudaMemcpyDeviceToDevice, c->s));
    return smooth_fused(c, level, (const float*)b, L->x2, X, L->x2);
  }
  if (c->mixed) return smooth<float>(c, level, (const float*)b, (float*)x, x_is_zero != 0);
  return smooth<double>(c, level, (const double*)b, (double*)x, x_is_zero != 0);
}

gmg_status gmg_level_smoother_pc(gmg_ctx* c, int level, const void* r, void* z) {
  LevelData* L = level_ptr(c, level);
  if (!L || !r || !z) return GMG_ERR_ARG;
  if (c->mixed) return smoother_pc<float>(c, *L, (const float*)r, (float*)z);
  return smoother_pc<double>(c, *L, (const double*)r, (double*)z);
}

gmg_status gmg_level_residual_restrict(gmg_ctx* c, int level, const void* b, const void* x, void* coarse) {
  LevelData* L = level_ptr(c, level);
  if (!L || level == 0 || !b || !x || !coarse) return GMG_ERR_ARG;
  if (c->mixed) return lv_residual_restrict<float>(c, *L, (const float*)b, (const float*)x, (float*)coarse);
  return lv_residual_restrict<double>(c, *L, (const double*)b, (const double*)x, (double*)coarse);
}

gmg_status gmg_level_prolong_add(gmg_ctx* c, int level, const void* e, void* x) {
  LevelData* L = level_ptr(c, level);
  if (!L || level == 0 || !e || !x) return GMG_ERR_ARG;
  if (c->mixed) return lv_prolong<float>(c, *L, (const float*)e, (float*)x);
  return lv_prolong<double>(c, *L, (const double*)e, (double*)x);
}

gmg_status gmg_coarse_solve(gmg_ctx* c, const void* b, void* x) {
  if (!c || !b || !x) return GMG_ERR_ARG;
  if (c->mixed) return (prof_coarse_apply<float>(c, c->nc, c->cinv64, (const float*)b, (float*)x, c->s));
  return (prof_coarse_apply<double>(c, c->nc, c->cinv64, (const double*)b, (double*)x, c->s));
}

gmg_status gmg_hessenberg_max_real_eig(const double* h_host, int m, double* out) {
  if (!h_host || !out || m < 1 || m > 64) return GMG_ERR_ARG;
  std::vector<double> H(h_host, h_host + (size_t)m * m), wr, wi;
  if (hessenberg_eigs(H, m, wr, wi) != 0) return GMG_ERR_BREAKDOWN;
  double lam = -INFINITY;
  for (int i = 0; i < m; ++i) lam = std::max(lam, wr[i]);
  *out = lam;
  return GMG_OK;
}

void gmg_test_fail_allocation_after(int n) { g_fail_alloc_countdown = n > 0 ? n : 0; }

gmg_status gmg_profile_enable(gmg_ctx* c, int on) {
  if (!c) return GMG_ERR_ARG;
  CK(cudaStreamSynchronize(c->s));
  prof_collect(c);
  c->prof_on = on != 0;
  return GMG_OK;
}

gmg_status gmg_profile_min_bytes(gmg_ctx* c, double min_bytes) {
  if (!c || !(min_bytes >= 0.0)) return GMG_ERR_ARG;
  c->prof_min_bytes = min_bytes;
  return GMG_OK;
}

gmg_status gmg_profile_reset(gmg_ctx* c) {
  if (!c) return GMG_ERR_ARG;
  CK(cudaStreamSynchronize(c->s));
  prof_collect(c);
  for (int k = 0; k < NK; ++k) {
    c->k_ms[k] = c->k_bytes[k] = 0.0;
    c->k_launch[k] = c->k_timed[k] = 0;
  }
  return GMG_OK;
}

int gmg_profile_num_kernels(void) { return NK; }

gmg_status gmg_profile_get(gmg_ctx* c, int k, const char** name, long long* launches, long long* timed_launches,
                           double* total_ms, double* total_bytes) {
  if (!c || k < 0 || k >= NK) return GMG_ERR_ARG;
  CK(cudaStreamSynchronize(c->s));
  prof_collect(c);
  if (name) *name = kKernelNames[k];
  if (launches) *launches = c->k_launch[k];
  if (timed_launches) *timed_launches = c->k_timed[k];
  if (total_ms) *total_ms = c->k_ms[k];
  if (total_bytes) *total_bytes = c->k_bytes[k];
  return GMG_OK;
}

}  // extern "C"
