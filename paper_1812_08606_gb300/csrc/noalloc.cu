// Coarsest-grid direct solve that allocates no memory.
//
// Some callers cannot allocate device memory: code whose device memory is
// wholly reserved up front by a framework's pool, real-time loops that must
// not take the implicit device-wide synchronisation (or the out-of-memory
// failure) of cudaMalloc, and embedded or library code that runs under a
// fixed memory budget.  For them this file provides the dense direct solve of
// the coarsest multigrid grid with its scratch -- the dense operator, the
// triangular-inverse workspace and the explicit inverse -- in one file-scope
// __device__ array of fixed size.  Every GPU that loads the library holds the
// array until the process exits.
//
// The array is shared by every call: a call overwrites all of it before
// reading it, and calls that overlap on the GPU (two streams, two host
// threads) race on it.
#include <cmath>

#include "../../include/gmg.h"
#include "gmg_internal.cuh"

using namespace gmg;

namespace {

constexpr int NMAX = GMG_NOALLOC_MAX_UNKNOWNS;
constexpr size_t MAT = (size_t)NMAX * NMAX;
// dense operator / Cholesky factor, inverse of the factor, explicit inverse, status word
constexpr size_t SCRATCH_DOUBLES = 3 * MAT + 32;

static __device__ __align__(256) double g_noalloc_scratch[SCRATCH_DOUBLES];

// Device address of the scratch array on the current device.  Looked up on
// every call, with the calling device current: the lookup is cheap, and a
// cached address would go stale if the module were loaded again (for
// instance after cudaDeviceReset).
cudaError_t scratch_address(double** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<double*>(p);
  return cudaSuccess;
}

gmg_status to_status(cudaError_t e) {
  if (e == cudaSuccess) return GMG_OK;
  (void)cudaGetLastError();
  return GMG_ERR_CUDA;
}

}  // namespace

extern "C" gmg_status gmg_coarse_solve_noalloc(const gmg_params* p, const double* a_dev, const double* b_dev,
                                               double* x_dev, void* stream) {
  if (!p || !a_dev || !b_dev || !x_dev) return GMG_ERR_ARG;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return GMG_ERR_ARG;
  if (!(p->lx > 0) || !(p->ly > 0) || !(p->lz > 0)) return GMG_ERR_ARG;
  if (!std::isfinite(p->lx) || !std::isfinite(p->ly) || !std::isfinite(p->lz)) return GMG_ERR_ARG;
  const long long n = (long long)p->nx * p->ny * p->nz;
  if (n > NMAX) return GMG_ERR_ARG;  // beyond the fixed scratch: nx*ny*nz <= GMG_NOALLOC_MAX_UNKNOWNS
  double* scratch = nullptr;
  gmg_status st = to_status(scratch_address(&scratch));
  if (st != GMG_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* A = scratch;            // n x n operator, then its Cholesky factor in place
  double* W = scratch + MAT;      // inverse of the factor
  double* Ainv = scratch + 2 * MAT;
  int* status = reinterpret_cast<int*>(scratch + 3 * MAT);
  const Grid3 g = make_grid(p->nx, p->ny, p->nz, p->lx, p->ly, p->lz);
  if ((st = to_status(launch_coarse_assemble(g, a_dev, A, s))) != GMG_OK) return st;
  if ((st = to_status(launch_coarse_factor((int)n, A, W, Ainv, nullptr, status, s))) != GMG_OK) return st;
  int host_status = -1;
  if ((st = to_status(cudaMemcpyAsync(&host_status, status, sizeof(int), cudaMemcpyDeviceToHost, s))) != GMG_OK)
    return st;
  if ((st = to_status(cudaStreamSynchronize(s))) != GMG_OK) return st;
  if (host_status != 0) return GMG_ERR_BREAKDOWN;  // the operator is not positive definite (a <= 0 somewhere)
  return to_status(launch_coarse_apply<double>((int)n, Ainv, b_dev, x_dev, s));
}
