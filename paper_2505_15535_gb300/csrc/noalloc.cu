// A variant of the FP64 Jacobi-CG linear solve that allocates nothing.
//
// Some callers cannot call cudaMalloc at the point where they need a solve: code that runs
// under a memory pool or budget that owns all device memory, code that must not trigger the
// implicit device synchronisation of cudaMalloc/cudaFree in a latency-sensitive loop, and
// plugins whose host forbids allocation after start-up.  nhmf_linear_solve keeps its work
// vectors in the context and allocates them on first use; this entry point instead keeps
// them in one file-scope __device__ array of fixed size.  nhmf_create resolves the array's
// device address (which loads this file's module, and with it the array, on that device), so
// after nhmf_create and nhmf_set_linearization (which may allocate, at set-up time) no
// further allocation occurs.
#include <cmath>

#include "blas.h"
#include "internal.h"

namespace nhmf {
namespace {

// Scratch: 6 FP64 vectors of up to kNoAllocMaxDofs entries (r, z, p, q, diagonal, inverse
// diagonal / true-residual workspace), the reduction partials and 8 scalars; 6.3 MB on
// every device on which a context was created, held until the process exits.
constexpr long long kNoAllocMaxDofs = 131072;
constexpr long long kVec = kNoAllocMaxDofs;
constexpr long long kScratchDoubles = 6 * kVec + kPartialSlots + 8;
static __device__ __align__(256) double g_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
double* g_scratch_ptr[kMaxDevices] = {};

nhmf_status read_dev(nhmf_ctx* c, const double* d, double* h, cudaStream_t s) {
  nhmf_status st = cuda_check(c, cudaMemcpyAsync(h, d, sizeof(double), cudaMemcpyDeviceToHost, s), "noalloc: read");
  if (st == NHMF_OK) st = cuda_check(c, cudaStreamSynchronize(s), "noalloc: sync");
  return st;
}

}  // namespace

// Device address of g_scratch on the context's device (current during nhmf_create).  In host
// code the symbol is a host-side stand-in, never a device address: it is translated once per
// device, and the lookup loads the array on that device.
nhmf_status noalloc_setup(nhmf_ctx* c) {
  const int dev = c->device;
  if (dev < 0 || dev >= kMaxDevices) return fail(c, NHMF_ERR_ARG, "noalloc: device index out of range");
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaError_t e = cudaGetSymbolAddress(&p, g_scratch); e != cudaSuccess)
      return cuda_check(c, e, "noalloc: cudaGetSymbolAddress");
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  return NHMF_OK;
}

}  // namespace nhmf

using namespace nhmf;

extern "C" nhmf_status nhmf_linear_solve_noalloc(nhmf_ctx* c, int strategy, double rtol, int max_iter,
                                                  const double* b, double* x, long long* iters, double* rel_res,
                                                  void* stream) {
  if (!c) return NHMF_ERR_ARG;
  // x aliasing b would be zeroed together with it below and look like a converged solve
  if (!b || !x || (const void*)b == (void*)x || !iters || !rel_res || max_iter < 1 || !(rtol > 0.0) ||
      (strategy != NHMF_ON_THE_FLY && strategy != NHMF_CACHED))
    return fail(c, NHMF_ERR_ARG, "linear_solve_noalloc: bad argument");
  const long long n = 3 * c->g.M3;
  if (n > kNoAllocMaxDofs)
    return fail(c, NHMF_ERR_ARG, "linear_solve_noalloc: " + std::to_string(n) + " DoFs exceed the static scratch limit of " +
                                     std::to_string(kNoAllocMaxDofs) + " DoFs");
  if (!c->have_lin) return fail(c, NHMF_ERR_STATE, "linear_solve_noalloc: no linearisation point set");
  if (strategy == NHMF_CACHED && !c->cache64) return fail(c, NHMF_ERR_STATE, "linear_solve_noalloc: no FP64 point cache");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = -1;
  if (cudaError_t e = cudaGetDevice(&dev); e != cudaSuccess) return cuda_check(c, e, "linear_solve_noalloc: cudaGetDevice");
  if (dev != c->device)
    return fail(c, NHMF_ERR_STATE, "linear_solve_noalloc: the current device is not the context's device");
  double* base = g_scratch_ptr[dev];  // resolved by nhmf_create
  if (!base) return fail(c, NHMF_ERR_STATE, "linear_solve_noalloc: scratch address not resolved");
  nhmf_status st = NHMF_OK;
  double *r = base, *z = base + kVec, *p = base + 2 * kVec, *q = base + 3 * kVec, *diag = base + 4 * kVec,
         *dinv = base + 5 * kVec, *partials = base + 6 * kVec, *sc = partials + kPartialSlots;
  const bool profiling = c->profiling;  // event creation is an allocation: keep it off here
  c->profiling = false;
  auto done = [&](nhmf_status v) {
    c->profiling = profiling;
    return v;
  };
  // scalars and partials keep the previous call's values: start from zero
  if ((st = cuda_check(c, cudaMemsetAsync(partials, 0, (kPartialSlots + 8) * sizeof(double), s), "noalloc: clear")) != NHMF_OK)
    return done(st);
  if ((st = launch_diagonal(c, diag, s)) != NHMF_OK) return done(st);
  reciprocal(n, diag, dinv, nullptr, s);
  double bnh = 0.0;
  norm2(n, b, sc + 4, partials, s);
  if ((st = read_dev(c, sc + 4, &bnh, s)) != NHMF_OK) return done(st);
  if ((st = cuda_check(c, cudaMemsetAsync(x, 0, n * sizeof(double), s), "noalloc: clear x")) != NHMF_OK)
    return done(st);
  *iters = 0;
  *rel_res = 0.0;
  if (!(bnh > 0.0)) return done(bnh == 0.0 ? NHMF_OK : fail(c, NHMF_ERR_NONFINITE, "linear_solve_noalloc: non-finite b"));
  if ((st = cuda_check(c, cudaMemcpyAsync(r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s), "noalloc: r = b")) !=
      NHMF_OK)
    return done(st);
  jacobi<double>(n, r, dinv, z, sc + 0, sc + 3, partials, s);
  pcg_direction<double>(n, sc + 0, nullptr, z, p, s);
  // the reciprocal, Jacobi and direction launches above: fail here, not after max_iter steps
  if ((st = cuda_check(c, cudaGetLastError(), "noalloc: set-up launches")) != NHMF_OK) return done(st);
  long long k = 0;
  double rrh = bnh * bnh;
  while (k < max_iter) {
    if ((st = launch_apply(c, NHMF_FP64, strategy, p, q, s)) != NHMF_OK) return done(st);
    dot(n, p, q, sc + 2, partials, s);
    pcg_update<double>(n, sc + (k & 1), sc + 2, x, r, p, q, dinv, z, sc + ((k + 1) & 1), sc + 3, partials, c->status, s);
    pcg_direction<double>(n, sc + ((k + 1) & 1), sc + (k & 1), z, p, s);
    ++k;
    if (k % 10 == 0 || k == max_iter) {
      if ((st = read_dev(c, sc + 3, &rrh, s)) != NHMF_OK) return done(st);
      if (!std::isfinite(rrh)) return done(fail(c, NHMF_ERR_NONFINITE, "linear_solve_noalloc: non-finite residual"));
      if (std::sqrt(rrh) <= rtol * bnh) break;
    }
  }
  *iters = k;
  if ((st = nhmf_check_status(c, stream)) != NHMF_OK) return done(st);
  // true relative residual ||b - A x|| / ||b||, with dinv's slot as workspace
  if ((st = launch_apply(c, NHMF_FP64, strategy, x, dinv, s)) != NHMF_OK) return done(st);
  axpby(n, 1.0, nullptr, b, -1.0, nullptr, dinv, s);
  double rn = 0.0;
  norm2(n, dinv, sc + 5, partials, s);
  if ((st = read_dev(c, sc + 5, &rn, s)) != NHMF_OK) return done(st);
  *rel_res = rn / bnh;
  return done(cuda_check(c, cudaGetLastError(), "linear_solve_noalloc"));
}
