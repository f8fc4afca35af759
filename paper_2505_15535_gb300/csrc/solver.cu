// Newton's method with load steps and the Krylov solvers on the matrix-free operator
// (Sections 2.1-2.3).  Host code drives device kernels; every vector operation, reduction
// and scalar of the iterations lives on the device, and the host reads the residual norm
// only every `check_every` iterations.
#include <chrono>
#include <cmath>
#include <limits>
#include <type_traits>
#include <vector>

#include "blas.h"
#include "gmg.h"
#include "internal.h"
#include "unet.h"

namespace nhmf {
namespace {

// Dirichlet data of a load step: mode 0 writes d = g - u on constrained DoFs (0 elsewhere
// is the caller's memset); mode 1 sets u = g there.  g = top_uz for u_z on z = 1 of the
// compression preset, 0 elsewhere.
__global__ void k_bc(int bc, int M, long long M3, double top_uz, double* u, double* d, int mode) {
  const long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long M2 = (long long)M * M;
  if (f >= M2) return;
  const int x = int(f % M), y = int(f / M);
  auto set = [&](int c, long long node, double g) {
    const long long i = c * M3 + node;
    if (mode == 0)
      d[i] = g - u[i];
    else
      u[i] = g;
  };
  if (bc == NHMF_BC_CLAMP_X0) {
    const long long node = (long long)M * (x + (long long)M * y);
    for (int c = 0; c < 3; ++c) set(c, node, 0.0);
  } else if (bc == NHMF_BC_COMPRESSION) {
    const long long bottom = x + (long long)M * y;
    for (int c = 0; c < 3; ++c) set(c, bottom, 0.0);
    set(2, bottom + M2 * (M - 1), top_uz);
  }
}

enum Slot { CT = 24, CAC = 25, OMEGA = 26, CNORM = 27,  // the learned correction's step length
            RZ0 = 0, RZ1 = 1, PQ = 2, RR = 3, BN = 4, ALPHA = 5, BETA = 6, ZQ = 7, PR = 8, PQPREV = 9,
            RNORM = 10, TMP = 11, IN_RZ0 = 16, IN_RZ1 = 17, IN_PQ = 18, IN_RR = 19, IN_BN = 20 };

struct Ctx {
  nhmf_ctx* c;
  cudaStream_t s;
  long long n;
  SolverWork& w;
  int outer = NHMF_FP64;  // arithmetic of the flexible solvers' outer applies (FP64 or DF64)
};

}  // namespace

nhmf_status ensure_work(nhmf_ctx* c) {
  const long long n = 3 * c->g.M3;
  if (c->work && c->work->n == n) return NHMF_OK;
  free_work(c);
  c->work = new SolverWork();
  SolverWork& w = *c->work;
  w.n = n;
  double** d64[] = {&w.r, &w.z, &w.p, &w.q, &w.qprev, &w.x, &w.b, &w.R, &w.d, &w.t, &w.du, &w.utry, &w.diag, &w.dinv,
                    &w.b2, &w.x2};
  for (double** p : d64)
    if (cudaMalloc(p, n * sizeof(double)) != cudaSuccess) return fail(c, NHMF_ERR_OOM, "solver work alloc");
  float** d32[] = {&w.r32, &w.z32, &w.p32, &w.q32, &w.x32, &w.b32, &w.dinv32};
  for (float** p : d32)
    if (cudaMalloc(p, n * sizeof(float)) != cudaSuccess) return fail(c, NHMF_ERR_OOM, "solver work alloc");
  if (cudaMalloc(&w.sc, 64 * sizeof(double)) != cudaSuccess) return fail(c, NHMF_ERR_OOM, "solver scalars");
  if (cudaMalloc(&w.partials, kPartialSlots * sizeof(double)) != cudaSuccess) return fail(c, NHMF_ERR_OOM, "partials");
  if (cudaMallocHost(&w.host, 8 * sizeof(double)) != cudaSuccess) return fail(c, NHMF_ERR_OOM, "pinned scalar");
  cudaMemset(w.sc, 0, 64 * sizeof(double));
  if (cudaStreamCreateWithFlags(&w.stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&w.ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&w.ev_out, cudaEventDisableTiming) != cudaSuccess)
    return fail(c, NHMF_ERR_CUDA, "solver stream");
  return NHMF_OK;
}

namespace {

nhmf_status read_scalar(Ctx& x, const double* dev, double* out) {
  nhmf_status st = cuda_check(x.c, cudaMemcpyAsync(x.w.host, dev, sizeof(double), cudaMemcpyDeviceToHost, x.s), "scalar read");
  if (st == NHMF_OK) st = cuda_check(x.c, cudaStreamSynchronize(x.s), "scalar sync");
  *out = x.w.host[0];
  return st;
}

nhmf_status norm(Ctx& x, const double* v, int slot, double* out) {
  norm2(x.n, v, x.w.sc + slot, x.w.partials, x.s);
  return read_scalar(x, x.w.sc + slot, out);
}

// Jacobi-preconditioned CG from x = 0 on A in precision T.  Scalars use slots base..base+4.
struct NoSnap {
  void operator()(long long, const void*, const void*) const {}
};

template <typename T> struct Prec;
template <> struct Prec<double> { static constexpr int id = NHMF_FP64; };
template <> struct Prec<float> { static constexpr int id = NHMF_FP32; };

// `chunk` (even) PCG iterations starting at an even iteration count, as plain launches.
template <typename T>
nhmf_status pcg_chunk(Ctx& x, int strat, T* sol, T* r, T* z, T* p, T* q, const T* dinv, double* rz0, double* rz1,
                      double* pq, double* rr, int chunk) {
  nhmf_status st = NHMF_OK;
  double* rz[2] = {rz0, rz1};
  for (int j = 0; j < chunk; ++j) {
    if ((st = launch_apply(x.c, Prec<T>::id, strat, p, q, x.s)) != NHMF_OK) return st;
    dot(x.n, p, q, pq, x.w.partials, x.s);
    pcg_update<T>(x.n, rz[j & 1], pq, sol, r, p, q, dinv, z, rz[(j + 1) & 1], rr, x.w.partials, x.c->status, x.s);
    pcg_direction<T>(x.n, rz[(j + 1) & 1], rz[j & 1], z, p, x.s);
  }
  return st;
}

// The CUDA graph of one chunk for these buffers (captured on first use and whenever a buffer
// or the linearisation state changed); null if capture is not possible.
template <typename T>
cudaGraphExec_t chunk_graph(Ctx& x, int strat, T* sol, T* r, T* z, T* p, T* q, const T* dinv, double* rz0,
                            double* rz1, double* pq, double* rr, int chunk) {
  nhmf_ctx* c = x.c;
  SolverWork::Graph& G = x.w.graph[sizeof(T) == 4 ? 1 : 0];
  const void* key[16] = {sol, r, z, p, q, dinv, rz0, rz1, pq, rr, (const void*)(long long)chunk,
                         (const void*)(long long)strat, c->ubar, c->ubar32, c->cache64, c->cache32};
  bool same = G.exec != nullptr;
  for (int i = 0; i < 16 && same; ++i) same = G.key[i] == key[i];
  if (same) return G.exec;
  if (G.exec) {
    cudaGraphExecDestroy(G.exec);
    G.exec = nullptr;
  }
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(x.s, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  const nhmf_status st = pcg_chunk<T>(x, strat, sol, r, z, p, q, dinv, rz0, rz1, pq, rr, chunk);
  const cudaError_t e = cudaStreamEndCapture(x.s, &graph);
  if (st != NHMF_OK || e != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return nullptr;
  }
  cudaGraphExec_t exec = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  G.exec = exec;
  for (int i = 0; i < 16; ++i) G.key[i] = key[i];
  return exec;
}

template <typename T, class Snap = NoSnap>
nhmf_status pcg(Ctx& x, int strat, const T* b, T* sol, const T* dinv, T* r, T* z, T* p, T* q, double rtol,
                int maxit, int check_every, int base, long long* iters, double* relres, Snap snap = Snap()) {
  nhmf_ctx* c = x.c;
  double* sc = x.w.sc;
  double* rz[2] = {sc + base + 0, sc + base + 1};
  double* pq = sc + base + 2;
  double* rr = sc + base + 3;
  double* bn = sc + base + 4;
  norm2(x.n, b, bn, x.w.partials, x.s);
  double bnh;
  nhmf_status st = read_scalar(x, bn, &bnh);
  if (st != NHMF_OK) return st;
  cudaMemsetAsync(sol, 0, x.n * sizeof(T), x.s);
  *iters = 0;
  *relres = 0.0;
  if (!(bnh > 0.0)) return bnh == 0.0 ? NHMF_OK : fail(c, NHMF_ERR_NONFINITE, "pcg: non-finite right-hand side");
  cudaMemcpyAsync(r, b, x.n * sizeof(T), cudaMemcpyDeviceToDevice, x.s);
  jacobi<T>(x.n, r, dinv, z, rz[0], rr, x.w.partials, x.s);
  pcg_direction<T>(x.n, rz[0], nullptr, z, p, x.s);
  long long k = 0;
  double rrh = bnh * bnh;
  // chunks of check_every iterations replay one CUDA graph (not while recording snapshots)
  const bool graphs = std::is_same<Snap, NoSnap>::value && !c->profiling && check_every % 2 == 0;
  while (graphs && k + check_every <= maxit) {
    cudaGraphExec_t exec = chunk_graph<T>(x, strat, sol, r, z, p, q, dinv, rz[0], rz[1], pq, rr, check_every);
    if (!exec) break;
    if ((st = cuda_check(c, cudaGraphLaunch(exec, x.s), "pcg graph")) != NHMF_OK) return st;
    k += check_every;
    if ((st = read_scalar(x, rr, &rrh)) != NHMF_OK) return st;
    if (!std::isfinite(rrh)) return fail(c, NHMF_ERR_NONFINITE, "pcg: non-finite residual");
    if (std::sqrt(rrh) <= rtol * bnh) {
      *iters = k;
      *relres = std::sqrt(rrh) / bnh;
      return nhmf_check_status(c, x.s);
    }
  }
  if (k % 2 == 1) std::swap(rz[0], rz[1]);  // keep the parity convention below
  while (k < maxit) {
    if ((st = launch_apply(c, Prec<T>::id, strat, p, q, x.s)) != NHMF_OK) return st;
    dot(x.n, p, q, pq, x.w.partials, x.s);
    pcg_update<T>(x.n, rz[k & 1], pq, sol, r, p, q, dinv, z, rz[(k + 1) & 1], rr, x.w.partials, c->status, x.s);
    pcg_direction<T>(x.n, rz[(k + 1) & 1], rz[k & 1], z, p, x.s);
    ++k;
    snap(k, r, sol);
    if (k % check_every == 0 || k == maxit) {
      if ((st = read_scalar(x, rr, &rrh)) != NHMF_OK) return st;
      if (!std::isfinite(rrh)) return fail(c, NHMF_ERR_NONFINITE, "pcg: non-finite residual");
      if (std::sqrt(rrh) <= rtol * bnh) break;
    }
  }
  *iters = k;
  *relres = std::sqrt(rrh) / bnh;
  return nhmf_check_status(c, x.s);
}

// Flexible CG (Notay's FCG with one-term A-orthogonalisation) in FP64 from x = 0:
//   z = M(r); p = z - (z.q_prev / p_prev.q_prev) p_prev; alpha = p.r / p.q.
// Returns NHMF_ERR_NOT_CONVERGED (with sol, w.r the current iterate and residual) when the
// residual drops by less than stall_factor over stall_window iterations or maxit is reached.
template <class Precond>
nhmf_status fcg(Ctx& x, int strat, const double* b, double* sol, double rtol, int maxit, Precond&& precond,
                long long* iters, double* relres, int stall_window = 0, double stall_factor = 1.0) {
  nhmf_ctx* c = x.c;
  SolverWork& w = x.w;
  double* sc = w.sc;
  double bnh;
  nhmf_status st = norm(x, b, BN, &bnh);
  if (st != NHMF_OK) return st;
  cudaMemsetAsync(sol, 0, x.n * sizeof(double), x.s);
  *iters = 0;
  *relres = 0.0;
  if (!(bnh > 0.0)) return bnh == 0.0 ? NHMF_OK : fail(c, NHMF_ERR_NONFINITE, "fcg: non-finite right-hand side");
  cudaMemcpyAsync(w.r, b, x.n * sizeof(double), cudaMemcpyDeviceToDevice, x.s);
  double* q = w.q;
  double* qprev = w.qprev;
  double rn = bnh;
  long long k = 0;
  std::vector<double> hist;
  hist.push_back(bnh);
  for (; k < maxit;) {
    if ((st = precond(w.r, w.z)) != NHMF_OK) return st;
    if (k == 0) {
      cudaMemcpyAsync(w.p, w.z, x.n * sizeof(double), cudaMemcpyDeviceToDevice, x.s);
    } else {
      dot(x.n, w.z, qprev, sc + ZQ, w.partials, x.s);
      ratio(sc + ZQ, sc + PQPREV, -1.0, sc + BETA, x.s);
      axpby(x.n, 1.0, nullptr, w.z, 1.0, sc + BETA, w.p, x.s);
    }
    if ((st = launch_apply(c, x.outer, strat, w.p, q, x.s)) != NHMF_OK) return st;
    dot(x.n, w.p, q, sc + PQ, w.partials, x.s);
    dot(x.n, w.p, w.r, sc + PR, w.partials, x.s);
    ratio(sc + PR, sc + PQ, 1.0, sc + ALPHA, x.s);
    axpby(x.n, 1.0, sc + ALPHA, w.p, 1.0, nullptr, sol, x.s);
    axpby(x.n, -1.0, sc + ALPHA, q, 1.0, nullptr, w.r, x.s);
    cudaMemcpyAsync(sc + PQPREV, sc + PQ, sizeof(double), cudaMemcpyDeviceToDevice, x.s);
    std::swap(q, qprev);
    ++k;
    double pqh;
    if ((st = read_scalar(x, sc + PQ, &pqh)) != NHMF_OK) return st;
    if (!(pqh > 0.0)) return fail(c, NHMF_ERR_BREAKDOWN, "fcg: p^T A p <= 0");
    if ((st = norm(x, w.r, RNORM, &rn)) != NHMF_OK) return st;
    if (!std::isfinite(rn)) return fail(c, NHMF_ERR_NONFINITE, "fcg: non-finite residual");
    hist.push_back(rn);
    if (rn <= rtol * bnh) break;
    if (stall_window > 0 && (long long)hist.size() > stall_window &&
        rn > stall_factor * hist[hist.size() - 1 - stall_window]) {
      *iters = k;
      *relres = rn / bnh;
      return NHMF_ERR_NOT_CONVERGED;
    }
  }
  *iters = k;
  *relres = rn / bnh;
  return rn <= rtol * bnh ? NHMF_OK : NHMF_ERR_NOT_CONVERGED;
}

nhmf_status update_diagonal(Ctx& x) {
  nhmf_status st = launch_diagonal(x.c, x.w.diag, x.s);
  if (st != NHMF_OK) return st;
  reciprocal(x.n, x.w.diag, x.w.dinv, x.w.dinv32, x.s);
  return cuda_check(x.c, cudaGetLastError(), "diagonal inverse");
}

// z = ||r|| * A32^{-1}(r / ||r||) approximately, by FP32 Jacobi-CG (the mixed preconditioner).
nhmf_status mixed_inner(Ctx& x, const nhmf_solve_opts& o, const double* r, double* z, long long* inner) {
  SolverWork& w = x.w;
  norm2(x.n, r, w.sc + TMP, w.partials, x.s);
  to_fp32_scaled(x.n, r, w.sc + TMP, true, w.b32, x.s);
  long long it = 0;
  double rel = 0.0;
  // the spatial cache is FP64 only: the FP32 inner operator then runs on the fly
  const int s32 = o.strategy == NHMF_SPATIAL ? NHMF_ON_THE_FLY : o.strategy;
  nhmf_status st = pcg<float>(x, s32, w.b32, w.x32, w.dinv32, w.r32, w.z32, w.p32, w.q32, o.inner_rtol,
                              o.inner_max_iter, o.check_every, IN_RZ0, &it, &rel);
  *inner += it;
  if (st != NHMF_OK) return st;
  to_fp64_scaled(x.n, w.x32, w.sc + TMP, z, x.s);
  return cuda_check(x.c, cudaGetLastError(), "mixed preconditioner");
}

// Multi-preconditioned CG with two directions per iteration (Bridson and Greif, 2006),
// truncated to one previous block: Z = [M1(r), M2(r)], P = Z - P_prev G_prev^-1 (AP_prev)^T Z,
// alpha = (P^T A P)^-1 P^T r, x += P alpha, r -= AP alpha.  A direction is dropped when the
// 2x2 Gram matrix is near singular.  Returns NHMF_ERR_NOT_CONVERGED on stagnation.
template <class P1, class P2>
nhmf_status mpcg2(Ctx& x, int strat, const double* b, double* sol, double rtol, int maxit, P1&& m1, P2&& m2,
                  long long* iters, double* relres, int stall_window, double stall_factor) {
  nhmf_ctx* c = x.c;
  SolverWork& w = x.w;
  double* sc = w.sc;
  double bnh;
  nhmf_status st = norm(x, b, BN, &bnh);
  if (st != NHMF_OK) return st;
  cudaMemsetAsync(sol, 0, x.n * sizeof(double), x.s);
  *iters = 0;
  *relres = 0.0;
  if (!(bnh > 0.0)) return bnh == 0.0 ? NHMF_OK : fail(c, NHMF_ERR_NONFINITE, "mpcg: non-finite right-hand side");
  cudaMemcpyAsync(w.r, b, x.n * sizeof(double), cudaMemcpyDeviceToDevice, x.s);
  double *z1 = w.z, *z2 = w.t, *a1 = w.q, *a2 = w.qprev, *p1 = w.p, *p2 = w.x, *q1 = w.R, *q2 = w.d;
  double G[3] = {0, 0, 0};  // previous block Gram matrix (00, 01, 11)
  bool have_prev = false, prev_two = false;
  std::vector<double> hist{bnh};
  double rn = bnh;
  long long k = 0;
  auto dots = [&](std::initializer_list<std::pair<const double*, const double*>> prs, double* out) -> nhmf_status {
    int i = 0;
    for (auto& pr : prs) dot(x.n, pr.first, pr.second, sc + 32 + i++, w.partials, x.s);
    nhmf_status s2 = cuda_check(c, cudaMemcpyAsync(w.host, sc + 32, i * sizeof(double), cudaMemcpyDeviceToHost, x.s), "dots");
    if (s2 == NHMF_OK) s2 = cuda_check(c, cudaStreamSynchronize(x.s), "dots sync");
    for (int j = 0; j < i; ++j) out[j] = w.host[j];
    return s2;
  };
  for (; k < maxit;) {
    if ((st = m1(w.r, z1)) != NHMF_OK) return st;
    if ((st = m2(w.r, z2)) != NHMF_OK) return st;
    if ((st = launch_apply(c, x.outer, strat, z1, a1, x.s)) != NHMF_OK) return st;
    if ((st = launch_apply(c, x.outer, strat, z2, a2, x.s)) != NHMF_OK) return st;
    if (have_prev) {
      // beta = G_prev^-1 [q1.z1 q1.z2; q2.z1 q2.z2]
      double C[4] = {0, 0, 0, 0};
      if (prev_two) {
        if ((st = dots({{q1, z1}, {q1, z2}, {q2, z1}, {q2, z2}}, C)) != NHMF_OK) return st;
      } else {
        if ((st = dots({{q1, z1}, {q1, z2}}, C)) != NHMF_OK) return st;
      }
      double B[4];
      if (prev_two) {
        const double det = G[0] * G[2] - G[1] * G[1];
        B[0] = (G[2] * C[0] - G[1] * C[2]) / det;
        B[1] = (G[2] * C[1] - G[1] * C[3]) / det;
        B[2] = (G[0] * C[2] - G[1] * C[0]) / det;
        B[3] = (G[0] * C[3] - G[1] * C[1]) / det;
      } else {
        B[0] = C[0] / G[0];
        B[1] = C[1] / G[0];
        B[2] = B[3] = 0.0;
      }
      axpby(x.n, -B[0], nullptr, p1, 1.0, nullptr, z1, x.s);
      axpby(x.n, -B[1], nullptr, p1, 1.0, nullptr, z2, x.s);
      axpby(x.n, -B[0], nullptr, q1, 1.0, nullptr, a1, x.s);
      axpby(x.n, -B[1], nullptr, q1, 1.0, nullptr, a2, x.s);
      if (prev_two) {
        axpby(x.n, -B[2], nullptr, p2, 1.0, nullptr, z1, x.s);
        axpby(x.n, -B[3], nullptr, p2, 1.0, nullptr, z2, x.s);
        axpby(x.n, -B[2], nullptr, q2, 1.0, nullptr, a1, x.s);
        axpby(x.n, -B[3], nullptr, q2, 1.0, nullptr, a2, x.s);
      }
    }
    double D[5];
    if ((st = dots({{z1, a1}, {z1, a2}, {z2, a2}, {z1, w.r}, {z2, w.r}}, D)) != NHMF_OK) return st;
    if (!(D[0] > 0.0)) return fail(c, NHMF_ERR_BREAKDOWN, "mpcg: p^T A p <= 0");
    double al0, al1;
    const double det = D[0] * D[2] - D[1] * D[1];
    const bool two = D[2] > 0.0 && det > 1e-10 * D[0] * D[2];
    if (two) {
      al0 = (D[2] * D[3] - D[1] * D[4]) / det;
      al1 = (D[0] * D[4] - D[1] * D[3]) / det;
    } else {
      al0 = D[3] / D[0];
      al1 = 0.0;
    }
    axpby(x.n, al0, nullptr, z1, 1.0, nullptr, sol, x.s);
    axpby(x.n, -al0, nullptr, a1, 1.0, nullptr, w.r, x.s);
    if (two) {
      axpby(x.n, al1, nullptr, z2, 1.0, nullptr, sol, x.s);
      axpby(x.n, -al1, nullptr, a2, 1.0, nullptr, w.r, x.s);
    }
    // the new block becomes the previous one (a dropped direction is not kept)
    std::swap(p1, z1);
    std::swap(q1, a1);
    if (two) {
      std::swap(p2, z2);
      std::swap(q2, a2);
    }
    G[0] = D[0];
    G[1] = two ? D[1] : 0.0;
    G[2] = two ? D[2] : 0.0;
    have_prev = true;
    prev_two = two;
    ++k;
    if ((st = norm(x, w.r, RNORM, &rn)) != NHMF_OK) return st;
    if (!std::isfinite(rn)) return fail(c, NHMF_ERR_NONFINITE, "mpcg: non-finite residual");
    hist.push_back(rn);
    if (rn <= rtol * bnh) break;
    if (stall_window > 0 && (long long)hist.size() > stall_window &&
        rn > stall_factor * hist[hist.size() - 1 - stall_window]) {
      *iters = k;
      *relres = rn / bnh;
      return NHMF_ERR_NOT_CONVERGED;
    }
  }
  *iters = k;
  *relres = rn / bnh;
  return rn <= rtol * bnh ? NHMF_OK : NHMF_ERR_NOT_CONVERGED;
}

// One geometric-multigrid V-cycle for A_l x = b on level l (x overwritten).
template <typename T>
nhmf_status vcycle(nhmf_ctx* c, int l, const nhmf_solve_opts& o, const T* b, T* x, cudaStream_t s,
                   long long* coarse_iters) {
  Gmg& G = *c->gmg;
  GmgLevel& L = G.L[l];
  const bool fp32 = sizeof(T) == 4;
  const int strat = (fp32 && o.strategy == NHMF_SPATIAL) ? NHMF_ON_THE_FLY : o.strategy;
  nhmf_status st;
  if (l == 0) {
    Ctx cx{L.ctx, s, L.n, *L.ctx->work};
    long long it = 0;
    double rel = 0.0;
    // near-exact in FP64, to 1e-4 in FP32 (which cannot reach FP64 tolerances)
    st = pcg<T>(cx, strat, b, x, Buf<T>::dinv(L), Buf<T>::r(L), Buf<T>::d(L), Buf<T>::t1(L), Buf<T>::t2(L),
                fp32 ? 1e-4 : 1e-6, 5000, 10, fp32 ? IN_RZ0 : RZ0, &it, &rel);
    *coarse_iters += it;
    return st;
  }
  GmgLevel& C = G.L[l - 1];
  const int deg = o.smoother_degree > 0 ? o.smoother_degree : 3;
  const double range = o.smoother_range > 1.0 ? o.smoother_range : 15.0;
  if ((st = chebyshev<T>(L, strat, b, x, deg, range, true, s)) != NHMF_OK) return st;
  if ((st = launch_apply(L.ctx, Buf<T>::prec, strat, x, Buf<T>::r(L), s)) != NHMF_OK) return st;
  gmg_bminus<T>(L.n, b, Buf<T>::r(L), s);
  gmg_restrict<T>(L, Buf<T>::r(L), Buf<T>::b(C), s);
  if (fp32)
    st = fix_rows32(C.ctx, nullptr, reinterpret_cast<float*>(Buf<T>::b(C)), 1, 0.f, s);
  else
    st = fix_rows64(C.ctx, nullptr, reinterpret_cast<double*>(Buf<T>::b(C)), 1, 0.0, s);
  if (st != NHMF_OK) return st;
  if ((st = vcycle<T>(c, l - 1, o, Buf<T>::b(C), Buf<T>::x(C), s, coarse_iters)) != NHMF_OK) return st;
  gmg_prolong_add<T>(L, Buf<T>::x(C), x, Buf<T>::q(L), s);
  return chebyshev<T>(L, strat, b, x, deg, range, false, s);
}

// One linear solve A(ubar) sol = b with the chosen solver; the diagonal must be current.
nhmf_status linear(Ctx& x, const nhmf_solve_opts& o, const double* b, double* sol, long long* outer,
                   long long* inner, double* relres, int* fallbacks) {
  SolverWork& w = x.w;
  *inner = 0;
  x.outer = o.outer_apply == NHMF_DF64 ? NHMF_DF64 : NHMF_FP64;  // the flexible solvers' outer applies
  // host-side fault injection: a preconditioner that returns z = 0 (a stalled flexible solve),
  // a network whose output is noise
  const bool learned_any = o.solver == NHMF_SOLVER_LEARNED_FCG || o.solver == NHMF_SOLVER_MIXED_LEARNED ||
                           o.solver == NHMF_SOLVER_MIXED_GMG_LEARNED;
  const bool stall = o.solver != NHMF_SOLVER_JACOBI_CG && take_inject(x.c, NHMF_INJECT_CG_STALL);
  const bool garbage = learned_any && take_inject(x.c, NHMF_INJECT_UNET_GARBAGE);
  auto zero = [&](double* z) -> nhmf_status {
    return cuda_check(x.c, cudaMemsetAsync(z, 0, x.n * sizeof(double), x.s), "injected stall");
  };
  // a flexible solve that broke down (p^T A p <= 0) is solved again by Jacobi-CG from scratch
  auto restart_cg = [&]() -> nhmf_status {
    *fallbacks += 1;
    cudaMemsetAsync(x.c->status, 0, sizeof(unsigned), x.s);
    return pcg<double>(x, o.strategy, b, sol, w.dinv, w.r, w.z, w.p, w.q, o.linear_rtol, o.linear_max_iter,
                       o.check_every, RZ0, outer, relres);
  };
  if (o.solver == NHMF_SOLVER_JACOBI_CG) {
    UNet* u = x.c->unet;
    if (!(o.record_pairs && u && u->npairs < u->cap))
      return pcg<double>(x, o.strategy, b, sol, w.dinv, w.r, w.z, w.p, w.q, o.linear_rtol, o.linear_max_iter,
                         o.check_every, RZ0, outer, relres);
    // record CG pairs (r_j, x* - x_j) at j = k, 4k, 16k
    std::vector<int> slots;
    const long long every = o.cg_pair_every > 0 ? o.cg_pair_every : 8;
    auto snap = [&](long long j, const void* r, const void* xj) {
      if (j == every || j == 4 * every || j == 16 * every) {
        const int slot = unet_snapshot_begin(x.c, static_cast<const double*>(r), static_cast<const double*>(xj), x.s);
        if (slot >= 0) slots.push_back(slot);
      }
    };
    nhmf_status st = pcg<double>(x, o.strategy, b, sol, w.dinv, w.r, w.z, w.p, w.q, o.linear_rtol,
                                 o.linear_max_iter, o.check_every, RZ0, outer, relres, snap);
    if (st != NHMF_OK) return st;
    for (int slot : slots) unet_snapshot_finish(x.c, slot, sol, x.s);
    return cuda_check(x.c, cudaGetLastError(), "pair recording");
  }
  if (o.solver == NHMF_SOLVER_MIXED_FCG) {
    auto precond = [&](const double* r, double* z) -> nhmf_status {
      return stall ? zero(z) : mixed_inner(x, o, r, z, inner);
    };
    const nhmf_status st = fcg(x, o.strategy, b, sol, o.linear_rtol, o.linear_max_iter, precond, outer, relres);
    return st == NHMF_ERR_BREAKDOWN ? restart_cg() : st;
  }
  // fall back to Jacobi-CG on the remaining residual w.r of a stalled flexible solve:
  // A d = r, sol += d
  auto fallback_cg = [&]() -> nhmf_status {
    *fallbacks += 1;
    double bnh, rnh;
    nhmf_status st = norm(x, b, TMP, &bnh);
    if (st != NHMF_OK) return st;
    if ((st = norm(x, w.r, TMP, &rnh)) != NHMF_OK) return st;
    cudaMemcpyAsync(w.b2, w.r, x.n * sizeof(double), cudaMemcpyDeviceToDevice, x.s);
    long long it2 = 0;
    double rel2 = 0.0;
    const double rtol2 = rnh > 0.0 ? std::min(1.0, o.linear_rtol * bnh / rnh) : 1.0;
    st = pcg<double>(x, o.strategy, w.b2, w.x2, w.dinv, w.r, w.z, w.p, w.q, rtol2, o.linear_max_iter,
                     o.check_every, RZ0, &it2, &rel2);
    if (st != NHMF_OK) return st;
    axpby(x.n, 1.0, nullptr, w.x2, 1.0, nullptr, sol, x.s);
    *outer += it2;
    *relres = rel2 * rnh / bnh;
    return cuda_check(x.c, cudaGetLastError(), "fallback");
  };
  if (o.solver == NHMF_SOLVER_GMG || o.solver == NHMF_SOLVER_MIXED_GMG || o.solver == NHMF_SOLVER_MIXED_GMG_LEARNED) {
    const bool f32 = o.solver != NHMF_SOLVER_GMG;
    const bool learned = o.solver == NHMF_SOLVER_MIXED_GMG_LEARNED;
    UNet* un = x.c->unet;
    if (learned && !un) return fail(x.c, NHMF_ERR_STATE, "learned correction: no network in this context");
    // training pairs of the learned correction, recorded by MIXED_GMG solves (see below)
    const bool record = o.solver == NHMF_SOLVER_MIXED_GMG && o.record_pairs && un;
    const long long rec_iters = o.cg_pair_every > 0 ? o.cg_pair_every : 8;
    std::vector<int> slots;
    long long jprec = 0;
    nhmf_status st = gmg_prepare(x.c, o.strategy, f32, x.s, false, w.diag);
    if (st == NHMF_ERR_NONPOS_J) st = gmg_prepare(x.c, o.strategy, f32, x.s, true, w.diag);  // folded coarse state
    if (st != NHMF_OK) return st;
    {
      // SPD probe of the coarsest level: Jacobi-CG on a fixed right-hand side.  If the coarse
      // tangent at the interpolated state is indefinite, the coarse levels are linearised at
      // zero instead (linear elasticity, SPD).
      GmgLevel& C0 = x.c->gmg->L[0];
      if (x.c->gmg->L.size() > 1) {
        Ctx cx{C0.ctx, x.s, C0.n, *C0.ctx->work};
        gmg_start_vector(C0.n, C0.b, x.s);
        long long it = 0;
        double rel = 0.0;
        nhmf_status ps = pcg<double>(cx, o.strategy, C0.b, C0.x, C0.dinv, C0.r, C0.d, C0.t1, C0.t2, 1e-6, 300, 10, RZ0,
                                     &it, &rel);
        if (ps == NHMF_ERR_BREAKDOWN) {
          if ((st = gmg_prepare(x.c, o.strategy, f32, x.s, true, w.diag)) != NHMF_OK) return st;
        } else if (ps != NHMF_OK) {
          return ps;
        }
      }
    }
    GmgLevel& top = x.c->gmg->L.back();
    const int ltop = (int)x.c->gmg->L.size() - 1;
    const int strat32 = o.strategy == NHMF_SPATIAL ? NHMF_ON_THE_FLY : o.strategy;
    auto precond = [&](const double* r, double* z) -> nhmf_status {
      if (stall) return zero(z);
      if (!f32) return vcycle<double>(x.c, ltop, o, r, z, x.s, inner);
      norm2(x.n, r, w.sc + TMP, w.partials, x.s);
      to_fp32_scaled(x.n, r, w.sc + TMP, true, top.b32, x.s);
      nhmf_status s2 = vcycle<float>(x.c, ltop, o, top.b32, top.x32, x.s, inner);
      if (s2 != NHMF_OK) return s2;
      to_fp64_scaled(x.n, top.x32, w.sc + TMP, z, x.s);
      const bool rec_now = record && un->npairs < un->cap && jprec < rec_iters;
      ++jprec;
      if (learned || rec_now) {
        // residual the V-cycle leaves, t = r - A z, from an FP32 apply to its FP32 output
        if ((s2 = launch_apply(x.c, NHMF_FP32, strat32, top.x32, top.r32, x.s)) != NHMF_OK) return s2;
        to_fp64_scaled(x.n, top.r32, w.sc + TMP, w.t, x.s);
        axpby(x.n, 1.0, nullptr, r, -1.0, nullptr, w.t, x.s);
        if (rec_now) {
          // pair (t, x* - (x_j + z)): the error left after the V-cycle, A (x* - x_j - z) = t
          cudaMemcpyAsync(w.x2, sol, x.n * sizeof(double), cudaMemcpyDeviceToDevice, x.s);
          axpby(x.n, 1.0, nullptr, z, 1.0, nullptr, w.x2, x.s);
          const int slot = unet_snapshot_begin(x.c, w.t, w.x2, x.s);
          if (slot >= 0) slots.push_back(slot);
        }
        if (learned) {
          // c = N(t) has the direction of the remaining error but no meaningful scale (the
          // training pairs are normalised): z += omega c with the A-optimal step
          // omega = (c . t) / (c . A c), A c from an FP32 apply
          unet_precondition(x.c, w.t, w.x2, x.s);
          if (garbage) fill_noise(x.n, w.x2, 0x5EEDull + (unsigned long long)jprec, x.s);
          norm2(x.n, w.x2, w.sc + CNORM, w.partials, x.s);
          to_fp32_scaled(x.n, w.x2, w.sc + CNORM, true, top.b32, x.s);
          if ((s2 = launch_apply(x.c, NHMF_FP32, strat32, top.b32, top.r32, x.s)) != NHMF_OK) return s2;
          to_fp64_scaled(x.n, top.r32, w.sc + CNORM, w.b2, x.s);
          dot(x.n, w.x2, w.t, w.sc + CT, w.partials, x.s);
          dot(x.n, w.x2, w.b2, w.sc + CAC, w.partials, x.s);
          ratio_or_zero(w.sc + CT, w.sc + CAC, w.sc + OMEGA, x.s);
          axpby(x.n, 1.0, w.sc + OMEGA, w.x2, 1.0, nullptr, z, x.s);
        }
      }
      return cuda_check(x.c, cudaGetLastError(), "mixed gmg");
    };
    if (learned) {
      st = fcg(x, o.strategy, b, sol, o.linear_rtol, std::max(1, o.linear_max_iter / 4), precond, outer, relres,
               o.learned_stall_window, o.learned_stall_factor);
      if (st == NHMF_ERR_BREAKDOWN) return restart_cg();
      return st == NHMF_ERR_NOT_CONVERGED ? fallback_cg() : st;
    }
    st = fcg(x, o.strategy, b, sol, o.linear_rtol, o.linear_max_iter, precond, outer, relres);
    if (st == NHMF_OK && !slots.empty()) {
      for (int slot : slots) unet_snapshot_finish(x.c, slot, sol, x.s);
      return cuda_check(x.c, cudaGetLastError(), "pair recording");
    }
    if (st != NHMF_ERR_BREAKDOWN) return st;
    // a breakdown left: solve with Jacobi-CG from scratch (the reference solver of the method)
    return restart_cg();
  }
  if (o.solver == NHMF_SOLVER_LEARNED_FCG || o.solver == NHMF_SOLVER_MIXED_LEARNED) {
    if (!x.c->unet) return fail(x.c, NHMF_ERR_STATE, "learned preconditioner: no network in this context");
    long long napp = 0;
    auto network = [&](const double* r, double* z) -> nhmf_status {
      if (stall) return zero(z);
      unet_precondition(x.c, r, z, x.s);
      if (garbage) fill_noise(x.n, z, 0x5EEDull + (unsigned long long)napp++, x.s);
      return cuda_check(x.c, cudaGetLastError(), "network direction");
    };
    auto inner_cg = [&](const double* r, double* z) -> nhmf_status {
      return stall ? zero(z) : mixed_inner(x, o, r, z, inner);
    };
    const int cap = std::max(1, o.linear_max_iter / 4);
    nhmf_status st =
        o.solver == NHMF_SOLVER_LEARNED_FCG
            ? fcg(x, o.strategy, b, sol, o.linear_rtol, cap, network, outer, relres, o.learned_stall_window,
                  o.learned_stall_factor)
            : mpcg2(x, o.strategy, b, sol, o.linear_rtol, cap, inner_cg, network, outer, relres,
                    o.learned_stall_window, o.learned_stall_factor);
    if (st == NHMF_ERR_BREAKDOWN) return restart_cg();
    if (st != NHMF_ERR_NOT_CONVERGED) return st;
    return fallback_cg();
  }
  return fail(x.c, NHMF_ERR_ARG, "unknown solver");
}

int cache_mask(const nhmf_solve_opts& o) {
  if (o.strategy == NHMF_SPATIAL) return NHMF_CACHE_SPATIAL;
  if (o.strategy != NHMF_CACHED) return 0;
  const int df = o.outer_apply == NHMF_DF64 && o.solver != NHMF_SOLVER_JACOBI_CG ? NHMF_CACHE_DF64 : 0;
  return ((o.solver == NHMF_SOLVER_MIXED_FCG || o.solver == NHMF_SOLVER_MIXED_LEARNED ||
           o.solver == NHMF_SOLVER_MIXED_GMG || o.solver == NHMF_SOLVER_MIXED_GMG_LEARNED)
              ? (NHMF_CACHE_FP64 | NHMF_CACHE_FP32)
              : NHMF_CACHE_FP64) | df;
}

nhmf_status check_opts(nhmf_ctx* c, const nhmf_solve_opts* o) {
  if (!o || o->solver < 0 || o->solver > NHMF_SOLVER_MIXED_GMG_LEARNED ||
      (o->strategy != NHMF_ON_THE_FLY && o->strategy != NHMF_CACHED && o->strategy != NHMF_SPATIAL) ||
      o->load_steps < 1 || o->newton_max_iter < 1 || o->linear_max_iter < 1 || o->check_every < 1 ||
      o->inner_max_iter < 1 || !(o->linear_rtol > 0) || !(o->newton_rtol > 0) || o->max_backtracks < 0 ||
      (o->outer_apply != NHMF_FP64 && o->outer_apply != NHMF_DF64) ||
      (o->outer_apply == NHMF_DF64 && o->strategy != NHMF_CACHED))
    return fail(c, NHMF_ERR_ARG, "solve: bad options");
  return NHMF_OK;
}

}  // namespace

void free_work(nhmf_ctx* c) {
  if (!c->work) return;
  SolverWork& w = *c->work;
  void* ptrs[] = {w.r, w.z, w.p, w.q, w.qprev, w.x, w.b, w.R, w.d, w.t, w.du, w.utry, w.diag, w.dinv, w.b2, w.x2,
                  w.r32, w.z32, w.p32, w.q32, w.x32, w.b32, w.dinv32, w.sc, w.partials};
  for (void* p : ptrs) cudaFree(p);
  if (w.host) cudaFreeHost(w.host);
  for (auto& G : w.graph)
    if (G.exec) cudaGraphExecDestroy(G.exec);
  if (w.ev_in) cudaEventDestroy(w.ev_in);
  if (w.ev_out) cudaEventDestroy(w.ev_out);
  if (w.stream) cudaStreamDestroy(w.stream);
  delete c->work;
  c->work = nullptr;
}

}  // namespace nhmf

using namespace nhmf;

extern "C" {

void nhmf_solve_opts_default(nhmf_solve_opts* o) {
  if (!o) return;
  o->solver = NHMF_SOLVER_JACOBI_CG;
  o->strategy = NHMF_CACHED;
  o->load_steps = 1;
  o->first_step = 1;
  o->last_step = 0;
  o->compression = 0.0;
  o->newton_rtol = 1e-8;
  o->newton_max_iter = 20;
  o->max_backtracks = 8;
  o->linear_rtol = 1e-6;
  o->linear_max_iter = 20000;
  o->inner_rtol = 1e-3;
  o->inner_max_iter = 1000;
  o->check_every = 10;
  o->record_pairs = 0;
  o->cg_pair_every = 8;
  o->learned_stall_window = 10;
  o->learned_stall_factor = 0.9;
  o->synthetic_pairs = 0;
  o->seed = 1;
  o->smoother_degree = 3;
  o->smoother_range = 15.0;
  o->outer_apply = NHMF_FP64;
}

nhmf_status nhmf_linear_solve(nhmf_ctx* c, const nhmf_solve_opts* o, const double* b, double* xsol, long long* iters,
                              long long* inner_iters, double* rel_res, void* stream) {
  if (!c) return NHMF_ERR_ARG;
  if (!b || !xsol || !iters || !inner_iters || !rel_res) return fail(c, NHMF_ERR_ARG, "linear_solve: bad argument");
  nhmf_status st = check_opts(c, o);
  if (st != NHMF_OK) return st;
  if (!c->have_lin) return fail(c, NHMF_ERR_STATE, "linear_solve: no linearisation point set");
  if (o->strategy == NHMF_SPATIAL && !c->cachesp)
    return fail(c, NHMF_ERR_STATE, "linear_solve: the spatial strategy needs the NHMF_CACHE_SPATIAL cache");
  if (o->strategy == NHMF_CACHED && (!c->cache64 || ((cache_mask(*o) & NHMF_CACHE_FP32) && !c->cache32) ||
                                     ((cache_mask(*o) & NHMF_CACHE_DF64) && !c->cachedf)))
    return fail(c, NHMF_ERR_STATE, "linear_solve: the cached strategy needs the point caches");
  if ((st = ensure_work(c)) != NHMF_OK) return st;
  NvtxRange range("nhmf_linear_solve");
  const auto t0 = std::chrono::steady_clock::now();
  Ctx x{c, c->work->stream, 3 * c->g.M3, *c->work};
  cudaEventRecord(x.w.ev_in, static_cast<cudaStream_t>(stream));
  cudaStreamWaitEvent(x.s, x.w.ev_in, 0);
  auto finish = [&](nhmf_status v) {
    cudaEventRecord(x.w.ev_out, x.s);
    cudaStreamWaitEvent(static_cast<cudaStream_t>(stream), x.w.ev_out, 0);
    cudaStreamSynchronize(x.s);
    return v;
  };
  if ((st = update_diagonal(x)) != NHMF_OK) return finish(st);
  double rel = 0.0;
  int fb = 0;
  if ((st = linear(x, *o, b, xsol, iters, inner_iters, &rel, &fb)) != NHMF_OK) return finish(st);
  // true residual with an FP64 apply
  if ((st = launch_apply(c, NHMF_FP64, o->strategy, xsol, x.w.t, x.s)) != NHMF_OK) return finish(st);
  axpby(x.n, 1.0, nullptr, b, -1.0, nullptr, x.w.t, x.s);
  double rn, bn;
  if ((st = norm(x, x.w.t, TMP, &rn)) != NHMF_OK) return finish(st);
  if ((st = norm(x, b, TMP, &bn)) != NHMF_OK) return finish(st);
  *rel_res = bn > 0 ? rn / bn : 0.0;
  const nhmf_status done = finish(NHMF_OK);
  metrics_line(c, "\"event\": \"linear_solve\", \"solver\": %d, \"iters\": %lld, \"inner_iters\": %lld, "
               "\"fallbacks\": %d, \"rel_residual\": %.6e, \"seconds\": %.6f",
               o->solver, *iters, *inner_iters, fb, *rel_res,
               std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count());
  return done;
}

static nhmf_status solve_impl(nhmf_ctx* c, const nhmf_solve_opts* o, double* u, nhmf_solve_stats* stats) {
  using clk = std::chrono::steady_clock;
  if (!c) return NHMF_ERR_ARG;
  nhmf_status st = check_opts(c, o);
  if (st != NHMF_OK) return st;
  if (!u || !stats) return fail(c, NHMF_ERR_ARG, "solve: bad argument");
  const int S = o->load_steps;
  const int first = o->first_step > 0 ? o->first_step : 1;
  const int last = o->last_step > 0 ? o->last_step : S;
  if (first > last || last > S || last - first + 1 > NHMF_MAX_STEPS) return fail(c, NHMF_ERR_ARG, "solve: bad step range");
  if ((st = ensure_work(c)) != NHMF_OK) return st;
  *stats = nhmf_solve_stats{};
  Ctx x{c, c->work->stream, 3 * c->g.M3, *c->work};
  SolverWork& w = x.w;
  const long long M2 = (long long)c->g.M * c->g.M;
  const unsigned bc_blocks = (unsigned)((M2 + 255) / 256);
  const auto t_all = clk::now();
  for (int step = first; step <= last; ++step) {
    const int k = step - first;
    NvtxRange step_range("load step");
    const auto t0 = clk::now();
    const double top = c->prm.bc == NHMF_BC_COMPRESSION ? -o->compression * step / S : 0.0;
    double ref = -1.0, bnh = 0.0;
    bool converged = false;
    int it = 0;
    for (; it <= o->newton_max_iter; ++it) {
      NvtxRange iter_range("newton iteration");
      const auto t_it = clk::now();
      if ((st = launch_residual(c, u, w.R, x.s)) != NHMF_OK) return st;
      if ((st = nhmf_check_status(c, x.s)) != NHMF_OK) return st;
      cudaMemsetAsync(w.d, 0, x.n * sizeof(double), x.s);
      if (c->prm.bc != NHMF_BC_NONE) k_bc<<<bc_blocks, 256, 0, x.s>>>(c->prm.bc, c->g.M, c->g.M3, top, u, w.d, 0);
      double dn;
      if ((st = norm(x, w.d, TMP, &dn)) != NHMF_OK) return st;
      if ((st = nhmf_set_linearization(c, u, cache_mask(*o), x.s)) != NHMF_OK) return st;
      axpby(x.n, -1.0, nullptr, w.R, 0.0, nullptr, w.b, x.s);          // b = -R
      if (dn > 0.0) {
        if ((st = launch_apply(c, NHMF_FP64, o->strategy, w.d, w.t, x.s, true)) != NHMF_OK) return st;
        axpby(x.n, -1.0, nullptr, w.t, 1.0, nullptr, w.b, x.s);        // b -= K d
      }
      if ((st = fix_rows64(c, w.d, w.b, 0, 0.0, x.s)) != NHMF_OK) return st;  // b_D = d_D
      if ((st = norm(x, w.b, TMP, &bnh)) != NHMF_OK) return st;
      if (ref < 0.0) ref = bnh;
      if (dn == 0.0 && (bnh <= o->newton_rtol * ref || bnh == 0.0)) {
        converged = true;
        break;
      }
      if (it == o->newton_max_iter) break;
      if ((st = update_diagonal(x)) != NHMF_OK) return st;
      long long outer = 0, inner = 0;
      double rel = 0.0;
      if (c->metrics) cudaStreamSynchronize(x.s);  // split the iteration's time at the linear solve
      const auto t_lin = clk::now();
      if ((st = linear(x, *o, w.b, w.du, &outer, &inner, &rel, &stats->fallbacks[k])) != NHMF_OK) return st;
      if (c->metrics) cudaStreamSynchronize(x.s);
      const auto t_lin_end = clk::now();
      if (take_inject(c, NHMF_INJECT_NAN_DU)) {  // host-side fault injection: a NaN in the update
        const double nan = std::numeric_limits<double>::quiet_NaN();
        if ((st = cuda_check(c, cudaMemcpyAsync(w.du + x.n / 2, &nan, sizeof(double), cudaMemcpyHostToDevice, x.s),
                             "injected NaN")) != NHMF_OK)
          return st;
      }
      if (o->record_pairs && o->solver == NHMF_SOLVER_JACOBI_CG && c->unet) {
        if ((st = unet_record(c, w.b, w.du, x.s)) != NHMF_OK) return st;   // Newton pair (b, du)
        for (int q = 0; q < o->synthetic_pairs; ++q) {                     // (K e, e), smooth e
          unet_smooth_field(c, w.t, o->seed + 0x100000ull * (unsigned long long)(step * 64 + it) + q, x.s);  // scale = seed mod levels
          if ((st = launch_apply(c, NHMF_FP64, o->strategy, w.t, w.x2, x.s)) != NHMF_OK) return st;
          if ((st = unet_record(c, w.x2, w.t, x.s)) != NHMF_OK) return st;
        }
      }
      stats->linear_iters[k] += outer;
      stats->inner_iters[k] += inner;
      // backtracking: halve the step while det F <= 0 somewhere
      double theta = 1.0;
      bool ok = false;
      for (int bt = 0; bt <= o->max_backtracks; ++bt) {
        cudaMemcpyAsync(w.utry, u, x.n * sizeof(double), cudaMemcpyDeviceToDevice, x.s);
        axpby(x.n, theta, nullptr, w.du, 1.0, nullptr, w.utry, x.s);
        st = launch_residual(c, w.utry, w.R, x.s);
        if (st != NHMF_OK) return st;
        st = nhmf_check_status(c, x.s);
        if (st == NHMF_OK) {
          ok = true;
          break;
        }
        if (st != NHMF_ERR_NONPOS_J) return st;
        theta *= 0.5;
      }
      if (!ok) return fail(c, NHMF_ERR_NONPOS_J, "Newton: backtracking could not keep det F > 0");
      metrics_line(c, "\"event\": \"newton_iteration\", \"step\": %d, \"iteration\": %d, \"rel_residual\": %.6e, "
                   "\"linear_iters\": %lld, \"inner_iters\": %lld, \"linear_rel_residual\": %.6e, \"theta\": %.6g, "
                   "\"setup_seconds\": %.6f, \"linear_seconds\": %.6f, \"update_seconds\": %.6f, \"seconds\": %.6f",
                   step, it, ref > 0.0 ? bnh / ref : 0.0, outer, inner, rel, theta,
                   std::chrono::duration<double>(t_lin - t_it).count(),
                   std::chrono::duration<double>(t_lin_end - t_lin).count(),
                   std::chrono::duration<double>(clk::now() - t_lin_end).count(),
                   std::chrono::duration<double>(clk::now() - t0).count());
      cudaMemcpyAsync(u, w.utry, x.n * sizeof(double), cudaMemcpyDeviceToDevice, x.s);
      if (theta == 1.0 && c->prm.bc != NHMF_BC_NONE)
        k_bc<<<bc_blocks, 256, 0, x.s>>>(c->prm.bc, c->g.M, c->g.M3, top, u, nullptr, 1);  // u_D = g exactly
    }
    cudaStreamSynchronize(x.s);
    stats->newton_iters[k] = it;
    stats->rel_residual[k] = ref > 0.0 ? bnh / ref : 0.0;
    stats->seconds[k] = std::chrono::duration<double>(clk::now() - t0).count();
    stats->total_linear_iters += stats->linear_iters[k];
    stats->total_inner_iters += stats->inner_iters[k];
    stats->steps_done = k + 1;
    metrics_line(c, "\"event\": \"load_step\", \"step\": %d, \"newton_iters\": %d, \"linear_iters\": %lld, "
                 "\"inner_iters\": %lld, \"fallbacks\": %d, \"rel_residual\": %.6e, \"seconds\": %.6f, "
                 "\"converged\": %s",
                 step, it, stats->linear_iters[k], stats->inner_iters[k], stats->fallbacks[k], stats->rel_residual[k],
                 stats->seconds[k], converged ? "true" : "false");
    if (!converged) {
      stats->total_seconds = std::chrono::duration<double>(clk::now() - t_all).count();
      return fail(c, NHMF_ERR_NOT_CONVERGED, "Newton: load step " + std::to_string(step) + " did not converge");
    }
  }
  stats->total_seconds = std::chrono::duration<double>(clk::now() - t_all).count();
  return NHMF_OK;
}

}

nhmf_status nhmf_solve(nhmf_ctx* c, const nhmf_solve_opts* o, double* u, nhmf_solve_stats* stats, void* stream) {
  if (!c) return NHMF_ERR_ARG;
  nhmf_status st = ensure_work(c);
  if (st != NHMF_OK) return st;
  NvtxRange range("nhmf_solve");
  // the solver runs on the context's own stream, ordered after the caller's stream
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  cudaEventRecord(c->work->ev_in, cs);
  cudaStreamWaitEvent(c->work->stream, c->work->ev_in, 0);
  st = solve_impl(c, o, u, stats);
  cudaEventRecord(c->work->ev_out, c->work->stream);
  cudaStreamWaitEvent(cs, c->work->ev_out, 0);
  cudaStreamSynchronize(c->work->stream);
  return st;
}  // extern "C"
