// Geometric multigrid preconditioner (Section 2.3 of the paper): nested structured meshes
// N, N/2, N/4, ... with the same Q_p space, level operators K(u_l) at the linearisation point
// interpolated to each level, Chebyshev iteration on the inverse diagonal as smoother, the
// transfer between levels by interpolation (prolongation) and its transpose (restriction),
// and a near-exact Jacobi-CG solve on the coarsest level.
//
// Each level is a context of its own (same degree, material and boundary preset), so every
// operator kernel of the library serves every level.  The 3D transfers are tensor products
// of 1D maps applied as three passes.
#include <cmath>
#include <cstdio>
#include <vector>

#include "blas.h"
#include "gmg.h"
#include "internal.h"

namespace nhmf {
namespace {

// ------------------------------------------------------------------ kernels
// One 1D pass along `dir` of a [3][nz][ny][nx] field: out(.., i_dir, ..) = sum_k w_k in(.., col_k, ..).
template <typename T>
__global__ void k_map1d(const T* __restrict__ in, T* __restrict__ out, int dir, int nx, int ny, int nz, int mout,
                        const int* __restrict__ ptr, const int* __restrict__ col, const T* __restrict__ w) {
  const int ox = dir == 0 ? mout : nx, oy = dir == 1 ? mout : ny, oz = dir == 2 ? mout : nz;
  const long long plane = (long long)ox * oy * oz;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < 3 * plane;
       idx += (long long)gridDim.x * blockDim.x) {
    const int c = int(idx / plane);
    const long long rem = idx % plane;
    const int i = int(rem % ox), j = int((rem / ox) % oy), k = int(rem / ((long long)ox * oy));
    const int row = dir == 0 ? i : (dir == 1 ? j : k);
    T s = T(0);
    for (int e = ptr[row]; e < ptr[row + 1]; ++e) {
      const int cc = col[e];
      const int ii = dir == 0 ? cc : i, jj = dir == 1 ? cc : j, kk = dir == 2 ? cc : k;
      s = fma(w[e], in[(long long)c * nx * ny * nz + ii + (long long)nx * (jj + (long long)ny * kk)], s);
    }
    out[idx] = s;
  }
}

// Chebyshev step: d = c_old d + c_new D^-1 (b - q), x += d (q null: q = 0).
template <typename T>
__global__ void k_cheb(long long n, const T* __restrict__ b, const T* __restrict__ q, const T* __restrict__ dinv,
                       T* __restrict__ d, T* __restrict__ x, T c_old, T c_new) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const T r = q ? b[i] - q[i] : b[i];
    const T di = c_old == T(0) ? c_new * dinv[i] * r : fma(c_old, d[i], c_new * dinv[i] * r);
    d[i] = di;
    x[i] = q ? x[i] + di : di;
  }
}

// y = b - y
template <typename T>
__global__ void k_bminus(long long n, const T* __restrict__ b, T* __restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = b[i] - y[i];
}

// x += y
template <typename T>
__global__ void k_add(long long n, const T* __restrict__ y, T* __restrict__ x) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] += y[i];
}

// deterministic start vector of the power iteration: values in [0.5, 1.5) from a hash of i
__global__ void k_start(long long n, double* v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    unsigned long long z = (unsigned long long)i * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 31)) * 0xBF58476D1CE4E5B9ull;
    v[i] = 0.5 + double(z >> 11) * 0x1.0p-53;
  }
}

// x *= 1 / *nrm (x stays as it is when *nrm is not positive)
template <typename T>
__global__ void k_scale_inv(long long n, const double* __restrict__ nrm, T* __restrict__ x) {
  const double s = *nrm > 0.0 ? 1.0 / *nrm : 1.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = T(x[i] * s);
}

template <typename T>
__global__ void k_mul_t(long long n, const T* __restrict__ a, T* __restrict__ x) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] *= a[i];
}

template <typename T>
__global__ void k_to(long long n, const double* __restrict__ x, T* __restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = T(x[i]);
}

constexpr int kB = 1216, kT = 256;

// ------------------------------------------------------------------ host helpers
double lagrange(const double* z, int n, int i, double x) {
  double v = 1.0;
  for (int j = 0; j < n; ++j)
    if (j != i) v *= (x - z[j]) / (z[i] - z[j]);
  return v;
}

double node_coord(const double* t, int p, int N, int i) {
  const int e = std::min(i / p, N - 1);
  return (e + t[i - p * e]) / N;
}

// Node i of the output mesh (N_out elements of degree p_out, GLL nodes t_out) gets the value of
// the FE function of the input mesh (N_in elements of degree p_in, nodes t_in) at its position:
// the weights of the p_in + 1 Lagrange functions of the containing input element.
void build_eval_map(const double* t_out, int p_out, int N_out, const double* t_in, int p_in, int N_in,
                    std::vector<int>& ptr, std::vector<int>& col, std::vector<double>& w) {
  const int M_out = p_out * N_out + 1, n = p_in + 1;
  ptr.assign(1, 0);
  col.clear();
  w.clear();
  for (int i = 0; i < M_out; ++i) {
    const double x = node_coord(t_out, p_out, N_out, i);
    int e = int(std::floor(x * N_in + 1e-12));
    e = std::max(0, std::min(e, N_in - 1));
    const double xi = x * N_in - e;
    for (int b = 0; b < n; ++b) {
      const double v = lagrange(t_in, n, b, xi);
      if (std::fabs(v) < 1e-15) continue;
      col.push_back(p_in * e + b);
      w.push_back(v);
    }
    ptr.push_back((int)col.size());
  }
}

void transpose_map(int rows, int cols, const std::vector<int>& ptr, const std::vector<int>& col,
                   const std::vector<double>& w, std::vector<int>& tp, std::vector<int>& tc, std::vector<double>& tw) {
  std::vector<std::vector<std::pair<int, double>>> r(cols);
  for (int i = 0; i < rows; ++i)
    for (int e = ptr[i]; e < ptr[i + 1]; ++e) r[col[e]].push_back({i, w[e]});
  tp.assign(1, 0);
  tc.clear();
  tw.clear();
  for (int j = 0; j < cols; ++j) {
    for (auto& pr : r[j]) {
      tc.push_back(pr.first);
      tw.push_back(pr.second);
    }
    tp.push_back((int)tc.size());
  }
}

bool upload(Map1D& m, int rows, int cols, const std::vector<int>& ptr, const std::vector<int>& col,
            const std::vector<double>& w) {
  m.rows = rows;
  m.cols = cols;
  std::vector<float> w32(w.begin(), w.end());
  bool ok = cudaMalloc(&m.ptr, ptr.size() * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&m.col, std::max<size_t>(1, col.size()) * sizeof(int)) == cudaSuccess &&
            cudaMalloc(&m.w64, std::max<size_t>(1, w.size()) * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&m.w32, std::max<size_t>(1, w.size()) * sizeof(float)) == cudaSuccess;
  if (!ok) return false;
  cudaMemcpy(m.ptr, ptr.data(), ptr.size() * sizeof(int), cudaMemcpyHostToDevice);
  cudaMemcpy(m.col, col.data(), col.size() * sizeof(int), cudaMemcpyHostToDevice);
  cudaMemcpy(m.w64, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemcpy(m.w32, w32.data(), w32.size() * sizeof(float), cudaMemcpyHostToDevice);
  return true;
}

void free_map(Map1D& m) {
  cudaFree(m.ptr);
  cudaFree(m.col);
  cudaFree(m.w64);
  cudaFree(m.w32);
  m = Map1D{};
}

template <typename T> const T* wts(const Map1D& m);
template <> const double* wts<double>(const Map1D& m) { return m.w64; }
template <> const float* wts<float>(const Map1D& m) { return m.w32; }

// out (M_out^3) = (map x map x map) in (M_in^3), using two temporaries
template <typename T>
void map3d(const Map1D& m, const T* in, T* out, T* t1, T* t2, cudaStream_t s) {
  const int mi = m.cols, mo = m.rows;
  k_map1d<T><<<kB, kT, 0, s>>>(in, t1, 0, mi, mi, mi, mo, m.ptr, m.col, wts<T>(m));
  k_map1d<T><<<kB, kT, 0, s>>>(t1, t2, 1, mo, mi, mi, mo, m.ptr, m.col, wts<T>(m));
  k_map1d<T><<<kB, kT, 0, s>>>(t2, out, 2, mo, mo, mi, mo, m.ptr, m.col, wts<T>(m));
}

}  // namespace

void gmg_free(nhmf_ctx* c) {
  if (!c->gmg) return;
  for (size_t i = 0; i < c->gmg->L.size(); ++i) {
    GmgLevel& l = c->gmg->L[i];
    void* v[] = {l.diag, l.dinv, l.dinv32, l.x, l.b, l.r, l.d, l.q, l.t1, l.t2,
                 l.x32, l.b32, l.r32, l.d32, l.q32, l.t132, l.t232};
    for (void* p : v) cudaFree(p);
    free_map(l.P);
    free_map(l.R);
    free_map(l.I);
    if (i + 1 < c->gmg->L.size()) nhmf_destroy(l.ctx);
  }
  delete c->gmg;
  c->gmg = nullptr;
}

// Builds the hierarchy: meshes N, N/2, ... (halving while N is even and N/2 >= 2) with the fine
// degree p, then, for p > 1, one more level of degree 1 on the coarsest mesh (p-coarsening:
// the coarsest solve then has at most a few hundred DoFs).
nhmf_status gmg_build(nhmf_ctx* c) {
  if (c->gmg) return NHMF_OK;
  std::vector<int> Ns{c->g.N}, Ps{c->g.p};
  while (Ns.back() % 2 == 0 && Ns.back() / 2 >= 2 && Ns.size() < 12) {
    Ns.push_back(Ns.back() / 2);
    Ps.push_back(c->g.p);
  }
  if (c->g.p > 1) {
    Ns.push_back(Ns.back());
    Ps.push_back(1);
  }
  c->gmg = new Gmg();
  Gmg& G = *c->gmg;
  const int nl = (int)Ns.size();
  G.L.resize(nl);
  // material factors per level (fine to coarse index k = nl - 1 - l): coarse elements take the
  // mean of their eight children; a p-coarsened level keeps its mesh's factors
  std::vector<std::vector<double>> fac(nl);
  if (c->factor) {
    fac[0].resize(c->g.E);
    cudaMemcpy(fac[0].data(), c->factor, c->g.E * sizeof(double), cudaMemcpyDeviceToHost);
    for (int k = 1; k < nl; ++k) {
      const int Nf = Ns[k - 1], Ncs = Ns[k];
      if (Nf == Ncs) {
        fac[k] = fac[k - 1];
        continue;
      }
      fac[k].assign((size_t)Ncs * Ncs * Ncs, 0.0);
      for (int z = 0; z < Nf; ++z)
        for (int y = 0; y < Nf; ++y)
          for (int x = 0; x < Nf; ++x)
            fac[k][(x / 2) + (size_t)Ncs * ((y / 2) + (size_t)Ncs * (z / 2))] +=
                0.125 * fac[k - 1][x + (size_t)Nf * (y + (size_t)Nf * z)];
    }
  }
  for (int l = 0; l < nl; ++l) {
    const int k = nl - 1 - l;  // index in Ns / Ps (0 = finest)
    GmgLevel& L = G.L[l];
    if (l == nl - 1) {
      L.ctx = c;
    } else {
      nhmf_params prm = c->prm;
      prm.n_el = Ns[k];
      prm.degree = Ps[k];
      nhmf_status st = create_context(&prm, &L.ctx);
      if (st != NHMF_OK) {
        gmg_free(c);
        return fail(c, st, "gmg: level context");
      }
      if (c->factor) {
        double* dev = nullptr;
        bool fok = cudaMalloc(&dev, fac[k].size() * sizeof(double)) == cudaSuccess &&
                   cudaMemcpy(dev, fac[k].data(), fac[k].size() * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess;
        if (fok) st = nhmf_set_material_factors(L.ctx, dev, nullptr);
        cudaFree(dev);
        if (!fok || st != NHMF_OK) {
          gmg_free(c);
          return fail(c, NHMF_ERR_OOM, "gmg: level factors");
        }
      }
    }
    if (ensure_work(L.ctx) != NHMF_OK) {
      gmg_free(c);
      return fail(c, NHMF_ERR_OOM, "gmg: level work");
    }
    L.M = Ps[k] * Ns[k] + 1;
    L.n = 3LL * L.M * L.M * L.M;
    bool ok = true;
    for (double** p : {&L.diag, &L.dinv, &L.x, &L.b, &L.r, &L.d, &L.q, &L.t1, &L.t2})
      ok = ok && cudaMalloc(p, L.n * sizeof(double)) == cudaSuccess;
    for (float** p : {&L.dinv32, &L.x32, &L.b32, &L.r32, &L.d32, &L.q32, &L.t132, &L.t232})
      ok = ok && cudaMalloc(p, L.n * sizeof(float)) == cudaSuccess;
    if (!ok) {
      gmg_free(c);
      return fail(c, NHMF_ERR_OOM, "gmg: level vectors");
    }
  }
  for (int l = 1; l < nl; ++l) {
    GmgLevel& L = G.L[l];
    GmgLevel& C = G.L[l - 1];
    const nhmf_ctx* fc = L.ctx;
    const nhmf_ctx* cc = C.ctx;
    std::vector<int> ptr, col, tp, tc;
    std::vector<double> w, tw;
    // prolongation: fine nodes from the coarse function; restriction: its transpose;
    // interpolation of the linearisation point: coarse nodes from the fine function
    build_eval_map(fc->tab.nodes, fc->g.p, fc->g.N, cc->tab.nodes, cc->g.p, cc->g.N, ptr, col, w);
    bool ok = upload(L.P, L.M, C.M, ptr, col, w);
    transpose_map(L.M, C.M, ptr, col, w, tp, tc, tw);
    ok = ok && upload(L.R, C.M, L.M, tp, tc, tw);
    build_eval_map(cc->tab.nodes, cc->g.p, cc->g.N, fc->tab.nodes, fc->g.p, fc->g.N, ptr, col, w);
    ok = ok && upload(L.I, C.M, L.M, ptr, col, w);
    if (!ok) {
      gmg_free(c);
      return fail(c, NHMF_ERR_OOM, "gmg: transfer maps");
    }
  }
  return NHMF_OK;
}

// Power iteration for the largest eigenvalue of D^-1 A on level L in precision T (12 steps).
// The vector is normalised on the device; the host reads the two norms once at the end.
template <typename T>
nhmf_status power_iteration(nhmf_ctx* c, GmgLevel& L, int strategy, cudaStream_t s) {
  T* x = Buf<T>::x(L);
  T* q = Buf<T>::q(L);
  const T* dinv = Buf<T>::dinv(L);
  double* sc = L.ctx->work->sc;
  nhmf_status st;
  k_start<<<kB, kT, 0, s>>>(L.n, L.x);
  if constexpr (sizeof(T) == 4) k_to<float><<<kB, kT, 0, s>>>(L.n, L.x, L.x32);
  for (int it = 0; it < 12; ++it) {
    if ((st = launch_apply(L.ctx, sizeof(T) == 8 ? NHMF_FP64 : NHMF_FP32, strategy, x, q, s)) != NHMF_OK) return st;
    k_mul_t<T><<<kB, kT, 0, s>>>(L.n, dinv, q);
    norm2(L.n, x, sc + 40, L.ctx->work->partials, s);
    norm2(L.n, q, sc + 41, L.ctx->work->partials, s);
    cudaMemcpyAsync(x, q, L.n * sizeof(T), cudaMemcpyDeviceToDevice, s);
    k_scale_inv<T><<<kB, kT, 0, s>>>(L.n, sc + 41, x);
  }
  double h[2];
  cudaMemcpyAsync(h, sc + 40, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if ((st = cuda_check(c, cudaStreamSynchronize(s), "gmg power iteration")) != NHMF_OK) return st;
  L.lmax = (h[0] > 0.0 && h[1] > 0.0) ? h[1] / h[0] : 2.0;
  return NHMF_OK;
}

// Level linearisation points, diagonals and eigenvalue estimates at the fine point c->ubar.
nhmf_status gmg_prepare(nhmf_ctx* c, int strategy, bool fp32, cudaStream_t s, bool coarse_at_zero,
                        const double* fine_diag) {
  nhmf_status st = gmg_build(c);
  if (st != NHMF_OK) return st;
  Gmg& G = *c->gmg;
  const int nl = (int)G.L.size();
  const int mask = strategy == NHMF_CACHED ? (NHMF_CACHE_FP64 | (fp32 ? NHMF_CACHE_FP32 : 0))
                   : strategy == NHMF_SPATIAL ? NHMF_CACHE_SPATIAL : 0;
  for (int l = nl - 2; l >= 0; --l) {
    GmgLevel& F = G.L[l + 1];
    GmgLevel& C = G.L[l];
    if (coarse_at_zero)
      cudaMemsetAsync(C.x, 0, C.n * sizeof(double), s);  // linear elasticity on the coarse levels
    else
      map3d<double>(F.I, F.ctx->ubar, C.x, F.t1, F.t2, s);
    if ((st = nhmf_set_linearization(C.ctx, C.x, mask, s)) != NHMF_OK)
      return fail(c, st, std::string("gmg: coarse linearisation: ") + nhmf_last_error(C.ctx));
  }
  for (int l = 0; l < nl; ++l) {
    GmgLevel& L = G.L[l];
    if (l == nl - 1 && fine_diag)  // the fine level's diagonal, computed by the caller
      cudaMemcpyAsync(L.diag, fine_diag, L.n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    else if ((st = launch_diagonal(L.ctx, L.diag, s)) != NHMF_OK)
      return st;
    reciprocal(L.n, L.diag, L.dinv, L.dinv32, s);
    if (l == 0) continue;  // the coarsest level is solved, not smoothed
    // in the precision of the V-cycle (Algorithm 2 has no FP32 apply)
    st = (fp32 && strategy != NHMF_SPATIAL) ? power_iteration<float>(c, L, strategy, s)
                                            : power_iteration<double>(c, L, strategy, s);
    if (st != NHMF_OK) return st;
  }
  return cuda_check(c, cudaGetLastError(), "gmg prepare");
}



// Chebyshev iteration of `degree` steps on D^-1 A for A x = b, on the interval
// [lmax/range, lmax] (lmax = 1.2 x the power-iteration estimate); x = 0 on entry if zero_start.
template <typename T>
nhmf_status chebyshev(GmgLevel& L, int strat, const T* b, T* x, int degree, double range, bool zero_start,
                      cudaStream_t s) {
  const double lmax = 1.2 * L.lmax, lmin = lmax / range;
  const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma = theta / delta;
  double rho = 1.0 / sigma;
  T* d = Buf<T>::d(L);
  T* q = Buf<T>::q(L);
  nhmf_status st = NHMF_OK;
  for (int j = 0; j < degree; ++j) {
    const bool first = j == 0;
    const T* qq = nullptr;
    if (!(first && zero_start)) {
      if ((st = launch_apply(L.ctx, Buf<T>::prec, strat, x, q, s)) != NHMF_OK) return st;
      qq = q;
    }
    T c_old, c_new;
    if (first) {
      c_old = T(0);
      c_new = T(1.0 / theta);
    } else {
      const double rho_new = 1.0 / (2.0 * sigma - rho);
      c_old = T(rho_new * rho);
      c_new = T(2.0 * rho_new / delta);
      rho = rho_new;
    }
    if (first && !zero_start) {
      // d = D^-1 (b - A x) / theta, x += d
      k_cheb<T><<<kB, kT, 0, s>>>(L.n, b, qq, Buf<T>::dinv(L), d, x, T(0), c_new);
    } else {
      k_cheb<T><<<kB, kT, 0, s>>>(L.n, b, qq, Buf<T>::dinv(L), d, x, c_old, c_new);
    }
  }
  return cuda_check(L.ctx, cudaGetLastError(), "chebyshev");
}

// r_coarse = R r_fine (transpose of the prolongation), fine level `F`
template <typename T>
void gmg_restrict(GmgLevel& F, const T* r_fine, T* r_coarse, cudaStream_t s) {
  map3d<T>(F.R, r_fine, r_coarse, Buf<T>::t1(F), Buf<T>::t2(F), s);
}

// x_fine += P e_coarse, through the fine level's q buffer
template <typename T>
void gmg_prolong_add(GmgLevel& F, const T* e_coarse, T* x_fine, T* scratch, cudaStream_t s) {
  map3d<T>(F.P, e_coarse, scratch, Buf<T>::t1(F), Buf<T>::t2(F), s);
  k_add<T><<<kB, kT, 0, s>>>(F.n, scratch, x_fine);
}

void gmg_start_vector(long long n, double* v, cudaStream_t s) { k_start<<<kB, kT, 0, s>>>(n, v); }

template <typename T>
void gmg_bminus(long long n, const T* b, T* y, cudaStream_t s) {
  k_bminus<T><<<kB, kT, 0, s>>>(n, b, y);
}

template nhmf_status chebyshev<double>(GmgLevel&, int, const double*, double*, int, double, bool, cudaStream_t);
template nhmf_status chebyshev<float>(GmgLevel&, int, const float*, float*, int, double, bool, cudaStream_t);
template void gmg_restrict<double>(GmgLevel&, const double*, double*, cudaStream_t);
template void gmg_restrict<float>(GmgLevel&, const float*, float*, cudaStream_t);
template void gmg_prolong_add<double>(GmgLevel&, const double*, double*, double*, cudaStream_t);
template void gmg_prolong_add<float>(GmgLevel&, const float*, float*, float*, cudaStream_t);
template void gmg_bminus<double>(long long, const double*, double*, cudaStream_t);
template void gmg_bminus<float>(long long, const float*, float*, cudaStream_t);

}  // namespace nhmf
