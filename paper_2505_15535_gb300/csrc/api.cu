// C ABI of the library (declarations and contracts in include/nhmf.h).
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "gmg.h"
#include "internal.h"

namespace nhmf {

nhmf_status fail(nhmf_ctx* c, nhmf_status st, const std::string& msg) {
  if (c) c->err = msg;
  return st;
}

nhmf_status cuda_check(nhmf_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return NHMF_OK;
  return fail(c, e == cudaErrorMemoryAllocation ? NHMF_ERR_OOM : NHMF_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

static void build_geometry(const nhmf_params& p, Geometry* g) {
  g->N = p.n_el;
  g->p = p.degree;
  g->n = p.degree + 1;
  g->M = p.degree * p.n_el + 1;
  g->M3 = (long long)g->M * g->M * g->M;
  g->E = (long long)p.n_el * p.n_el * p.n_el;
  g->nq = g->E * g->n * g->n * g->n;
  g->h = 1.0 / p.n_el;
  long long slot = 0;
  for (int k = 0; k < 8; ++k) {
    Colour& c = g->colour[k];
    c.cx = k & 1;
    c.cy = (k >> 1) & 1;
    c.cz = (k >> 2) & 1;
    c.nx = (p.n_el - c.cx + 1) / 2;
    c.ny = (p.n_el - c.cy + 1) / 2;
    c.nz = (p.n_el - c.cz + 1) / 2;
    c.count = c.nx * c.ny * c.nz;
    c.slot0 = slot;
    c.stride = 2;
    slot += c.count;
  }
  g->all = Colour{0, 0, 0, p.n_el, p.n_el, p.n_el, (int)g->E, 0, 1};
}

static cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

void metrics_line(nhmf_ctx* c, const char* fmt, ...) {
  if (!c || !c->metrics) return;
  va_list ap;
  va_start(ap, fmt);
  std::fputc('{', c->metrics);
  std::vfprintf(c->metrics, fmt, ap);
  std::fputs("}\n", c->metrics);
  va_end(ap);
  std::fflush(c->metrics);
}

static nhmf_status open_metrics(nhmf_ctx* c, const char* path) {
  if (c->metrics) std::fclose(c->metrics);
  c->metrics = nullptr;
  if (!path || !*path) return NHMF_OK;
  c->metrics = std::fopen(path, "a");
  return c->metrics ? NHMF_OK : fail(c, NHMF_ERR_ARG, std::string("metrics log: cannot open ") + path);
}

nhmf_status create_context(const nhmf_params* prm, nhmf_ctx** out) {
  if (!prm || !out) return NHMF_ERR_ARG;
  *out = nullptr;
  if (prm->n_el < 1 || prm->n_el > 4096 || prm->degree < 1 || prm->degree > 4 || !(prm->mu > 0.0) ||
      !(prm->lambda >= 0.0) || prm->bc < NHMF_BC_NONE || prm->bc > NHMF_BC_COMPRESSION ||
      (prm->model != NHMF_MODEL_COMPRESSIBLE && prm->model != NHMF_MODEL_SPLIT))
    return NHMF_ERR_ARG;
  nhmf_ctx* c = new (std::nothrow) nhmf_ctx();
  if (!c) return NHMF_ERR_OOM;
  c->prm = *prm;
  build_geometry(*prm, &c->g);
  build_tables(prm->degree, &c->tab);
  long long min_colour = c->g.colour[0].count;
  for (int k = 1; k < 8; ++k) min_colour = std::min<long long>(min_colour, c->g.colour[k].count);
  c->reg32 = prm->degree <= kRegMaxP && min_colour >= kRegMinColour;
  cudaGetDevice(&c->device);
  nhmf_status st = cuda_check(c, cudaMalloc(&c->status, sizeof(unsigned)), "status alloc");
  if (st == NHMF_OK) st = cuda_check(c, cudaMemset(c->status, 0, sizeof(unsigned)), "status clear");
  if (st == NHMF_OK) st = cuda_check(c, cudaMalloc(&c->ubar, sizeof(double) * 3 * c->g.M3), "ubar alloc");
  if (st == NHMF_OK) st = cuda_check(c, cudaMalloc(&c->ubar32, sizeof(float) * 3 * c->g.M3), "ubar32 alloc");
  if (st == NHMF_OK) st = noalloc_setup(c);
  if (st != NHMF_OK) {
    nhmf_destroy(c);
    return st;
  }
  *out = c;
  return NHMF_OK;
}

static const char* precision_name(int p) { return p == NHMF_FP64 ? "fp64" : p == NHMF_FP32 ? "fp32" : "df64"; }
static const char* strategy_name(int s) {
  return s == NHMF_CACHED ? "cached" : s == NHMF_ON_THE_FLY ? "on_the_fly" : "spatial";
}

}  // namespace nhmf

using namespace nhmf;

extern "C" {

nhmf_status nhmf_create(const nhmf_params* prm, nhmf_ctx** out) {
  nhmf_status st = create_context(prm, out);
  if (st != NHMF_OK) return st;
  nhmf_ctx* c = *out;
  c->inject = nhmf_parse_inject(std::getenv("NHMF_INJECT")) & ~(unsigned)NHMF_INJECT_UNKNOWN;
  if ((st = open_metrics(c, std::getenv("NHMF_METRICS_JSONL"))) != NHMF_OK) {
    nhmf_destroy(c);
    *out = nullptr;
  }
  return st;
}

void nhmf_destroy(nhmf_ctx* c) {
  if (!c) return;
  cudaDeviceSynchronize();
  for (auto& r : c->prof) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  cudaFree(c->status);
  cudaFree(c->ubar);
  cudaFree(c->ubar32);
  cudaFree(c->cache64);
  cudaFree(c->cache32);
  cudaFree(c->vloc);
  cudaFree(c->cachedf);
  cudaFree(c->cachesp);
  gmg_free(c);
  free_work(c);
  unet_free(c);
  if (c->metrics) std::fclose(c->metrics);
  delete c;
}

unsigned nhmf_parse_inject(const char* spec) {
  unsigned flags = 0;
  if (!spec) return 0;
  const char* p = spec;
  while (*p) {
    while (*p == ',' || *p == ' ') ++p;
    const char* q = p;
    while (*q && *q != ',' && *q != ' ') ++q;
    const std::string name(p, (size_t)(q - p));
    if (name == "nan_in_du")
      flags |= NHMF_INJECT_NAN_DU;
    else if (name == "cg_stall")
      flags |= NHMF_INJECT_CG_STALL;
    else if (name == "unet_garbage")
      flags |= NHMF_INJECT_UNET_GARBAGE;
    else if (!name.empty())
      flags |= NHMF_INJECT_UNKNOWN;
    p = q;
  }
  return flags;
}

nhmf_status nhmf_set_inject(nhmf_ctx* c, unsigned flags) {
  if (!c) return NHMF_ERR_ARG;
  if (flags & ~(unsigned)(NHMF_INJECT_NAN_DU | NHMF_INJECT_CG_STALL | NHMF_INJECT_UNET_GARBAGE))
    return fail(c, NHMF_ERR_ARG, "set_inject: unknown flag");
  c->inject = flags;
  return NHMF_OK;
}

unsigned nhmf_inject_pending(const nhmf_ctx* c) { return c ? c->inject : 0; }

nhmf_status nhmf_set_metrics_log(nhmf_ctx* c, const char* path) {
  if (!c) return NHMF_ERR_ARG;
  return open_metrics(c, path);
}

size_t nhmf_num_dofs(const nhmf_ctx* c) { return c ? (size_t)(3 * c->g.M3) : 0; }

const char* nhmf_last_error(const nhmf_ctx* c) { return c ? c->err.c_str() : "null context"; }

nhmf_status nhmf_set_material_factors(nhmf_ctx* c, const double* factors, void* stream) {
  if (!c) return NHMF_ERR_ARG;
  cudaStream_t s = as_stream(stream);
  gmg_free(c);  // the coarse levels carry the factors: rebuild them on next use
  if (!factors) {
    cudaFree(c->factor);
    c->factor = nullptr;
    return NHMF_OK;
  }
  nhmf_status st = NHMF_OK;
  if (!c->factor) st = cuda_check(c, cudaMalloc(&c->factor, c->g.E * sizeof(double)), "factor alloc");
  if (st == NHMF_OK)
    st = cuda_check(c, cudaMemcpyAsync(c->factor, factors, c->g.E * sizeof(double), cudaMemcpyDeviceToDevice, s),
                    "factor copy");
  if (st == NHMF_OK) st = cuda_check(c, cudaStreamSynchronize(s), "factor sync");
  return st;
}

nhmf_status nhmf_check_status(nhmf_ctx* c, void* stream) {
  if (!c) return NHMF_ERR_ARG;
  unsigned h = 0;
  cudaStream_t s = as_stream(stream);
  nhmf_status st = cuda_check(c, cudaMemcpyAsync(&h, c->status, sizeof(unsigned), cudaMemcpyDeviceToHost, s), "status read");
  if (st == NHMF_OK) st = cuda_check(c, cudaStreamSynchronize(s), "status sync");
  if (st == NHMF_OK) st = cuda_check(c, cudaMemsetAsync(c->status, 0, sizeof(unsigned), s), "status clear");
  if (st != NHMF_OK) return st;
  if (h & kStatusNonPosJ) return fail(c, NHMF_ERR_NONPOS_J, "det F <= 0 at a quadrature point");
  if (h & kStatusNonFinite) return fail(c, NHMF_ERR_NONFINITE, "non-finite value");
  if (h & kStatusBreakdown) return fail(c, NHMF_ERR_BREAKDOWN, "Krylov breakdown: p^T A p <= 0");
  if (h & kStatusTcTimeout) return fail(c, NHMF_ERR_CUDA, "tensor-core completion wait timed out");
  if (h & kStatusTmaSetup) return fail(c, NHMF_ERR_CUDA, "tensor-map encoding for a convolution failed");
  return NHMF_OK;
}

nhmf_status nhmf_set_linearization(nhmf_ctx* c, const double* u, int mask, void* stream) {
  if (!c || !u || mask < 0 || mask > 15) return fail(c, NHMF_ERR_ARG, "set_linearization: bad argument");
  if (c->prm.model == NHMF_MODEL_SPLIT && (mask & (NHMF_CACHE_FP64 | NHMF_CACHE_FP32 | NHMF_CACHE_DF64)))
    return fail(c, NHMF_ERR_ARG, "set_linearization: the split model has only the spatial (Algorithm 2) cache");
  NvtxRange range("nhmf_set_linearization");
  cudaStream_t s = as_stream(stream);
  const size_t n = 3 * c->g.M3;
  c->have_lin = false;
  nhmf_status st = cuda_check(c, cudaMemcpyAsync(c->ubar, u, n * sizeof(double), cudaMemcpyDeviceToDevice, s), "ubar copy");
  if (st != NHMF_OK) return st;
  if ((st = launch_to_fp32(c->ubar, c->ubar32, (long long)n, s)) != NHMF_OK)
    return fail(c, st, "ubar fp32 copy");
  const size_t cache_elems = 10 * (size_t)c->g.nq;
  // element-local results of the FP32 apply (allocated here, before any solver captures an
  // FP32 apply in a CUDA graph)
  const size_t tiled_nq = (size_t)tiled_elems(c->g.E) * c->g.n * c->g.n * c->g.n;
  if (!c->vloc)
    if ((st = cuda_check(c, cudaMalloc(&c->vloc, 3 * tiled_nq * sizeof(float)), "vloc alloc")) != NHMF_OK) return st;
  if ((mask & NHMF_CACHE_FP64) && !c->cache64)
    if ((st = cuda_check(c, cudaMalloc(&c->cache64, cache_elems * sizeof(double)), "cache64 alloc")) != NHMF_OK) return st;
  if ((mask & NHMF_CACHE_FP32) && !c->cache32)
    if ((st = cuda_check(c, cudaMalloc(&c->cache32, 10 * tiled_nq * sizeof(float)), "cache32 alloc")) != NHMF_OK) return st;
  if ((mask & NHMF_CACHE_SPATIAL) && !c->cachesp)
    if ((st = cuda_check(c, cudaMalloc(&c->cachesp, 36 * (size_t)c->g.nq * sizeof(double)), "cachesp alloc")) != NHMF_OK)
      return st;
  if (!(mask & NHMF_CACHE_SPATIAL) && c->cachesp) { cudaFree(c->cachesp); c->cachesp = nullptr; }
  if ((mask & NHMF_CACHE_DF64) && !c->cachedf)
    if ((st = cuda_check(c, cudaMalloc(&c->cachedf, cache_elems * sizeof(float2)), "cachedf alloc")) != NHMF_OK) return st;
  if (!(mask & NHMF_CACHE_DF64) && c->cachedf) { cudaFree(c->cachedf); c->cachedf = nullptr; }
  if (!(mask & NHMF_CACHE_FP64) && c->cache64) { cudaFree(c->cache64); c->cache64 = nullptr; }
  if (!(mask & NHMF_CACHE_FP32) && c->cache32) { cudaFree(c->cache32); c->cache32 = nullptr; }
  if (mask) {
    if ((st = launch_cache_build(c, s)) != NHMF_OK) return st;
  }
  if ((st = nhmf_check_status(c, stream)) != NHMF_OK) return st;
  c->have_lin = true;
  return NHMF_OK;
}

nhmf_status nhmf_tangent_apply(nhmf_ctx* c, int precision, int strategy, const void* du, void* v, void* stream) {
  if (!c) return NHMF_ERR_ARG;
  if (!du || !v || du == v || (precision != NHMF_FP64 && precision != NHMF_FP32 && precision != NHMF_DF64) ||
      (strategy != NHMF_ON_THE_FLY && strategy != NHMF_CACHED && strategy != NHMF_SPATIAL))
    return fail(c, NHMF_ERR_ARG, "tangent_apply: bad argument");
  if (c->prm.model == NHMF_MODEL_SPLIT && (strategy == NHMF_CACHED || precision == NHMF_DF64))
    return fail(c, NHMF_ERR_ARG, "tangent_apply: the split model supports NHMF_ON_THE_FLY and NHMF_SPATIAL");
  if (strategy == NHMF_SPATIAL && precision != NHMF_FP64)
    return fail(c, NHMF_ERR_ARG, "tangent_apply: NHMF_SPATIAL is FP64 only");
  if (strategy == NHMF_SPATIAL && !c->cachesp)
    return fail(c, NHMF_ERR_STATE, "tangent_apply: no NHMF_CACHE_SPATIAL cache");
  if (!c->have_lin) return fail(c, NHMF_ERR_STATE, "tangent_apply: no linearisation point set");
  if (precision == NHMF_DF64 && strategy != NHMF_CACHED)
    return fail(c, NHMF_ERR_ARG, "tangent_apply: NHMF_DF64 supports the cached strategy only");
  if (strategy == NHMF_CACHED && ((precision == NHMF_FP64 && !c->cache64) || (precision == NHMF_FP32 && !c->cache32) ||
                                  (precision == NHMF_DF64 && !c->cachedf)))
    return fail(c, NHMF_ERR_STATE, "tangent_apply: no point cache of this precision");
  NvtxRange range("nhmf_tangent_apply");
  if (!c->metrics) return launch_apply(c, precision, strategy, du, v, as_stream(stream));
  // timed with events on the caller's stream for the metrics line
  cudaEvent_t e0, e1;
  nhmf_status st = cuda_check(c, cudaEventCreate(&e0), "metrics event");
  if (st != NHMF_OK) return st;
  if ((st = cuda_check(c, cudaEventCreate(&e1), "metrics event")) != NHMF_OK) {
    cudaEventDestroy(e0);
    return st;
  }
  cudaEventRecord(e0, as_stream(stream));
  st = launch_apply(c, precision, strategy, du, v, as_stream(stream));
  cudaEventRecord(e1, as_stream(stream));
  float ms = 0.f;
  if (st == NHMF_OK) st = cuda_check(c, cudaEventSynchronize(e1), "metrics sync");
  if (st == NHMF_OK) st = cuda_check(c, cudaEventElapsedTime(&ms, e0, e1), "metrics time");
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st == NHMF_OK)
    metrics_line(c, "\"event\": \"tangent_apply\", \"precision\": \"%s\", \"strategy\": \"%s\", \"dofs\": %lld, "
                 "\"ms\": %.6f, \"gdofs\": %.6f",
                 precision_name(precision), strategy_name(strategy), 3 * c->g.M3, (double)ms,
                 ms > 0.f ? 3.0 * c->g.M3 / (ms * 1e6) : 0.0);
  return st;
}

nhmf_status nhmf_tangent_apply_at(nhmf_ctx* c, const double* u, const double* du, double* v, void* stream) {
  if (!c) return NHMF_ERR_ARG;
  if (!u || !du || !v || (const void*)du == (void*)v || (const void*)u == (void*)v)
    return fail(c, NHMF_ERR_ARG, "tangent_apply_at: bad argument");
  c->u_at = u;
  const nhmf_status st = launch_apply(c, NHMF_FP64, NHMF_ON_THE_FLY, du, v, as_stream(stream));
  c->u_at = nullptr;
  return st;
}

nhmf_status nhmf_residual(nhmf_ctx* c, const double* u, double* r, void* stream) {
  if (!c) return NHMF_ERR_ARG;
  if (!u || !r || (const void*)u == (void*)r) return fail(c, NHMF_ERR_ARG, "residual: bad argument");
  NvtxRange range("nhmf_residual");
  nhmf_status st = launch_residual(c, u, r, as_stream(stream));
  if (st != NHMF_OK) return st;
  return nhmf_check_status(c, stream);
}

nhmf_status nhmf_diagonal(nhmf_ctx* c, double* d, void* stream) {
  if (!c) return NHMF_ERR_ARG;
  if (!d) return fail(c, NHMF_ERR_ARG, "diagonal: bad argument");
  if (!c->have_lin) return fail(c, NHMF_ERR_STATE, "diagonal: no linearisation point set");
  NvtxRange range("nhmf_diagonal");
  return launch_diagonal(c, d, as_stream(stream));
}

nhmf_status nhmf_profile_enable(nhmf_ctx* c, int enable) {
  if (!c) return NHMF_ERR_ARG;
  c->profiling = enable != 0;
  return NHMF_OK;
}

nhmf_status nhmf_profile_read(nhmf_ctx* c, int kind, double* ms, long long* launches) {
  if (!c || !ms || !launches) return fail(c, NHMF_ERR_ARG, "profile_read: bad argument");
  double total = 0.0;
  long long n = 0;
  std::vector<nhmf_ctx::Rec> keep;
  for (auto& r : c->prof) {
    if (r.kind != kind) {
      keep.push_back(r);
      continue;
    }
    float t = 0.f;
    nhmf_status st = cuda_check(c, cudaEventSynchronize(r.b), "profile sync");
    if (st == NHMF_OK) st = cuda_check(c, cudaEventElapsedTime(&t, r.a, r.b), "profile elapsed");
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
    if (st != NHMF_OK) return st;
    total += t;
    n += r.launches;
  }
  c->prof.swap(keep);
  *ms = total;
  *launches = n;
  return NHMF_OK;
}

}  // extern "C"
