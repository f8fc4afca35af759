// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdio>

#include <string>
#include <vector>

#include "../../include/nhmf.h"

namespace nhmf {

constexpr int kMaxN = 5;  // p + 1 for p <= 4

// FP32 applies up to degree kRegMaxP use the one-element-per-thread register kernel (with its
// [10][n^3][E] point-cache layout) when every colour class has at least kRegMinColour
// elements; smaller meshes (coarse multigrid levels) and higher degrees use the shared-memory
// kernel, whose latency per launch does not grow with the element's work.
#ifndef NHMF_REG_MAXP
#define NHMF_REG_MAXP 2
#endif
#ifndef NHMF_REG_MIN_COLOUR
#define NHMF_REG_MIN_COLOUR 32768
#endif
constexpr int kRegMaxP = NHMF_REG_MAXP;
constexpr long long kRegMinColour = NHMF_REG_MIN_COLOUR;

// Element tiles of the FP32 apply's arrays: per-element data of 32 consecutive elements (in
// natural order) are stored value-row by value-row, [E / kTile][values][kTile], so that a
// warp of one-thread-per-element code reads and writes whole 128-byte rows and every warp's
// data is one contiguous block (DRAM pages and TLB entries stay few).
constexpr int kTile = 32;
inline long long tiled_elems(long long E) { return (E + kTile - 1) / kTile * kTile; }

// 1D tables of the Q_p element on [0, 1] (Section 2.2, 2.4), FP64.
//   B[q][i]  = l_i(x_q): GLL Lagrange basis at the Gauss points
//   Dc[q][r] = derivative of the Lagrange basis on the Gauss points, at Gauss point q
//              (collocation derivative: exact for polynomials of degree <= p)
//   D[q][i]  = l_i'(x_q) = sum_r Dc[q][r] B[r][i]
//   w[q]     = Gauss weights on [0, 1]
struct Tables1D {
  int n;
  double nodes[kMaxN], xq[kMaxN], w[kMaxN];
  double B[kMaxN][kMaxN], Dc[kMaxN][kMaxN], D[kMaxN][kMaxN];
};
void build_tables(int p, Tables1D* t);

// Geometry of one element colour class: elements (cx + s ix, cy + s iy, cz + s iz), s = stride:
// 2 for the eight classes of the colour-by-colour scatter, 1 for the class of all elements
// (natural order), which the element-local FP32 apply uses.
struct Colour {
  int cx, cy, cz;
  int nx, ny, nz;
  int count;        // nx * ny * nz
  long long slot0;  // first colour-major element slot of this class
  int stride;
};

struct Geometry {
  int N, p, n, M;
  long long M3;      // nodes
  long long E;       // elements
  long long nq;      // quadrature points, E * n^3
  double h;
  Colour colour[8];
  Colour all;        // every element, natural order ex + N (ey + N ez)
};

}  // namespace nhmf

namespace nhmf {
struct UNet;
struct Gmg;
// Work vectors of the solvers, allocated on first use.
struct SolverWork {
  long long n = 0;
  double *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *qprev = nullptr, *x = nullptr;
  double *b = nullptr, *R = nullptr, *d = nullptr, *t = nullptr, *du = nullptr, *utry = nullptr;
  double *diag = nullptr, *dinv = nullptr, *b2 = nullptr, *x2 = nullptr;
  float *r32 = nullptr, *z32 = nullptr, *p32 = nullptr, *q32 = nullptr, *x32 = nullptr, *b32 = nullptr, *dinv32 = nullptr;
  double* sc = nullptr;        // device scalars
  double* partials = nullptr;  // reduction scratch
  double* host = nullptr;      // pinned host scalar
  cudaStream_t stream = nullptr;  // the solvers' own stream (graph capture needs a non-legacy stream)
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  // CUDA graphs of `check_every` CG iterations, keyed by the buffers they were captured with
  struct Graph {
    cudaGraphExec_t exec = nullptr;
    const void* key[16] = {};
  } graph[2];  // [0] FP64, [1] FP32
};
}  // namespace nhmf

struct nhmf_ctx {
  nhmf_params prm;
  nhmf::Geometry g;
  nhmf::Tables1D tab;
  int device = 0;
  double* ubar = nullptr;     // linearisation point, FP64
  float* ubar32 = nullptr;    // its FP32 copy (FP32 on-the-fly apply)
  double* cache64 = nullptr;  // [10][nq]
  float* cache32 = nullptr;   // FP32 point cache, elements in natural order (see kTile)
  float* vloc = nullptr;      // element-local results of the FP32 apply, [E/32][3][(p+1)^3][32]
  float2* cachedf = nullptr;  // [10][nq] (hi, lo) double-float pairs
  double* cachesp = nullptr;  // [36][nq] J c (21), tau (6), F^-1 (9): Algorithm 2
  double* factor = nullptr;   // [E] per-element material factors (natural order), or null
  unsigned* status = nullptr; // device status word: bit 0 det F <= 0, bit 1 non-finite
  bool have_lin = false;
  bool reg32 = false;  // FP32 applies on the register kernel (see kRegMinColour)
  const double* u_at = nullptr;  // set only while nhmf_tangent_apply_at launches its apply
  std::string err;
  // kernel timing (nhmf_profile_enable): event pairs per operator kind
  bool profiling = false;
  struct Rec { int kind; int launches; cudaEvent_t a, b; };
  std::vector<Rec> prof;
  nhmf::SolverWork* work = nullptr;
  nhmf::UNet* unet = nullptr;
  nhmf::Gmg* gmg = nullptr;    // multigrid hierarchy, built on first use
  unsigned inject = 0;         // pending NHMF_INJECT_* flags (host-side fault injection)
  FILE* metrics = nullptr;     // JSONL metrics file (nhmf_set_metrics_log), or null
};

namespace nhmf {

// NVTX range for the lifetime of the object (no cost without a profiler attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
// One JSON object (printf-style body without the braces) as a line of the metrics file.
void metrics_line(nhmf_ctx* c, const char* fmt, ...);
// Takes a pending injection flag: true (and the flag cleared) if it was set.
inline bool take_inject(nhmf_ctx* c, unsigned flag) {
  if (!(c->inject & flag)) return false;
  c->inject &= ~flag;
  return true;
}

enum : unsigned { kStatusNonPosJ = 1u, kStatusNonFinite = 2u, kStatusBreakdown = 4u, kStatusTcTimeout = 8u, kStatusTmaSetup = 16u };
void free_work(nhmf_ctx* c);
nhmf_status ensure_work(nhmf_ctx* c);

// U-Net preconditioner (unet.cu)
nhmf_status unet_alloc(nhmf_ctx* c, int pair_capacity);
void unet_free(nhmf_ctx* c);
void unet_refresh_weights(UNet& u, cudaStream_t s);
void unet_forward(UNet& u, cudaStream_t s);
void unet_backward(UNet& u, cudaStream_t s);
void unet_input_planar32(UNet& u, const float* x, cudaStream_t s);
void unet_loss_and_grad(nhmf_ctx* c, const float* target, bool accumulate, cudaStream_t s);
void unet_adam(UNet& u, float lr, cudaStream_t s);
void unet_precondition(nhmf_ctx* c, const double* r, double* z, cudaStream_t s);
nhmf_status unet_record(nhmf_ctx* c, const double* r, const double* e, cudaStream_t s);
void unet_smooth_field(nhmf_ctx* c, double* e, unsigned long long seed, cudaStream_t s);
int unet_snapshot_begin(nhmf_ctx* c, const double* r, const double* xj, cudaStream_t s);
void unet_snapshot_finish(nhmf_ctx* c, int slot, const double* xstar, cudaStream_t s);

// raw = true applies the unconstrained operator K (no Dirichlet masking or identity rows).
nhmf_status launch_apply(nhmf_ctx* c, int precision, int strategy, const void* du, void* v,
                         cudaStream_t s, bool raw = false);
// On every constrained DoF: out = src (mode 0) or out = value (mode 1).
nhmf_status fix_rows64(nhmf_ctx* c, const double* src, double* out, int mode, double value, cudaStream_t s);
nhmf_status fix_rows32(nhmf_ctx* c, const float* src, float* out, int mode, float value, cudaStream_t s);
nhmf_status launch_cache_build(nhmf_ctx* c, cudaStream_t s);
nhmf_status launch_residual(nhmf_ctx* c, const double* u, double* r, cudaStream_t s);
nhmf_status launch_diagonal(nhmf_ctx* c, double* d, cudaStream_t s);
nhmf_status launch_to_fp32(const double* x, float* y, long long n, cudaStream_t s);

nhmf_status fail(nhmf_ctx* c, nhmf_status st, const std::string& msg);
nhmf_status cuda_check(nhmf_ctx* c, cudaError_t e, const char* what);

// Resolves, once per device, the device address of the allocation-free solve's static
// scratch array (noalloc.cu); called by nhmf_create with the context's device current.
nhmf_status noalloc_setup(nhmf_ctx* c);
// nhmf_create without the environment (NHMF_INJECT, NHMF_METRICS_JSONL): internal contexts.
nhmf_status create_context(const nhmf_params* prm, nhmf_ctx** out);

}  // namespace nhmf
