// Geometric multigrid on the nested structured meshes (see gmg.cu).
#pragma once
#include <vector>

#include "internal.h"

namespace nhmf {

// A 1D linear map between node lines, as CSR rows: out[i] = sum_k w[k] in[col[k]], k in [ptr[i], ptr[i+1]).
struct Map1D {
  int rows = 0, cols = 0;
  int *ptr = nullptr, *col = nullptr;  // device
  double* w64 = nullptr;
  float* w32 = nullptr;
};

struct GmgLevel {
  nhmf_ctx* ctx = nullptr;  // level context (owned; index 0 = coarsest)
  long long n = 0;          // DoFs
  int M = 0;
  double lmax = 0.0;        // estimate of the largest eigenvalue of D^-1 A
  double *diag = nullptr, *dinv = nullptr;
  float* dinv32 = nullptr;
  double *x = nullptr, *b = nullptr, *r = nullptr, *d = nullptr, *q = nullptr, *t1 = nullptr, *t2 = nullptr;
  float *x32 = nullptr, *b32 = nullptr, *r32 = nullptr, *d32 = nullptr, *q32 = nullptr, *t132 = nullptr, *t232 = nullptr;
  Map1D P;   // prolongation from the next coarser level to this one (rows: this level's M)
  Map1D R;   // its transpose (rows: the coarser level's M)
  Map1D I;   // interpolation of the linearisation point from this level to the coarser one
};

struct Gmg {
  std::vector<GmgLevel> L;  // L.back() mirrors the fine context (its ctx pointer is not owned)
};

void gmg_free(nhmf_ctx* c);
nhmf_status gmg_build(nhmf_ctx* c);
// Level linearisation points (interpolated from the fine one, or zero on the coarse levels),
// diagonals and eigenvalue estimates.
// fine_diag: the fine operator's diagonal if the caller has it (else it is computed).
nhmf_status gmg_prepare(nhmf_ctx* c, int strategy, bool fp32, cudaStream_t s, bool coarse_at_zero,
                        const double* fine_diag = nullptr);
// per-level buffers by precision
template <typename T> struct Buf;
template <> struct Buf<double> {
  static double* x(GmgLevel& l) { return l.x; }
  static double* b(GmgLevel& l) { return l.b; }
  static double* r(GmgLevel& l) { return l.r; }
  static double* d(GmgLevel& l) { return l.d; }
  static double* q(GmgLevel& l) { return l.q; }
  static double* t1(GmgLevel& l) { return l.t1; }
  static double* t2(GmgLevel& l) { return l.t2; }
  static const double* dinv(GmgLevel& l) { return l.dinv; }
  static constexpr int prec = NHMF_FP64;
};
template <> struct Buf<float> {
  static float* x(GmgLevel& l) { return l.x32; }
  static float* b(GmgLevel& l) { return l.b32; }
  static float* r(GmgLevel& l) { return l.r32; }
  static float* d(GmgLevel& l) { return l.d32; }
  static float* q(GmgLevel& l) { return l.q32; }
  static float* t1(GmgLevel& l) { return l.t132; }
  static float* t2(GmgLevel& l) { return l.t232; }
  static const float* dinv(GmgLevel& l) { return l.dinv32; }
  static constexpr int prec = NHMF_FP32;
};

template <typename T>
nhmf_status chebyshev(GmgLevel& L, int strat, const T* b, T* x, int degree, double range, bool zero_start,
                      cudaStream_t s);
template <typename T> void gmg_restrict(GmgLevel& F, const T* r_fine, T* r_coarse, cudaStream_t s);
template <typename T> void gmg_prolong_add(GmgLevel& F, const T* e_coarse, T* x_fine, T* scratch, cudaStream_t s);
template <typename T> void gmg_bminus(long long n, const T* b, T* y, cudaStream_t s);
void gmg_start_vector(long long n, double* v, cudaStream_t s);

}  // namespace nhmf
