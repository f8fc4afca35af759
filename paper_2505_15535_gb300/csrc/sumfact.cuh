// Device building blocks of the matrix-free operators: launch shapes, shared-memory sum
// factorisation passes and the neo-Hookean point code.
//
// Sum factorisation (Section 2.4): values of a Q_p field at the (p+1)^3 Gauss points of an
// element are three 1D passes with B[q][i] = l_i(x_q), one per direction; reference-cell
// gradients at the points are then one collocation pass Dc per direction.  The transposed
// contraction with the test-function gradients is one combined Dc^T pass followed by three
// B^T passes.  Every pass maps an [n][n][n] block (x fastest) to another, with n = p + 1.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "internal.h"

namespace nhmf {

// Elements per thread block and threads per block for each degree and precision.  Chosen so
// that NE * (p+1)^3 work items fill whole warps and the shared-memory footprint allows
// several blocks per SM.
template <int P, typename T> struct Cfg;
template <> struct Cfg<1, double> { static constexpr int NE = 32, THREADS = 256; };
#ifndef NHMF_Q2D_NE
#define NHMF_Q2D_NE 27
#define NHMF_Q2D_THREADS 256
#endif
#ifndef NHMF_Q4D_NE
#define NHMF_Q4D_NE 3
#define NHMF_Q4D_THREADS 192
#endif
template <> struct Cfg<2, double> { static constexpr int NE = NHMF_Q2D_NE, THREADS = NHMF_Q2D_THREADS; };
template <> struct Cfg<3, double> { static constexpr int NE = 8, THREADS = 256; };
template <> struct Cfg<4, double> { static constexpr int NE = NHMF_Q4D_NE, THREADS = NHMF_Q4D_THREADS; };
template <> struct Cfg<1, float> { static constexpr int NE = 32, THREADS = 256; };
#ifndef NHMF_Q2F_NE
#define NHMF_Q2F_NE 8
#define NHMF_Q2F_THREADS 224
#endif
template <> struct Cfg<2, float> { static constexpr int NE = NHMF_Q2F_NE, THREADS = NHMF_Q2F_THREADS; };
#ifndef NHMF_Q3F_NE
#define NHMF_Q3F_NE 8
#define NHMF_Q3F_THREADS 256
#endif
#ifndef NHMF_Q4F_NE
#define NHMF_Q4F_NE 4
#define NHMF_Q4F_THREADS 160
#endif
template <> struct Cfg<3, float> { static constexpr int NE = NHMF_Q3F_NE, THREADS = NHMF_Q3F_THREADS; };
template <> struct Cfg<4, float> { static constexpr int NE = NHMF_Q4F_NE, THREADS = NHMF_Q4F_THREADS; };
struct df64;
template <int P> struct Cfg<P, df64> : Cfg<P, double> {};
template <> struct Cfg<4, df64> { static constexpr int NE = 4, THREADS = 256; };
// Launch shape per strategy: Algorithm 2's point code (120 registers) keeps 256 threads at Q4
// so that two blocks fit an SM.
template <int P, typename T, int STRAT> struct LaunchCfg : Cfg<P, T> {};
template <> struct LaunchCfg<4, double, NHMF_SPATIAL> { static constexpr int NE = 4, THREADS = 256; };
#ifndef NHMF_Q2D_OTF_NE
#define NHMF_Q2D_OTF_NE NHMF_Q2D_NE
#define NHMF_Q2D_OTF_THREADS NHMF_Q2D_THREADS
#endif
template <> struct LaunchCfg<2, double, NHMF_ON_THE_FLY> {
  static constexpr int NE = NHMF_Q2D_OTF_NE, THREADS = NHMF_Q2D_OTF_THREADS;
};

// Coefficients of one n x n operator in even-odd form (odd n <= 5): S, A ((h+1) x h each) and C
// (h+1), h = n / 2.
constexpr int kEoSlots = 16;

// Kernel arguments (by value; lives in the constant bank).
struct OpArgs {
  int N, M, bc, model;
  long long M3, nq;
  double h, mu, lam;
  Colour col;
  double B[kMaxN * kMaxN], Dc[kMaxN * kMaxN], D[kMaxN * kMaxN], w[kMaxN];
  // Tables of the tangent apply, which carry the quadrature weight, mu and h so that its
  // point code returns dP / mu unweighted:
  //   BW[q][i] = B[q][i] w_q,  DcW[m][r] = Dc[m][r] w_m / w_r mu h,  Dch = Dc / h,
  //   eo[0..3]: even-odd coefficients of B, Dc, BW^T and DcW^T (odd n, see eo_line),
  //   r2mu = 2 lambda / mu.
  double BW[kMaxN * kMaxN], DcW[kMaxN * kMaxN], Dch[kMaxN * kMaxN];
  double eo[4][kEoSlots];
  double r2mu;
  int reg32;  // FP32 point cache in the register kernel's [10][n^3][E] layout (see kRegMaxP)
  float BWf[kMaxN * kMaxN], DcWf[kMaxN * kMaxN], Dchf[kMaxN * kMaxN], eof[4][kEoSlots];  // FP32 copies
  float Bf[kMaxN * kMaxN], Dcf[kMaxN * kMaxN], wf[kMaxN];  // FP32 copies (register kernels)
  const double* u64;
  const float* u32;
  const void* du;
  void* v;
  const void* cache;
  double* cache64_out;
  float* cache32_out;
  float2* cachedf_out;
  double* cachesp_out;
  const double* cachesp_in;
  const double* factor;  // per-element material factor (natural element order) or null
  unsigned* status;
  float* vloc;           // element-local FP32 results [3][n^3][E] (element-local apply) or null
};

// ------------------------------------------------------------------ memory helpers (PTX)
// L2 eviction-priority policies (createpolicy) and loads/stores that carry them: the applies
// stream their point caches with evict_first, so that the vectors they reuse stay in L2 (the
// FP64 colour launches re-read du and v eight times), and the FP32 apply writes its
// element-local results with evict_last, so that they are still in L2 when the gather reads them.
#ifndef NHMF_L2HINT
#define NHMF_L2HINT 1
#endif
__device__ __forceinline__ unsigned long long l2_evict_first() {
  unsigned long long p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ unsigned long long l2_evict_last() {
  unsigned long long p;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ float ld_policy(const float* a, unsigned long long pol) {
#if NHMF_L2HINT
  float v;
  asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(a), "l"(pol));
  return v;
#else
  return __ldg(a);
#endif
}
__device__ __forceinline__ double ld_policy(const double* a, unsigned long long pol) {
#if NHMF_L2HINT
  double v;
  asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(a), "l"(pol));
  return v;
#else
  return __ldg(a);
#endif
}
__device__ __forceinline__ void st_policy(float* a, float v, unsigned long long pol) {
#if NHMF_L2HINT
  asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(a), "f"(v), "l"(pol) : "memory");
#else
  *a = v;
#endif
}
__device__ __forceinline__ bool is_constrained(int bc, int c, int gi, int gk, int M) {
  if (bc == NHMF_BC_CLAMP_X0) return gi == 0;
  if (bc == NHMF_BC_COMPRESSION) return gk == 0 || (c == 2 && gk == M - 1);
  return false;
}

// Global node of work item t (element t / n^3 of this block, local point/node t % n^3).
template <int P>
__device__ __forceinline__ void item_node(const OpArgs& a, long long e_in_colour, int q, int& gi,
                                          int& gj, int& gk) {
  constexpr int n = P + 1;
  const Colour& c = a.col;
  const int ix = int(e_in_colour % c.nx);
  const int iy = int((e_in_colour / c.nx) % c.ny);
  const int iz = int(e_in_colour / ((long long)c.nx * c.ny));
  gi = P * (c.cx + c.stride * ix) + q % n;
  gj = P * (c.cy + c.stride * iy) + (q / n) % n;
  gk = P * (c.cz + c.stride * iz) + q / (n * n);
}

// Natural index ex + N (ey + N ez) of element e_in_colour of the launch's colour class.
__device__ __forceinline__ long long elem_natural(const OpArgs& a, long long e_in_colour) {
  const Colour& c = a.col;
  const long long ix = e_in_colour % c.nx, iy = (e_in_colour / c.nx) % c.ny, iz = e_in_colour / ((long long)c.nx * c.ny);
  const long long ex = c.cx + c.stride * ix, ey = c.cy + c.stride * iy, ez = c.cz + c.stride * iz;
  return ex + (long long)a.N * (ey + (long long)a.N * ez);
}

// Material factor of element e_in_colour of the launch's colour class (1 if homogeneous).
__device__ __forceinline__ double elem_factor(const OpArgs& a, long long e_in_colour) {
  if (!a.factor) return 1.0;
  const Colour& c = a.col;
  const long long ix = e_in_colour % c.nx, iy = (e_in_colour / c.nx) % c.ny, iz = e_in_colour / ((long long)c.nx * c.ny);
  const long long ex = c.cx + c.stride * ix, ey = c.cy + c.stride * iy, ez = c.cz + c.stride * iz;
  return a.factor[ex + (long long)a.N * (ey + (long long)a.N * ez)];
}

// One 1D pass along direction DIR over NC arrays of NI items:
//   out[c][t] (+)= sum_m Mat(r, m) in[c][t with coordinate r along DIR replaced by m]
// with Mat(r, m) = mat[r][m] (TR = false) or mat[m][r] (TR = true).
// Items t >= nitems (those of absent elements, which come last) are skipped.
template <int n, int NI, int NC, int DIR, bool TR, bool ACC, typename T>
__device__ __forceinline__ void sf_pass(const T* __restrict__ mat, const T* in, T* out, int nitems = NI) {
  constexpr int s = DIR == 0 ? 1 : (DIR == 1 ? n : n * n);
  for (int t = threadIdx.x; t < nitems; t += blockDim.x) {
    const int r = (t / s) % n;
    const int base = t - r * s;
    T acc[NC];
    {
      const T c0 = TR ? mat[r] : mat[r * n];
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[c] = c0 * in[c * NI + base];
    }
#pragma unroll
    for (int m = 1; m < n; ++m) {
      const T cm = TR ? mat[m * n + r] : mat[r * n + m];
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[c] = fma(cm, in[c * NI + base + m * s], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      if (ACC)
        out[c * NI + t] += acc[c];
      else
        out[c * NI + t] = acc[c];
    }
  }
}

// One line x[0..n-1] through a centro-symmetric operator (ANTI = false: M[n-1-r][n-1-m] =
// M[r][m], as B and B^T w have) or an anti-centro-symmetric one (ANTI = true: = -M[r][m], as the
// collocation derivative has), odd n, in even-odd form (h = n / 2, m < h, r < h):
//   e_m = x_m + x_{n-1-m},  o_m = x_m - x_{n-1-m},
//   E_r = C_r x_h + sum_m S_rm e_m,  O_r = sum_m A_rm o_m,
//   y_r = E_r + O_r,  y_{n-1-r} = +-(E_r - O_r),  y_h = E_h (symmetric) or O_h (anti),
// with S_rm = (M_rm + M_r,n-1-m) / 2, A_rm = (M_rm - M_r,n-1-m) / 2, C_r = M_rh.  n = 3 takes 8
// (symmetric) or 7 (anti) operations per line instead of 9; n = 5 takes 21 or 20 instead of 25.
// FORM uses that the middle Gauss point is the middle GLL node (x = 1/2) for odd n:
//   kEoCentreRow:  the centre row of M is e_h (M = B): y_h = x_h, 2 (n = 3) or 3 (n = 5) fewer;
//   kEoCentreCol:  the centre column of M vanishes off the centre (M = B^T w): C_r = 0 for r < h.
enum { kEoGeneral = 0, kEoCentreRow = 1, kEoCentreCol = 2 };
template <int n, bool ANTI, int FORM, typename T>
__device__ __forceinline__ void eo_line(const T (&k)[kEoSlots], const T (&x)[n], T (&y)[n]) {
  constexpr int h = n / 2, A0 = (h + 1) * h, C0 = 2 * (h + 1) * h;
  T e[h], o[h];
#pragma unroll
  for (int m = 0; m < h; ++m) {
    e[m] = x[m] + x[n - 1 - m];
    o[m] = x[m] - x[n - 1 - m];
  }
#pragma unroll
  for (int r = 0; r < h; ++r) {
    T E;
    if constexpr (FORM == kEoCentreCol) {
      E = k[r * h] * e[0];
#pragma unroll
      for (int m = 1; m < h; ++m) E = fma(k[r * h + m], e[m], E);
    } else {
      E = k[C0 + r] * x[h];
#pragma unroll
      for (int m = 0; m < h; ++m) E = fma(k[r * h + m], e[m], E);
    }
    T yp = E, ym = ANTI ? -E : E;
#pragma unroll
    for (int m = 0; m < h; ++m) {
      yp = fma(k[A0 + r * h + m], o[m], yp);
      ym = fma(ANTI ? k[A0 + r * h + m] : -k[A0 + r * h + m], o[m], ym);
    }
    y[r] = yp;
    y[n - 1 - r] = ym;
  }
  if constexpr (ANTI) {
    T c = k[A0 + h * h] * o[0];
#pragma unroll
    for (int m = 1; m < h; ++m) c = fma(k[A0 + h * h + m], o[m], c);
    y[h] = c;
  } else if constexpr (FORM == kEoCentreRow) {
    y[h] = x[h];
  } else {
    T c = k[C0 + h] * x[h];
#pragma unroll
    for (int m = 0; m < h; ++m) c = fma(k[h * h + m], e[m], c);
    y[h] = c;
  }
}

// The tasks of a pass over 3 fields with one thread per (field, line): this thread's field,
// line and line start for each direction, computed once per kernel instead of in every pass.
struct NoLineMap {};
template <int n, int NI, int TH>
struct LineMap {
  static constexpr int NL = NI / n, ITER = (3 * NL + TH - 1) / TH;
  int c[ITER], L[ITER], base[3][ITER];
  __device__ __forceinline__ LineMap() {
#pragma unroll
    for (int it = 0; it < ITER; ++it) {
      const int task = threadIdx.x + it * TH;
      c[it] = task / NL;  // >= 3: no task
      L[it] = task - c[it] * NL;
      base[0][it] = L[it] * n;
      base[1][it] = (L[it] % n) + (L[it] / n) * n * n;
      base[2][it] = (L[it] % (n * n)) + (L[it] / (n * n)) * n * n * n;
    }
  }
};

// One 1D pass along DIR over NC fields with one thread per (field, line of n items), odd n:
//   out[(c OS + OO)][line] (+)= M in[(c IS + IO)][line]  (+= when ACC)
// where M is given by its even-odd coefficients `coef` (see eo_line).
// TH is the block size; the task loop is unrolled so that independent lines interleave (not for
// double-float, whose unrolled lines would cost an SM its second block).
// Lines of absent elements (line index >= nlines; they come last) are skipped.
template <int n, int NI, int NC, int DIR, bool ANTI, int FORM, int TH, int OS = 1, int OO = 0, int IS = 1,
          int IO = 0, bool ACC = false, typename T, typename MAP = NoLineMap>
__device__ __forceinline__ void eo_pass(const T* __restrict__ coef, const T* __restrict__ in,
                                        T* __restrict__ out, int nlines = NI / n, const MAP& map = MAP()) {
  constexpr int s = DIR == 0 ? 1 : (DIR == 1 ? n : n * n), NL = NI / n, ITER = (NC * NL + TH - 1) / TH;
  constexpr int UNROLL = std::is_same<T, df64>::value ? 1 : ITER;
  T k[kEoSlots];
#pragma unroll
  for (int i = 0; i < kEoSlots; ++i) k[i] = coef[i];
#pragma unroll UNROLL
  for (int it = 0; it < ITER; ++it) {
    int c, L, base;
    if constexpr (std::is_same<MAP, NoLineMap>::value) {
      const int task = threadIdx.x + it * TH;
      if (ITER * TH != NC * NL && task >= NC * NL) break;
      c = task / NL;
      L = task - c * NL;
      base = DIR == 0 ? L * n
                      : (DIR == 1 ? (L % n) + (L / n) * n * n : (L % (n * n)) + (L / (n * n)) * n * n * n);
    } else {
      static_assert(NC == 3 && MAP::ITER == ITER && MAP::NL == NL, "a line map covers passes over 3 fields");
      c = map.c[it];
      if (ITER * TH != NC * NL && c >= NC) break;
      L = map.L[it];
      base = map.base[DIR][it];
    }
    if (L >= nlines) continue;
    T x[n], y[n];
#pragma unroll
    for (int m = 0; m < n; ++m) x[m] = in[(c * IS + IO) * NI + base + m * s];
    eo_line<n, ANTI, FORM>(k, x, y);
#pragma unroll
    for (int m = 0; m < n; ++m) {
      if (ACC)
        out[(c * OS + OO) * NI + base + m * s] += y[m];
      else
        out[(c * OS + OO) * NI + base + m * s] = y[m];
    }
  }
}

// Reference-cell gradient of NC fields at item t from their point values (collocation).
//   g[c][d] = sum_m Dc[r_d][m] val[c][t with coordinate d replaced by m]
template <int n, int NI, typename T>
__device__ __forceinline__ void colloc_grad(const T* __restrict__ Dc, const T* val, int t, T g[9]) {
  const int rx = t % n, ry = (t / n) % n, rz = (t / (n * n)) % n;
  const int bx = t - rx, by = t - ry * n, bz = t - rz * n * n;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const T* vc = val + c * NI;
    T gx = Dc[rx * n] * vc[bx];
    T gy = Dc[ry * n] * vc[by];
    T gz = Dc[rz * n] * vc[bz];
#pragma unroll
    for (int m = 1; m < n; ++m) {
      gx = fma(Dc[rx * n + m], vc[bx + m], gx);
      gy = fma(Dc[ry * n + m], vc[by + m * n], gy);
      gz = fma(Dc[rz * n + m], vc[bz + m * n * n], gz);
    }
    g[c * 3 + 0] = gx;
    g[c * 3 + 1] = gy;
    g[c * 3 + 2] = gz;
  }
}

// Combined transposed collocation pass: y[c][t] = sum_d sum_m Dc[m][r_d] G[3c+d][t_d(m)].
template <int n, int NI, typename T>
__device__ __forceinline__ void colloc_grad_T(const T* __restrict__ Dc, const T* G, T* y, int nitems = NI) {
  for (int t = threadIdx.x; t < nitems; t += blockDim.x) {
    const int rx = t % n, ry = (t / n) % n, rz = (t / (n * n)) % n;
    const int bx = t - rx, by = t - ry * n, bz = t - rz * n * n;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T* gx = G + (3 * c + 0) * NI;
      const T* gy = G + (3 * c + 1) * NI;
      const T* gz = G + (3 * c + 2) * NI;
      T acc = Dc[rx] * gx[bx];
      acc = fma(Dc[ry], gy[by], acc);
      acc = fma(Dc[rz], gz[bz], acc);
#pragma unroll
      for (int m = 1; m < n; ++m) {
        acc = fma(Dc[m * n + rx], gx[bx + m], acc);
        acc = fma(Dc[m * n + ry], gy[by + m * n], acc);
        acc = fma(Dc[m * n + rz], gz[bz + m * n * n], acc);
      }
      y[c * NI + t] = acc;
    }
  }
}

// ------------------------------------------------------------------ point code
// Kinematics at a point from the physical displacement gradient H (row-major H[3c+d]):
// J - 1 from the invariants of H (no cancellation near J = 1),
//   J - 1 = tr H + ((tr H)^2 - tr(H^2))/2 + det H,
// F^-1 = cof(F)^T / J, ln J = log1p(J - 1).  Returns J - 1.
template <typename T>
__device__ __forceinline__ T kinematics(const T H[9], T Fi[9], T& lnJ) {
  const T trH = H[0] + H[4] + H[8];
  const T trH2 = H[0] * H[0] + H[4] * H[4] + H[8] * H[8] +
                 T(2) * (H[1] * H[3] + H[2] * H[6] + H[5] * H[7]);
  const T detH = H[0] * (H[4] * H[8] - H[5] * H[7]) - H[1] * (H[3] * H[8] - H[5] * H[6]) +
                 H[2] * (H[3] * H[7] - H[4] * H[6]);
  const T Jm1 = trH + T(0.5) * (trH * trH - trH2) + detH;
  const T F0 = T(1) + H[0], F4 = T(1) + H[4], F8 = T(1) + H[8];
  const T F1 = H[1], F2 = H[2], F3 = H[3], F5 = H[5], F6 = H[6], F7 = H[7];
  const T invJ = T(1) / (T(1) + Jm1);
  Fi[0] = (F4 * F8 - F5 * F7) * invJ;
  Fi[1] = (F2 * F7 - F1 * F8) * invJ;
  Fi[2] = (F1 * F5 - F2 * F4) * invJ;
  Fi[3] = (F5 * F6 - F3 * F8) * invJ;
  Fi[4] = (F0 * F8 - F2 * F6) * invJ;
  Fi[5] = (F2 * F3 - F0 * F5) * invJ;
  Fi[6] = (F3 * F7 - F4 * F6) * invJ;
  Fi[7] = (F1 * F6 - F0 * F7) * invJ;
  Fi[8] = (F0 * F4 - F1 * F3) * invJ;
  lnJ = log1p(Jm1);
  return Jm1;
}

// Linearised first Piola stress at a point, scaled by s (Eq. LG: G = L : Grad du):
//   dP = mu dH + (mu - 2 lambda ln J) F^-T dH^T F^-T + 2 lambda tr(F^-1 dH) F^-T
// with K = F^-1 dH and Q = K F^-1 (so F^-T dH^T F^-T = Q^T).  Written into g[3i+J].
template <typename T>
__device__ __forceinline__ void linearised_stress(const T Fi[9], T lnJ, const T dH[9], T mu,
                                                  T lam, T s, T g[9]) {
  T K[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      K[3 * i + j] = fma(Fi[3 * i + 0], dH[j], fma(Fi[3 * i + 1], dH[3 + j], Fi[3 * i + 2] * dH[6 + j]));
  const T trK = K[0] + K[4] + K[8];
  const T smu = s * mu;
  const T sc1 = s * (mu - T(2) * lam * lnJ);
  const T sc2 = s * (T(2) * lam * trK);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      // Q[j][i] = sum_c K[j][c] Fi[c][i]
      const T Qji = fma(K[3 * j + 0], Fi[i], fma(K[3 * j + 1], Fi[3 + i], K[3 * j + 2] * Fi[6 + i]));
      g[3 * i + j] = fma(smu, dH[3 * i + j], fma(sc1, Qji, sc2 * Fi[3 * j + i]));
    }
}

// The same linearised stress divided by mu and without the point weight (the tangent apply
// carries w_q, mu and h on its transposed tables), r = 2 lambda / mu:
//   g = dH + (1 - r ln J) Q^T + r tr(K) F^-T.
template <typename T>
__device__ __forceinline__ void linearised_stress_unit(const T Fi[9], T lnJ, const T dH[9], T r, T g[9]) {
  T K[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      K[3 * i + j] = fma(Fi[3 * i + 0], dH[j], fma(Fi[3 * i + 1], dH[3 + j], Fi[3 * i + 2] * dH[6 + j]));
  const T c1 = fma(-r, lnJ, T(1));
  const T c2 = r * (K[0] + K[4] + K[8]);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const T Qji = fma(K[3 * j + 0], Fi[i], fma(K[3 * j + 1], Fi[3 + i], K[3 * j + 2] * Fi[6 + i]));
      g[3 * i + j] = fma(c1, Qji, fma(c2, Fi[3 * j + i], dH[3 * i + j]));
    }
}

// Split neo-Hookean model (Eq. hypcomplex), with a = J^(-2/3), I1 = F : F:
//   P  = mu a (F - I1/3 F^-T) + kappa/2 (J^2 - 1) F^-T
//   dP = mu a dH - 2/3 mu a tr(F^-1 dH) F
//        + (2/9 mu a I1 tr(F^-1 dH) - 2/3 mu a F:dH + kappa J^2 tr(F^-1 dH)) F^-T
//        + (mu a I1/3 - kappa/2 (J^2 - 1)) F^-T dH^T F^-T
template <typename T>
__device__ __forceinline__ void split_stress_dP(const T F[9], const T Fi[9], T lnJ, T Jm1, const T dH[9], T mu,
                                                T kappa, T s, T g[9]) {
  const T a = exp(T(-2) / T(3) * lnJ);
  const T J = T(1) + Jm1;
  const T J2 = J * J;
  T I1 = T(0), FdH = T(0);
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    I1 = fma(F[k], F[k], I1);
    FdH = fma(F[k], dH[k], FdH);
  }
  T K[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      K[3 * i + j] = fma(Fi[3 * i + 0], dH[j], fma(Fi[3 * i + 1], dH[3 + j], Fi[3 * i + 2] * dH[6 + j]));
  const T trK = K[0] + K[4] + K[8];
  const T mua = mu * a;
  const T c1 = s * mua;
  const T cF = -s * T(2) / T(3) * mua * trK;
  const T c3 = s * (T(2) / T(9) * mua * I1 * trK - T(2) / T(3) * mua * FdH + kappa * J2 * trK);
  const T c4 = s * (mua * I1 / T(3) - kappa / T(2) * (J2 - T(1)));
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const T Qji = fma(K[3 * j + 0], Fi[i], fma(K[3 * j + 1], Fi[3 + i], K[3 * j + 2] * Fi[6 + i]));
      g[3 * i + j] = fma(c1, dH[3 * i + j], fma(cF, F[3 * i + j], fma(c3, Fi[3 * j + i], c4 * Qji)));
    }
}

// P of the selected model
template <typename T>
__device__ __forceinline__ void model_piola(int model, const T F[9], const T Fi[9], T lnJ, T Jm1, T mu, T lam, T P[9]) {
  if (model == NHMF_MODEL_SPLIT) {
    const T a = exp(T(-2) / T(3) * lnJ);
    const T J = T(1) + Jm1;
    T I1 = T(0);
#pragma unroll
    for (int k = 0; k < 9; ++k) I1 = fma(F[k], F[k], I1);
    const T cT = -mu * a * I1 / T(3) + lam / T(2) * (J * J - T(1));
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) P[3 * i + j] = fma(mu * a, F[3 * i + j], cT * Fi[3 * j + i]);
  } else {
    const T c2 = T(2) * lam * lnJ - mu;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) P[3 * i + j] = fma(mu, F[3 * i + j], c2 * Fi[3 * j + i]);
  }
}

// dP[dH] of the selected model, scaled by s (F = I + H needed by the split model only)
template <typename T>
__device__ __forceinline__ void model_dP(int model, const T F[9], const T Fi[9], T lnJ, T Jm1, const T dH[9], T mu,
                                         T lam, T s, T g[9]) {
  if (model == NHMF_MODEL_SPLIT)
    split_stress_dP(F, Fi, lnJ, Jm1, dH, mu, lam, s, g);
  else
    linearised_stress(Fi, lnJ, dH, mu, lam, s, g);
}

// Voigt index of the pair (i, j): 11, 22, 33, 23, 13, 12 -> 0..5.
__host__ __device__ constexpr int voigt(int i, int j) {
  return i == j ? i : (i + j == 3 ? 3 : (i + j == 2 ? 4 : 5));
}
// Index of (I, K), I <= K, in the row-major upper triangle of a 6x6 matrix.
__host__ __device__ constexpr int tri6(int I, int K) { return I * 6 - I * (I - 1) / 2 + (K - I); }

// Algorithm 2 point code (current configuration, Eq. DF:cur), scaled by s:
//   g = dH F^-1 (spatial gradient), e_hat = (g00, g11, g22, g12+g21, g02+g20, g01+g10),
//   sig_I = sum_K Jc[I][K] e_hat_K (J c : sym(g)), X = sig + g tau, G = s X F^-T.
template <typename T>
__device__ __forceinline__ void spatial_stress(const T Jc[21], const T tau[6], const T Fi[9], const T dH[9], T s,
                                               T out[9]) {
  T gs[9];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int l = 0; l < 3; ++l)
      gs[3 * k + l] = fma(dH[3 * k + 0], Fi[l], fma(dH[3 * k + 1], Fi[3 + l], dH[3 * k + 2] * Fi[6 + l]));
  const T eh[6] = {gs[0], gs[4], gs[8], gs[5] + gs[7], gs[2] + gs[6], gs[1] + gs[3]};
  T sv[6];
#pragma unroll
  for (int I = 0; I < 6; ++I) {
    T acc = T(0);
#pragma unroll
    for (int K = 0; K < 6; ++K) acc = fma(Jc[I <= K ? tri6(I, K) : tri6(K, I)], eh[K], acc);
    sv[I] = acc;
  }
  T X[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      X[3 * i + j] = fma(gs[3 * i + 0], tau[voigt(0, j)],
                         fma(gs[3 * i + 1], tau[voigt(1, j)], fma(gs[3 * i + 2], tau[voigt(2, j)], sv[voigt(i, j)])));
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int J = 0; J < 3; ++J)
      out[3 * i + J] = s * fma(X[3 * i + 0], Fi[3 * J + 0], fma(X[3 * i + 1], Fi[3 * J + 1], X[3 * i + 2] * Fi[3 * J + 2]));
}

}  // namespace nhmf
