// Matrix-free operators of compressible neo-Hookean elasticity on the GPU:
//   k_apply         tangent application, on the fly (Algorithm 1) or from the point cache
//   k_apply_reg     FP32 tangent application, one element per thread in registers (p <= 2)
//   k_gather_local  FP32: sums the element-local results of the apply at the nodes
//   k_cache         point cache {F^-1, ln J} at the linearisation point (partial assembly, Section 3.2)
//   k_residual      residual R(u) (Eq. F)
//   k_diagonal      operator diagonal (Section 2.3)
// FP64 and double-float: each block processes NE elements of one colour class; elements of a
// class share no node, so the read-modify-write scatter of a launch is race-free and
// deterministic, and the eight classes run as eight launches in a fixed order.  FP32: one
// launch over all elements writes element-local results, and the gather adds each node's
// contributions in a fixed order (also deterministic, no atomics).
#include <algorithm>
#include <type_traits>

#include "df64.cuh"
#include "sumfact.cuh"

namespace nhmf {
namespace {

// Table slots ahead of the per-item arrays: B, Dc, D, n^3 weights and NE factors, or in the
// apply B, Dc, BW, DcW, Dch, 3 even-odd sets and NE factors (whichever is larger).
constexpr int kTabSlots = 3 * kMaxN * kMaxN + 128 + 32;
static_assert(5 * kMaxN * kMaxN + 4 * kEoSlots + 32 <= kTabSlots, "apply tables exceed the table slots");

template <int P, typename T>
__device__ __forceinline__ void load_tables(const OpArgs& a, T* sB, T* sDc, T* sD, T* sW, double wscale) {
  constexpr int n = P + 1;
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
    sB[i] = T(a.B[i]);
    sDc[i] = T(a.Dc[i]);
    sD[i] = T(a.D[i]);
  }
  for (int q = threadIdx.x; q < n * n * n; q += blockDim.x)
    sW[q] = T(a.w[q % n] * a.w[(q / n) % n] * a.w[q / (n * n)] * wscale);
}

// The apply's tables: B and Dc (forward), BW and DcW (transposed, carrying w, mu, h), Dch and
// the even-odd coefficient sets, laid out as in k_apply.
template <int P, typename T>
__device__ __forceinline__ void load_apply_tables(const OpArgs& a, T* tab) {
  constexpr int n = P + 1, S = kMaxN * kMaxN;
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
    tab[i] = T(a.B[i]);
    tab[S + i] = T(a.Dc[i]);
    tab[2 * S + i] = T(a.BW[i]);
    tab[3 * S + i] = T(a.DcW[i]);
    tab[4 * S + i] = T(a.Dch[i]);
  }
  for (int i = threadIdx.x; i < 4 * kEoSlots; i += blockDim.x)
    tab[5 * S + i] = T(a.eo[i / kEoSlots][i % kEoSlots]);
}

// Gather three components of a global vector into dst[c][t] for the block's elements,
// optionally zeroing constrained DoFs and scaling by a per-element factor fac[e]; items of
// absent elements are zero.
template <int P, int NI, typename TS, typename T>
__device__ __forceinline__ void gather(const OpArgs& a, const TS* __restrict__ src, long long e0,
                                       int nvalid, bool mask, T* dst, const T* fac = nullptr) {
  constexpr int n3 = (P + 1) * (P + 1) * (P + 1);
  for (int t = threadIdx.x; t < NI; t += blockDim.x) {
    const int e = t / n3;
    if (e < nvalid) {
      int gi, gj, gk;
      item_node<P>(a, e0 + e, t % n3, gi, gj, gk);
      const long long node = gi + (long long)a.M * (gj + (long long)a.M * gk);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        T val = T(src[c * a.M3 + node]);
        if (mask && is_constrained(a.bc, c, gi, gk, a.M)) val = T(0);
        dst[c * NI + t] = fac ? val * fac[e] : val;
      }
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c) dst[c * NI + t] = T(0);
    }
  }
}

template <typename T> struct Store { using type = T; };
template <> struct Store<df64> { using type = double; };
__device__ __forceinline__ double to_store(double x) { return x; }
__device__ __forceinline__ float to_store(float x) { return x; }
__device__ __forceinline__ double to_store(df64 x) { return to_double(x); }

template <int P, int NI, typename T>
__device__ __forceinline__ void scatter_add(const OpArgs& a, const T* src, long long e0, int nvalid,
                                            typename Store<T>::type* __restrict__ out) {
  constexpr int n3 = (P + 1) * (P + 1) * (P + 1);
  for (int t = threadIdx.x; t < NI; t += blockDim.x) {
    const int e = t / n3;
    if (e >= nvalid) continue;
    int gi, gj, gk;
    item_node<P>(a, e0 + e, t % n3, gi, gj, gk);
    const long long node = gi + (long long)a.M * (gj + (long long)a.M * gk);
#pragma unroll
    for (int c = 0; c < 3; ++c) out[c * a.M3 + node] += to_store(src[c * NI + t]);
  }
}

// Element-local results of the block's elements (launched on the class of all elements, so the
// slot is the natural element index) into the element tiles of vloc, [E/32][3][n^3][32]:
// consecutive threads write consecutive elements of one (c, q) row.
template <int P, int NE>
__device__ __forceinline__ void store_local(const OpArgs& a, const float* src, long long e0, int nvalid) {
  constexpr int n3 = (P + 1) * (P + 1) * (P + 1), NI = NE * n3;
  const long long slot = a.col.slot0 + e0;
  const unsigned long long keep_pol = l2_evict_last();
  for (int t = threadIdx.x; t < 3 * n3 * NE; t += blockDim.x) {
    const int e = t % NE, cq = t / NE;
    const long long el = slot + e;
    if (e < nvalid)
      st_policy(a.vloc + ((el / kTile) * 3 * n3 + cq) * kTile + el % kTile, src[(cq / n3) * NI + e * n3 + cq % n3],
                keep_pol);
  }
}

// Forward interpolation of three components to the points: in -> out (tmp is clobbered).
template <int n, int NI, typename T>
__device__ __forceinline__ void to_points(const T* sB, T* in, T* tmp, T* out, int nitems) {
  sf_pass<n, NI, 3, 0, false, false>(sB, in, tmp, nitems);
  __syncthreads();
  sf_pass<n, NI, 3, 1, false, false>(sB, tmp, in, nitems);
  __syncthreads();
  sf_pass<n, NI, 3, 2, false, false>(sB, in, out, nitems);
  __syncthreads();
}

// Transposed integration of the nine point fluxes G[3c+d] to nodal values in `out`
// (`tmp` clobbered; G's first three slots are reused).
template <int n, int NI, typename T>
__device__ __forceinline__ void from_points(const T* sB, const T* sDc, T* G, T* tmp, T* out, int nitems) {
  colloc_grad_T<n, NI>(sDc, G, tmp, nitems);
  __syncthreads();
  sf_pass<n, NI, 3, 0, true, false>(sB, tmp, G, nitems);
  __syncthreads();
  sf_pass<n, NI, 3, 1, true, false>(sB, G, tmp, nitems);
  __syncthreads();
  sf_pass<n, NI, 3, 2, true, false>(sB, tmp, out, nitems);
  __syncthreads();
}

// ------------------------------------------------------------------ tangent application
// The quadrature weight, mu and h ride on the transposed tables (BW, DcW) and the element's
// material factor on the gathered du (the operator is linear in du), so the point code returns
// dP / mu without any scaling.  For odd n (Q2, Q4) every non-accumulating pass (forward B,
// forward collocation derivative, transposed B) runs one thread per line in even-odd form, and
// the gradient of du reaches the point code through shared memory.
#ifndef NHMF_EO_GRADT
#define NHMF_EO_GRADT 1
#endif
#ifndef NHMF_LINEMAP
#define NHMF_LINEMAP 1
#endif
template <int P, typename T, int STRAT, int MODEL>
__global__ void __launch_bounds__(LaunchCfg<P, T, STRAT>::THREADS) k_apply(const OpArgs a) {
  constexpr int n = P + 1, n3 = n * n * n, NE = LaunchCfg<P, T, STRAT>::NE, NI = NE * n3;
  constexpr int S = kMaxN * kMaxN, TH = LaunchCfg<P, T, STRAT>::THREADS;
  constexpr bool EO = n % 2 == 1;
  static_assert(5 * S + 4 * kEoSlots + NE <= kTabSlots, "the factor table exceeds the table slots");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tab = reinterpret_cast<T*>(smem_raw);
  const T* sB = tab;
  const T* sDc = tab + S;
  const T* sBW = tab + 2 * S;
  const T* sDcW = tab + 3 * S;
  const T* sDch = tab + 4 * S;
  const T* kB = tab + 5 * S;                    // even-odd coefficients of B, Dc, BW^T, DcW^T
  const T* kDc = kB + kEoSlots;
  const T* kBW = kDc + kEoSlots;
  const T* kDcWT = kBW + kEoSlots;              // even-odd coefficients of DcW^T
  T* sF = tab + 5 * S + 4 * kEoSlots;          // [NE] material factors of the block's elements
  T* U = tab + kTabSlots;                       // [3][NI] ubar at the points (on the fly)
  T* Vq = U + (STRAT == NHMF_ON_THE_FLY ? 3 * NI : 0);  // [3][NI] du at the points
  T* G = Vq + 3 * NI;                           // [9][NI] gradients, then fluxes; G[0..2] gathers

  // FP32: the passes' task decomposition computed once (the FP32 kernel is issue bound)
  using LM = typename std::conditional<std::is_same<T, float>::value && NHMF_LINEMAP && EO, LineMap<n, NI, TH>,
                                       NoLineMap>::type;
  const LM lm{};
  load_apply_tables<P>(a, tab);
  const long long e0 = (long long)blockIdx.x * NE;
  const int nvalid = (int)min((long long)NE, (long long)a.col.count - e0);
  const int nitems = nvalid * n3, nlines = nvalid * n * n;  // items / lines of present elements
  for (int e = threadIdx.x; e < NE; e += blockDim.x) sF[e] = T(elem_factor(a, e0 + min(e, nvalid - 1)));
  __syncthreads();

  if constexpr (STRAT == NHMF_ON_THE_FLY) {
    if (sizeof(T) == 8)
      gather<P, NI>(a, a.u64, e0, nvalid, false, G);
    else
      gather<P, NI>(a, a.u32, e0, nvalid, false, G);
    __syncthreads();
    if constexpr (EO) {
      eo_pass<n, NI, 3, 0, false, kEoCentreRow, TH>(kB, G, Vq, nlines, lm);
      __syncthreads();
      eo_pass<n, NI, 3, 1, false, kEoCentreRow, TH>(kB, Vq, G, nlines, lm);
      __syncthreads();
      eo_pass<n, NI, 3, 2, false, kEoCentreRow, TH>(kB, G, U, nlines, lm);
      __syncthreads();
    } else {
      to_points<n, NI>(sB, G, Vq, U, nitems);
    }
  }
  gather<P, NI>(a, static_cast<const typename Store<T>::type*>(a.du), e0, nvalid, true, G,
                a.factor ? (const T*)sF : nullptr);
  __syncthreads();
  if constexpr (EO) {
    eo_pass<n, NI, 3, 0, false, kEoCentreRow, TH>(kB, G, Vq, nlines, lm);
    __syncthreads();
    eo_pass<n, NI, 3, 1, false, kEoCentreRow, TH>(kB, Vq, G, nlines, lm);
    __syncthreads();
    eo_pass<n, NI, 3, 2, false, kEoCentreRow, TH>(kB, G, Vq, nlines, lm);
    __syncthreads();
    // reference gradient of du: G[3c+d] = Dc along d of du[c]
    eo_pass<n, NI, 3, 0, true, kEoGeneral, TH, 3, 0>(kDc, Vq, G, nlines, lm);
    eo_pass<n, NI, 3, 1, true, kEoGeneral, TH, 3, 1>(kDc, Vq, G, nlines, lm);
    eo_pass<n, NI, 3, 2, true, kEoGeneral, TH, 3, 2>(kDc, Vq, G, nlines, lm);
    __syncthreads();
  } else {
    to_points<n, NI>(sB, G, Vq + 0, Vq, nitems);  // passes ping-pong via G: x G->Vq, y Vq->G, z G->Vq
  }

  const T inv_mu = T(1.0 / a.mu), r2 = T(a.r2mu);
  const typename Store<T>::type* cache = static_cast<const typename Store<T>::type*>(a.cache);
  const long long cbase = (a.col.slot0 + e0) * n3;
  bool bad = false;
  for (int t = threadIdx.x; t < nitems; t += blockDim.x) {
    T dH[9], g[9];
    if constexpr (EO) {
#pragma unroll
      for (int k = 0; k < 9; ++k) dH[k] = G[k * NI + t];
    } else {
      colloc_grad<n, NI>(sDc, Vq, t, dH);
    }
    if constexpr (STRAT == NHMF_SPATIAL) {
      // Algorithm 2: J c, tau and F^-1 from the 36-value cache
      T Jc[21], tau[6], Fs[9];
      if (t / n3 < nvalid) {
        const double* sp = a.cachesp_in;
#pragma unroll
        for (int k = 0; k < 21; ++k) Jc[k] = T(sp[k * a.nq + cbase + t]);
#pragma unroll
        for (int k = 0; k < 6; ++k) tau[k] = T(sp[(21 + k) * a.nq + cbase + t]);
#pragma unroll
        for (int k = 0; k < 9; ++k) Fs[k] = T(sp[(27 + k) * a.nq + cbase + t]);
      } else {
#pragma unroll
        for (int k = 0; k < 21; ++k) Jc[k] = T(0);
#pragma unroll
        for (int k = 0; k < 6; ++k) tau[k] = T(0);
#pragma unroll
        for (int k = 0; k < 9; ++k) Fs[k] = (k % 4 == 0) ? T(1) : T(0);
      }
      spatial_stress(Jc, tau, Fs, dH, inv_mu, g);
#pragma unroll
      for (int k = 0; k < 9; ++k) G[k * NI + t] = g[k];
      continue;
    }
    T Fi[9], lnJ, Jm1 = T(0), F[9];
    if constexpr (STRAT == NHMF_ON_THE_FLY) {
      T H[9];
      colloc_grad<n, NI>(sDch, U, t, H);  // physical gradient: Dch = Dc / h
      Jm1 = kinematics(H, Fi, lnJ);
      bad |= !(Jm1 > T(-1));
#pragma unroll
      for (int k = 0; k < 9; ++k) F[k] = (k % 4 == 0 ? T(1) : T(0)) + H[k];
    } else {
      if (t / n3 < nvalid) {
        if constexpr (std::is_same<T, df64>::value) {
          const float2* cdf = static_cast<const float2*>(a.cache);
#pragma unroll
          for (int k = 0; k < 9; ++k) {
            const float2 z = cdf[k * a.nq + cbase + t];
            Fi[k] = T(z.x, z.y);
          }
          const float2 z = cdf[9 * a.nq + cbase + t];
          lnJ = T(z.x, z.y);
        } else if (sizeof(typename Store<T>::type) == 8 || P > kRegMaxP || !a.reg32) {
          // the cache is read once per apply: evict it first, keep du and v in L2
          const unsigned long long pol = l2_evict_first();
#pragma unroll
          for (int k = 0; k < 9; ++k) Fi[k] = T(ld_policy(cache + k * a.nq + cbase + t, pol));
          lnJ = T(ld_policy(cache + 9 * a.nq + cbase + t, pol));
        } else {
          const long long slot = a.col.slot0 + e0 + t / n3, q = t % n3;
          const auto* tile = cache + (slot / kTile) * (10 * n3 * kTile) + slot % kTile;
#pragma unroll
          for (int k = 0; k < 9; ++k) Fi[k] = T(tile[(k * n3 + q) * kTile]);
          lnJ = T(tile[(9 * n3 + q) * kTile]);
        }
      } else {
#pragma unroll
        for (int k = 0; k < 9; ++k) Fi[k] = (k % 4 == 0) ? T(1) : T(0);
        lnJ = T(0);
      }
    }
    if constexpr (STRAT == NHMF_ON_THE_FLY && MODEL == NHMF_MODEL_SPLIT)
      split_stress_dP(F, Fi, lnJ, Jm1, dH, T(a.mu), T(a.lam), inv_mu, g);
    else
      linearised_stress_unit(Fi, lnJ, dH, r2, g);
#pragma unroll
    for (int k = 0; k < 9; ++k) G[k * NI + t] = g[k];
  }
  if (bad) atomicOr(a.status, kStatusNonPosJ);
  __syncthreads();
  if constexpr (EO) {
    if constexpr (std::is_same<T, float>::value && NHMF_EO_GRADT) {
      // FP32: the transposed derivative as three even-odd line passes, Vq[c] = sum_d DcW^T_d G[3c+d]
      eo_pass<n, NI, 3, 0, true, kEoGeneral, TH, 1, 0, 3, 0, false>(kDcWT, G, Vq, nlines, lm);
      __syncthreads();
      eo_pass<n, NI, 3, 1, true, kEoGeneral, TH, 1, 0, 3, 1, true>(kDcWT, G, Vq, nlines, lm);
      __syncthreads();
      eo_pass<n, NI, 3, 2, true, kEoGeneral, TH, 1, 0, 3, 2, true>(kDcWT, G, Vq, nlines, lm);
    } else {
      colloc_grad_T<n, NI>(sDcW, G, Vq, nitems);
    }
    __syncthreads();
    eo_pass<n, NI, 3, 0, false, kEoCentreCol, TH>(kBW, Vq, G, nlines, lm);
    __syncthreads();
    eo_pass<n, NI, 3, 1, false, kEoCentreCol, TH>(kBW, G, Vq, nlines, lm);
    __syncthreads();
    eo_pass<n, NI, 3, 2, false, kEoCentreCol, TH>(kBW, Vq, G + 3 * NI, nlines, lm);
    __syncthreads();
  } else {
    from_points<n, NI>(sBW, sDcW, G, Vq, G + 3 * NI, nitems);
  }
  if constexpr (std::is_same<T, float>::value) {
    if (a.vloc) {
      store_local<P, NE>(a, G + 3 * NI, e0, nvalid);
      return;
    }
  }
  scatter_add<P, NI>(a, G + 3 * NI, e0, nvalid, static_cast<typename Store<T>::type*>(a.v));
}

// ------------------------------------------------------------------ FP32 register kernel
// One thread per element: the element's three components (3 (p+1)^3 values), their values at
// the Gauss points and the transposed-derivative accumulators stay in registers; every 1D pass
// is fully unrolled, so its coefficients are compile-time-indexed kernel parameters (constant
// bank operands of the FMAs) and no shared memory is touched.  For p <= 2.  As in k_apply, w_q,
// mu and h ride on the transposed tables and the material factor on du.  The on-the-fly kernel
// runs its B and B^T passes in even-odd form at odd n; the cached kernel keeps the matrix form.
// Launched once over the class of all elements; each thread writes its element's results to
// its column of the element tile of vloc (a warp writes whole 128-byte rows) for
// k_gather_local, and reads the point cache from the same tiling.
#ifndef NHMF_REG_THREADS
#define NHMF_REG_THREADS 128
#endif
#ifndef NHMF_REG_MINB
#define NHMF_REG_MINB 1
#endif
constexpr int kRegThreads = NHMF_REG_THREADS;  // threads (= elements) per block

template <int P, int STRAT, int MODEL>
__global__ void __launch_bounds__(kRegThreads, NHMF_REG_MINB) k_apply_reg(const OpArgs a) {
  constexpr int n = P + 1, n3 = n * n * n;
  const long long ec = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (ec >= a.col.count) return;
  const Colour& col = a.col;
  const int ix = int(ec % col.nx), iy = int((ec / col.nx) % col.ny), iz = int(ec / ((long long)col.nx * col.ny));
  const int gi0 = P * (col.cx + col.stride * ix), gj0 = P * (col.cy + col.stride * iy),
            gk0 = P * (col.cz + col.stride * iz);
  const long long M = a.M;
  const long long slot = col.slot0 + ec;
  const float* __restrict__ du = static_cast<const float*>(a.du);
  // this element's column of its tile in the point cache and in vloc
  float* __restrict__ vloc = a.vloc + (slot / kTile) * (3 * n3 * kTile) + slot % kTile;
  const float* __restrict__ cache =
      static_cast<const float*>(a.cache) + (slot / kTile) * (10 * n3 * kTile) + slot % kTile;
  const unsigned long long stream_pol = l2_evict_first();  // the point cache is read once
  auto node = [&](int i, int j, int k) { return (gi0 + i) + M * ((gj0 + j) + M * (long long)(gk0 + k)); };
  auto idx = [](int i, int j, int k) { return i + n * (j + n * k); };

  // one 1D pass over the n^2 lines of direction DIR of f[c]: even-odd coefficients `eo` (odd
  // n) or the matrix Mat(r, m) = mat[r n + m] (TR = false) / mat[m n + r] (TR = true)
  auto pass = [&](float (&f)[n3], int dir, const float (&eo)[kEoSlots], const float* mat, bool tr) {
    // tr = false: the forward B (centre row e_h); tr = true: the transposed B^T w (centre
    // column zero off the centre) -- see eo_line
    const int st = dir == 0 ? 1 : (dir == 1 ? n : n * n);
#pragma unroll
    for (int b = 0; b < n * n; ++b) {
      const int base = dir == 0 ? b * n : (dir == 1 ? (b % n) + (b / n) * n * n : b);
      float x[n], y[n];
#pragma unroll
      for (int m = 0; m < n; ++m) x[m] = f[base + m * st];
      if constexpr (n % 2 == 1 && STRAT == NHMF_ON_THE_FLY) {
        if (tr)
          eo_line<n, false, kEoCentreCol>(eo, x, y);
        else
          eo_line<n, false, kEoCentreRow>(eo, x, y);
      } else {
#pragma unroll
        for (int r = 0; r < n; ++r) {
          float s = (tr ? mat[r] : mat[r * n]) * x[0];
#pragma unroll
          for (int m = 1; m < n; ++m) s = fmaf(tr ? mat[m * n + r] : mat[r * n + m], x[m], s);
          y[r] = s;
        }
      }
#pragma unroll
      for (int m = 0; m < n; ++m) f[base + m * st] = y[m];
    }
  };
  auto to_points = [&](float (&f)[3][n3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      pass(f[c], 0, a.eof[0], a.Bf, false);
      pass(f[c], 1, a.eof[0], a.Bf, false);
      pass(f[c], 2, a.eof[0], a.Bf, false);
    }
  };
  auto grad_at = [&](const float* Dc, const float (&f)[3][n3], int qx, int qy, int qz, float g[9]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float gx = Dc[qx * n] * f[c][idx(0, qy, qz)];
      float gy = Dc[qy * n] * f[c][idx(qx, 0, qz)];
      float gz = Dc[qz * n] * f[c][idx(qx, qy, 0)];
#pragma unroll
      for (int m = 1; m < n; ++m) {
        gx = fmaf(Dc[qx * n + m], f[c][idx(m, qy, qz)], gx);
        gy = fmaf(Dc[qy * n + m], f[c][idx(qx, m, qz)], gy);
        gz = fmaf(Dc[qz * n + m], f[c][idx(qx, qy, m)], gz);
      }
      g[3 * c + 0] = gx;
      g[3 * c + 1] = gy;
      g[3 * c + 2] = gz;
    }
  };

  float qv[3][n3];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int k = 0; k < n; ++k)
#pragma unroll
      for (int j = 0; j < n; ++j)
#pragma unroll
        for (int i = 0; i < n; ++i) {
          const bool fixed = is_constrained(a.bc, c, gi0 + i, gk0 + k, a.M);
          qv[c][idx(i, j, k)] = fixed ? 0.f : du[c * a.M3 + node(i, j, k)];
        }
  if (a.factor) {
    const float fac = float(elem_factor(a, ec));
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int q = 0; q < n3; ++q) qv[c][q] *= fac;
  }
  to_points(qv);
  float ub[STRAT == NHMF_ON_THE_FLY ? 3 : 1][STRAT == NHMF_ON_THE_FLY ? n3 : 1];
  if constexpr (STRAT == NHMF_ON_THE_FLY) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int k = 0; k < n; ++k)
#pragma unroll
        for (int j = 0; j < n; ++j)
#pragma unroll
          for (int i = 0; i < n; ++i) ub[c][idx(i, j, k)] = a.u32[c * a.M3 + node(i, j, k)];
    to_points(ub);
  }
  // Compressible model on the fly: the values of ubar at the points go to shared memory
  // ([3 n^3][T], one column per thread), and the kinematics (F^-1, J - 1, ln J) of each
  // qz-slice are computed in a rolled loop into a slice buffer ([10][n^2][T]) that the unrolled
  // point code then reads: the kinematics code exists once instead of n^3 times, which keeps
  // the unrolled kernel within the instruction cache, and ubar holds no registers there.
  constexpr bool KIN = STRAT == NHMF_ON_THE_FLY && MODEL == NHMF_MODEL_COMPRESSIBLE;
  constexpr int n2 = n * n;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* ubs = reinterpret_cast<float*>(smem_raw);
  float* kin = ubs + 3 * n3 * blockDim.x;
  const int T = blockDim.x;
  if constexpr (KIN) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int q = 0; q < n3; ++q) ubs[(c * n3 + q) * T + threadIdx.x] = ub[c][q];
  }

  float acc[3][n3];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int q = 0; q < n3; ++q) acc[c][q] = 0.f;
  const float r2 = float(a.r2mu), inv_mu = float(1.0 / a.mu);
  bool bad = false;
#pragma unroll
  for (int qz = 0; qz < n; ++qz) {
    if constexpr (KIN) {
#pragma unroll 1
      for (int pt = 0; pt < n2; ++pt) {
        const int qx = pt % n, qy = pt / n;
        const float* u0 = ubs + threadIdx.x;
        float H[9], Fi[9], lnJ;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
          for (int m = 0; m < n; ++m) {
            gx = fmaf(a.Dchf[qx * n + m], u0[(c * n3 + idx(m, qy, qz)) * T], gx);
            gy = fmaf(a.Dchf[qy * n + m], u0[(c * n3 + idx(qx, m, qz)) * T], gy);
            gz = fmaf(a.Dchf[qz * n + m], u0[(c * n3 + idx(qx, qy, m)) * T], gz);
          }
          H[3 * c + 0] = gx;
          H[3 * c + 1] = gy;
          H[3 * c + 2] = gz;
        }
        const float Jm1 = kinematics(H, Fi, lnJ);
        bad |= !(Jm1 > -1.f);
        float* k0 = kin + pt * T + threadIdx.x;
#pragma unroll
        for (int k = 0; k < 9; ++k) k0[k * n2 * T] = Fi[k];
        k0[9 * n2 * T] = lnJ;
      }
    }
#pragma unroll
    for (int qy = 0; qy < n; ++qy)
#pragma unroll
      for (int qx = 0; qx < n; ++qx) {
        const int q = idx(qx, qy, qz);
        float Fi[9], lnJ, Jm1 = 0.f, F[9];
        if constexpr (KIN) {
          const float* k0 = kin + (qx + n * qy) * T + threadIdx.x;
#pragma unroll
          for (int k = 0; k < 9; ++k) Fi[k] = k0[k * n2 * T];
          lnJ = k0[9 * n2 * T];
        } else if constexpr (STRAT == NHMF_ON_THE_FLY) {
          float H[9];
          grad_at(a.Dchf, ub, qx, qy, qz, H);  // physical gradient: Dch = Dc / h
          Jm1 = kinematics(H, Fi, lnJ);
          bad |= !(Jm1 > -1.f);
#pragma unroll
          for (int k = 0; k < 9; ++k) F[k] = (k % 4 == 0 ? 1.f : 0.f) + H[k];
        } else {
#pragma unroll
          for (int k = 0; k < 9; ++k) Fi[k] = ld_policy(cache + (k * n3 + q) * kTile, stream_pol);
          lnJ = ld_policy(cache + (9 * n3 + q) * kTile, stream_pol);
        }
        float dH[9], g[9];
        grad_at(a.Dcf, qv, qx, qy, qz, dH);
        if constexpr (STRAT == NHMF_ON_THE_FLY && MODEL == NHMF_MODEL_SPLIT)
          split_stress_dP(F, Fi, lnJ, Jm1, dH, float(a.mu), float(a.lam), inv_mu, g);
        else
          linearised_stress_unit(Fi, lnJ, dH, r2, g);
        // transposed collocation derivative with the weights, mu and h:
        //   acc[c][point on the line through q] += DcW[q][m] g
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int m = 0; m < n; ++m) {
            acc[c][idx(m, qy, qz)] = fmaf(a.DcWf[qx * n + m], g[3 * c + 0], acc[c][idx(m, qy, qz)]);
            acc[c][idx(qx, m, qz)] = fmaf(a.DcWf[qy * n + m], g[3 * c + 1], acc[c][idx(qx, m, qz)]);
            acc[c][idx(qx, qy, m)] = fmaf(a.DcWf[qz * n + m], g[3 * c + 2], acc[c][idx(qx, qy, m)]);
          }
      }
  }
  if (bad) atomicOr(a.status, kStatusNonPosJ);
  // transposed weighted interpolation back to the nodes: out[i] = sum_q B[q][i] w_q acc[q]
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    pass(acc[c], 0, a.eof[2], a.BWf, true);
    pass(acc[c], 1, a.eof[2], a.BWf, true);
    pass(acc[c], 2, a.eof[2], a.BWf, true);
  }
  const unsigned long long keep_pol = l2_evict_last();  // read back by the gather that follows
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int q = 0; q < n3; ++q) st_policy(vloc + (c * n3 + q) * kTile, acc[c][q], keep_pol);
}

// ------------------------------------------------------------------ element-local gather
// v[c][node] = sum of vloc(e; c, q) over the elements e whose closure holds the node (1, 2, 4
// or 8 of them; q the node's local index in e), always in increasing (ez, ey, ex) order, so
// the result is bitwise deterministic without atomics.  Dirichlet rows (unless raw):
// v = du there.  One thread per node.
template <int P>
__global__ void __launch_bounds__(256) k_gather_local(const float* __restrict__ vloc, const float* __restrict__ du,
                                                     float* __restrict__ v, int N, int M, int bc) {
  constexpr int n = P + 1, n3 = n * n * n;
  static_assert(kTile == 32, "tile index by shift and mask");
  // grid: x covers the M^2 nodes of one z-plane, y the plane (32-bit index arithmetic; the
  // launcher keeps the element count below 2^31)
  const int ij = blockIdx.x * blockDim.x + threadIdx.x;
  if (ij >= M * M) return;
  const int gj = ij / M;
  const int g[3] = {ij - gj * M, gj, (int)blockIdx.y};
  const long long node = ij + (long long)M * M * blockIdx.y, M3 = (long long)M * M * M;
  const unsigned long long done_pol = l2_evict_first();  // each element-local value is read once
  // per direction: the element below the node (local index P), if any, then the element at or
  // above it (local index g % P); an absent element in x gets a clamped (valid) index and is
  // masked after the load
  int el[3][2], lo[3][2];
  bool has[3][2];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int gp = g[d] / P, gr = g[d] - gp * P;
    const bool shared = gr == 0;
    has[d][0] = shared && g[d] > 0;
    el[d][0] = max(gp - 1, 0);
    lo[d][0] = P;
    has[d][1] = !shared || g[d] < M - 1;
    el[d][1] = min(gp, N - 1);
    lo[d][1] = gr;
  }
  // the (z, y) element pairs are the same for every node of a grid row, so a warp skips the
  // absent ones as a whole (a branch, not 6 issued loads); the loads of the present ones are
  // issued before any of them is used
  float val[3][8];
#pragma unroll
  for (int z = 0; z < 2; ++z)
#pragma unroll
    for (int y = 0; y < 2; ++y) {
#pragma unroll
      for (int c = 0; c < 3; ++c) val[c][4 * z + 2 * y] = val[c][4 * z + 2 * y + 1] = 0.f;
      if (!(has[2][z] && has[1][y])) continue;
#pragma unroll
      for (int x = 0; x < 2; ++x) {
        const unsigned e = (unsigned)el[0][x] + (unsigned)N * ((unsigned)el[1][y] + (unsigned)N * (unsigned)el[2][z]);
        const int q = lo[0][x] + n * (lo[1][y] + n * lo[2][z]);
        const float* src = vloc + (size_t)(e >> 5) * (3 * n3 * kTile) + q * kTile + (e & 31u);
#pragma unroll
        for (int c = 0; c < 3; ++c) val[c][4 * z + 2 * y + x] = ld_policy(src + c * n3 * kTile, done_pol);
      }
    }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float s = 0.f;
#pragma unroll
    for (int z = 0; z < 2; ++z)
#pragma unroll
      for (int y = 0; y < 2; ++y)
#pragma unroll
        for (int x = 0; x < 2; ++x)
          if (has[2][z] && has[1][y] && has[0][x]) s += val[c][4 * z + 2 * y + x];
    if (is_constrained(bc, c, g[0], g[2], M)) s = du[c * M3 + node];
    v[c * M3 + node] = s;
  }
}

// ------------------------------------------------------------------ point cache
template <int P>
__global__ void __launch_bounds__(Cfg<P, double>::THREADS) k_cache(const OpArgs a) {
  using T = double;
  constexpr int n = P + 1, n3 = n * n * n, NE = Cfg<P, T>::NE, NI = NE * n3;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sB = reinterpret_cast<T*>(smem_raw);
  T* sDc = sB + kMaxN * kMaxN;
  T* sD = sDc + kMaxN * kMaxN;
  T* sW = sD + kMaxN * kMaxN;
  T* A = sB + kTabSlots;  // [3][NI]
  T* Vq = A + 3 * NI;     // [3][NI]
  load_tables<P>(a, sB, sDc, sD, sW, 1.0);
  const long long e0 = (long long)blockIdx.x * NE;
  const int nvalid = (int)min((long long)NE, (long long)a.col.count - e0);
  gather<P, NI>(a, a.u64, e0, nvalid, false, A);
  __syncthreads();
  to_points<n, NI>(sB, A, Vq, Vq, nvalid * n3);
  const double invh = 1.0 / a.h;
  const long long cbase = (a.col.slot0 + e0) * n3;
  bool bad = false;
  for (int t = threadIdx.x; t < nvalid * n3; t += blockDim.x) {
    double H[9], Fi[9], lnJ;
    colloc_grad<n, NI>(sDc, Vq, t, H);
#pragma unroll
    for (int k = 0; k < 9; ++k) H[k] *= invh;
    const double Jm1 = kinematics(H, Fi, lnJ);
    bad |= !(Jm1 > -1.0);
    if (a.cache64_out) {
#pragma unroll
      for (int k = 0; k < 9; ++k) a.cache64_out[k * a.nq + cbase + t] = Fi[k];
      a.cache64_out[9 * a.nq + cbase + t] = lnJ;
    }
    if (a.cachesp_out) {
      // Algorithm 2 cache from the model's P and dP only: tau = P F^T;
      // J a_ijkl = (dP[e_k (x) F_l.] F^T)_ij, J c_ijkl = J a_ijkl - delta_ik tau_jl
      double F[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) F[k] = (k % 4 == 0 ? 1.0 : 0.0) + H[k];
      double P[9], tau[9];
      model_piola(a.model, F, Fi, lnJ, Jm1, a.mu, a.lam, P);
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
          tau[3 * i + j] = fma(P[3 * i], F[3 * j], fma(P[3 * i + 1], F[3 * j + 1], P[3 * i + 2] * F[3 * j + 2]));
      double* out = a.cachesp_out;
      const int pk[6] = {0, 1, 2, 1, 0, 0}, pl[6] = {0, 1, 2, 2, 2, 1};
#pragma unroll
      for (int K = 0; K < 6; ++K) {
        const int k = pk[K], l = pl[K];
        double X[9], dP[9];
#pragma unroll
        for (int m = 0; m < 3; ++m)
#pragma unroll
          for (int L = 0; L < 3; ++L) X[3 * m + L] = (m == k) ? F[3 * l + L] : 0.0;
        model_dP(a.model, F, Fi, lnJ, Jm1, X, a.mu, a.lam, 1.0, dP);
#pragma unroll
        for (int I = 0; I <= K; ++I) {
          const int i = pk[I], j = pl[I];
          const double Ja = fma(dP[3 * i], F[3 * j], fma(dP[3 * i + 1], F[3 * j + 1], dP[3 * i + 2] * F[3 * j + 2]));
          out[tri6(I, K) * a.nq + cbase + t] = Ja - (i == k ? tau[3 * j + l] : 0.0);
        }
      }
      const int vi[6] = {0, 4, 8, 5, 2, 1};  // tau in Voigt order 11, 22, 33, 23, 13, 12
#pragma unroll
      for (int V = 0; V < 6; ++V) out[(21 + V) * a.nq + cbase + t] = tau[vi[V]];
#pragma unroll
      for (int k = 0; k < 9; ++k) out[(27 + k) * a.nq + cbase + t] = Fi[k];
    }
    if (a.cachedf_out) {
      auto split = [](double d) {
        const float hi = __double2float_rn(d);
        return make_float2(hi, __double2float_rn(d - (double)hi));
      };
#pragma unroll
      for (int k = 0; k < 9; ++k) a.cachedf_out[k * a.nq + cbase + t] = split(Fi[k]);
      a.cachedf_out[9 * a.nq + cbase + t] = split(lnJ);
    }
    if (a.cache32_out) {
      // the FP32 applies run over all elements in natural order (element-local results)
      const long long en = elem_natural(a, e0 + t / n3), q = t % n3;
      if (P <= kRegMaxP && a.reg32) {
        // element tiles [E/32][10][n^3][32] for the register kernel (one thread per element)
        float* tile = a.cache32_out + (en / kTile) * (10 * n3 * kTile) + en % kTile;
#pragma unroll
        for (int k = 0; k < 9; ++k) tile[(k * n3 + q) * kTile] = float(Fi[k]);
        tile[(9 * n3 + q) * kTile] = float(lnJ);
      } else {
        // layout [10][E n^3] for the shared-memory kernel
#pragma unroll
        for (int k = 0; k < 9; ++k) a.cache32_out[k * a.nq + en * n3 + q] = float(Fi[k]);
        a.cache32_out[9 * a.nq + en * n3 + q] = float(lnJ);
      }
    }
  }
  if (bad) atomicOr(a.status, kStatusNonPosJ);
}

// ------------------------------------------------------------------ residual
template <int P>
__global__ void __launch_bounds__(LaunchCfg<P, double, 0>::THREADS) k_residual(const OpArgs a) {
  using T = double;
  constexpr int n = P + 1, n3 = n * n * n, NE = LaunchCfg<P, T, 0>::NE, NI = NE * n3;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sB = reinterpret_cast<T*>(smem_raw);
  T* sDc = sB + kMaxN * kMaxN;
  T* sD = sDc + kMaxN * kMaxN;
  T* sW = sD + kMaxN * kMaxN;
  T* Vq = sB + kTabSlots;  // [3][NI]
  T* G = Vq + 3 * NI;      // [9][NI]
  load_tables<P>(a, sB, sDc, sD, sW, a.h * a.h);
  const long long e0 = (long long)blockIdx.x * NE;
  const int nvalid = (int)min((long long)NE, (long long)a.col.count - e0);
  gather<P, NI>(a, a.u64, e0, nvalid, false, G);
  __syncthreads();
  const int nitems = nvalid * n3;
  to_points<n, NI>(sB, G, Vq, Vq, nitems);
  const double invh = 1.0 / a.h;
  unsigned flags = 0;
  for (int t = threadIdx.x; t < nitems; t += blockDim.x) {
    double H[9], Fi[9], lnJ;
    colloc_grad<n, NI>(sDc, Vq, t, H);
#pragma unroll
    for (int k = 0; k < 9; ++k) H[k] *= invh;
    const double Jm1 = kinematics(H, Fi, lnJ);
    // a NaN deformation gradient is a non-finite input; det F <= 0 makes P non-finite too,
    // but is reported as what it is (the Newton backtracking acts on it)
    const bool inverted = Jm1 <= -1.0;
    if (inverted) flags |= kStatusNonPosJ;
    const double s = sW[t % n3] * elem_factor(a, e0 + min(t / n3, nvalid - 1));
    double F[9], P[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) F[k] = (k % 4 == 0 ? 1.0 : 0.0) + H[k];
    model_piola(a.model, F, Fi, lnJ, Jm1, a.mu, a.lam, P);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      if (!inverted && !isfinite(P[k])) flags |= kStatusNonFinite;
      G[k * NI + t] = s * P[k];
    }
  }
  if (flags) atomicOr(a.status, flags);
  __syncthreads();
  from_points<n, NI>(sB, sDc, G, Vq, G + 3 * NI, nitems);
  scatter_add<P, NI>(a, G + 3 * NI, e0, nvalid, static_cast<double*>(a.v));
}

// ------------------------------------------------------------------ diagonal
// diag(K)_{c,I} = sum_q sum_{d,l} L_{cdcl} dphi_I/dX_d dphi_I/dX_l w_q h^3 with
// L_{cdcl} = mu delta_dl + (mu + 2 lambda (1 - ln J)) Finv[d][c] Finv[l][c].  The products
// of 1D factors are separable, so each (d, l) pair is three transposed passes with the
// elementwise-product tables BB, BD, DD.
template <int P> struct DiagCfg { static constexpr int NE = Cfg<P, double>::NE / 2 > 0 ? Cfg<P, double>::NE / 2 : 1; };

template <int P>
__global__ void __launch_bounds__(Cfg<P, double>::THREADS) k_diagonal(const OpArgs a) {
  using T = double;
  constexpr int n = P + 1, n3 = n * n * n, NE = DiagCfg<P>::NE, NI = NE * n3;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sB = reinterpret_cast<T*>(smem_raw);
  T* sDc = sB + kMaxN * kMaxN;
  T* sD = sDc + kMaxN * kMaxN;
  T* sW = sD + kMaxN * kMaxN;
  T* sBB = sB + kTabSlots;  // 3 product tables, n*n each
  T* sBD = sBB + kMaxN * kMaxN;
  T* sDD = sBD + kMaxN * kMaxN;
  T* Cq = sDD + kMaxN * kMaxN + 1;  // [20][NI]: Finv (9), ln J, and for the split model F (9), J - 1
  T* S = Cq + 20 * NI;              // [3][NI]
  T* tmp = S + 3 * NI;              // [3][NI]
  T* R = tmp + 3 * NI;              // [3][NI]
  load_tables<P>(a, sB, sDc, sD, sW, a.h);
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
    const int q = i / n, k = i % n;
    sBB[i] = a.B[q * n + k] * a.B[q * n + k];
    sBD[i] = a.B[q * n + k] * a.D[q * n + k];
    sDD[i] = a.D[q * n + k] * a.D[q * n + k];
  }
  const long long e0 = (long long)blockIdx.x * NE;
  const int nvalid = (int)min((long long)NE, (long long)a.col.count - e0);
  gather<P, NI>(a, a.u64, e0, nvalid, false, S);
  __syncthreads();
  const int nitems = nvalid * n3;
  to_points<n, NI>(sB, S, tmp, tmp, nitems);
  const double invh = 1.0 / a.h;
  for (int t = threadIdx.x; t < nitems; t += blockDim.x) {
    double H[9], Fi[9], lnJ;
    colloc_grad<n, NI>(sDc, tmp, t, H);
#pragma unroll
    for (int k = 0; k < 9; ++k) H[k] *= invh;
    const double Jm1 = kinematics(H, Fi, lnJ);
#pragma unroll
    for (int k = 0; k < 9; ++k) Cq[k * NI + t] = Fi[k];
    Cq[9 * NI + t] = lnJ;
    if (a.model == NHMF_MODEL_SPLIT) {
#pragma unroll
      for (int k = 0; k < 9; ++k) Cq[(10 + k) * NI + t] = (k % 4 == 0 ? 1.0 : 0.0) + H[k];
      Cq[19 * NI + t] = Jm1;
    }
    for (int c = 0; c < 3; ++c) R[c * NI + t] = 0.0;
  }
  __syncthreads();
  for (int d = 0; d < 3; ++d)
    for (int l = d; l < 3; ++l) {
      for (int t = threadIdx.x; t < nitems; t += blockDim.x) {
        const double s = sW[t % n3] * (d == l ? 1.0 : 2.0) * elem_factor(a, e0 + min(t / n3, nvalid - 1));
        if (a.model == NHMF_MODEL_SPLIT) {
          // L_cdcl = mu a d_dl - 2/3 mu a (F_cd Fi_lc + Fi_dc F_cl) + (2/9 mu a I1 + kappa J^2
          //          + mu a I1/3 - kappa/2 (J^2 - 1)) Fi_dc Fi_lc
          const double lnJ = Cq[9 * NI + t], J = 1.0 + Cq[19 * NI + t], J2 = J * J;
          const double mua = a.mu * exp(-2.0 / 3.0 * lnJ);
          double I1 = 0.0;
#pragma unroll
          for (int k = 0; k < 9; ++k) I1 += Cq[(10 + k) * NI + t] * Cq[(10 + k) * NI + t];
          const double cff = 2.0 / 9.0 * mua * I1 + a.lam * J2 + mua * I1 / 3.0 - 0.5 * a.lam * (J2 - 1.0);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const double Fidc = Cq[(3 * d + c) * NI + t], Filc = Cq[(3 * l + c) * NI + t];
            const double Fcd = Cq[(10 + 3 * c + d) * NI + t], Fcl = Cq[(10 + 3 * c + l) * NI + t];
            const double L = (d == l ? mua : 0.0) - 2.0 / 3.0 * mua * (Fcd * Filc + Fidc * Fcl) + cff * Fidc * Filc;
            S[c * NI + t] = s * L;
          }
        } else {
          const double kap = a.mu + 2.0 * a.lam * (1.0 - Cq[9 * NI + t]);
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const double L = (d == l ? a.mu : 0.0) + kap * Cq[(3 * d + c) * NI + t] * Cq[(3 * l + c) * NI + t];
            S[c * NI + t] = s * L;
          }
        }
      }
      __syncthreads();
      // direction x uses DD if d == l == 0, BD if exactly one of d, l is 0, else BB
      const T* mx = (d == 0 && l == 0) ? sDD : ((d == 0 || l == 0) ? sBD : sBB);
      const T* my = (d == 1 && l == 1) ? sDD : ((d == 1 || l == 1) ? sBD : sBB);
      const T* mz = (d == 2 && l == 2) ? sDD : ((d == 2 || l == 2) ? sBD : sBB);
      sf_pass<n, NI, 3, 0, true, false>(mx, S, tmp, nitems);
      __syncthreads();
      sf_pass<n, NI, 3, 1, true, false>(my, tmp, S, nitems);
      __syncthreads();
      sf_pass<n, NI, 3, 2, true, true>(mz, S, R, nitems);
      __syncthreads();
    }
  scatter_add<P, NI>(a, R, e0, nvalid, static_cast<double*>(a.v));
}

// ------------------------------------------------------------------ Dirichlet rows
// mode 0: out[d] = src[d]; mode 1: out[d] = value, on every constrained DoF.
template <typename T>
__global__ void k_fix_constrained(int bc, int M, long long M3, const T* src, T* out, int mode, T value) {
  const long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long M2 = (long long)M * M;
  if (f >= M2) return;
  const int x = int(f % M), y = int(f / M);
  auto fix = [&](int c, long long node) {
    const long long d = c * M3 + node;
    out[d] = mode == 0 ? src[d] : value;
  };
  if (bc == NHMF_BC_CLAMP_X0) {
    const long long node = (long long)M * (x + (long long)M * y);  // (0, x, y)
    for (int c = 0; c < 3; ++c) fix(c, node);
  } else if (bc == NHMF_BC_COMPRESSION) {
    const long long bottom = x + (long long)M * y;
    const long long top = bottom + M2 * (M - 1);
    for (int c = 0; c < 3; ++c) fix(c, bottom);
    fix(2, top);
  }
}

__global__ void k_to_fp32(const double* x, float* y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = float(x[i]);
}

// ------------------------------------------------------------------ host side
// Even-odd coefficients (see eo_line) of the n x n row-major operator M, odd n.
void eo_pack(const double* M, int n, double* k) {
  const int h = n / 2, A0 = (h + 1) * h, C0 = 2 * (h + 1) * h;
  for (int i = 0; i < kEoSlots; ++i) k[i] = 0.0;
  for (int r = 0; r <= h; ++r) {
    for (int m = 0; m < h; ++m) {
      k[r * h + m] = 0.5 * (M[r * n + m] + M[r * n + n - 1 - m]);
      k[A0 + r * h + m] = 0.5 * (M[r * n + m] - M[r * n + n - 1 - m]);
    }
    k[C0 + r] = M[r * n + h];
  }
}

OpArgs base_args(nhmf_ctx* c) {
  OpArgs a{};
  a.N = c->g.N;
  a.M = c->g.M;
  a.bc = c->prm.bc;
  a.model = c->prm.model;
  a.M3 = c->g.M3;
  a.nq = c->g.nq;
  a.h = c->g.h;
  a.mu = c->prm.mu;
  a.lam = c->prm.lambda;
  const int n = c->g.n;
  for (int q = 0; q < n; ++q) {
    a.w[q] = c->tab.w[q];
    for (int i = 0; i < n; ++i) {
      a.B[q * n + i] = c->tab.B[q][i];
      a.Dc[q * n + i] = c->tab.Dc[q][i];
      a.D[q * n + i] = c->tab.D[q][i];
      a.Bf[q * n + i] = float(c->tab.B[q][i]);
      a.Dcf[q * n + i] = float(c->tab.Dc[q][i]);
    }
    a.wf[q] = float(c->tab.w[q]);
  }
  // tables of the tangent apply (see OpArgs)
  double BWt[kMaxN * kMaxN], DcWt[kMaxN * kMaxN];
  for (int q = 0; q < n; ++q)
    for (int i = 0; i < n; ++i) {
      const double wq = c->tab.w[q];
      a.BW[q * n + i] = c->tab.B[q][i] * wq;
      BWt[i * n + q] = a.BW[q * n + i];
      a.DcW[q * n + i] = c->tab.Dc[q][i] * wq / c->tab.w[i] * c->prm.mu * c->g.h;
      DcWt[i * n + q] = a.DcW[q * n + i];
      a.Dch[q * n + i] = c->tab.Dc[q][i] / c->g.h;
    }
  if (n % 2 == 1) {
    eo_pack(a.B, n, a.eo[0]);
    eo_pack(a.Dc, n, a.eo[1]);
    eo_pack(BWt, n, a.eo[2]);
    eo_pack(DcWt, n, a.eo[3]);  // DcW^T is anti-centro-symmetric like Dc (symmetric weights)
  }
  a.r2mu = 2.0 * c->prm.lambda / c->prm.mu;
  a.reg32 = c->reg32 ? 1 : 0;
  for (int i = 0; i < kMaxN * kMaxN; ++i) {
    a.BWf[i] = float(a.BW[i]);
    a.DcWf[i] = float(a.DcW[i]);
    a.Dchf[i] = float(a.Dch[i]);
  }
  for (int k = 0; k < 4; ++k)
    for (int i = 0; i < kEoSlots; ++i) a.eof[k][i] = float(a.eo[k][i]);
  a.status = c->status;
  a.factor = c->factor;
  return a;
}

template <typename KernelT>
cudaError_t prepare(KernelT kernel, size_t smem) {
  if (smem > 48 * 1024)
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaSuccess;
}

// Runs `kernel` once per colour class with NE elements per block.
template <typename KernelT>
nhmf_status run_colours(nhmf_ctx* c, KernelT kernel, OpArgs a, int NE, int threads, size_t smem,
                        cudaStream_t s, const char* what, int kind) {
  if (cudaError_t e = prepare(kernel, smem); e != cudaSuccess) return cuda_check(c, e, what);
  nhmf_ctx::Rec rec{kind, 0, nullptr, nullptr};
  if (c->profiling) {
    cudaEventCreate(&rec.a);
    cudaEventCreate(&rec.b);
    cudaEventRecord(rec.a, s);
  }
  for (int k = 0; k < 8; ++k) {
    const Colour& col = c->g.colour[k];
    if (col.count == 0) continue;
    a.col = col;
    const int blocks = (col.count + NE - 1) / NE;
    kernel<<<blocks, threads, smem, s>>>(a);
    ++rec.launches;
  }
  if (c->profiling) {
    cudaEventRecord(rec.b, s);
    c->prof.push_back(rec);
  }
  return cuda_check(c, cudaGetLastError(), what);
}

// The element-local FP32 apply: `kernel` once over the class of all elements (NE per block),
// writing c->vloc, then k_gather_local<P> onto v with the Dirichlet rows (bc of `a`).
template <int P, typename KernelT>
nhmf_status run_local(nhmf_ctx* c, KernelT kernel, OpArgs a, int NE, int threads, size_t smem, const float* du,
                      float* v, cudaStream_t s) {
  if (cudaError_t e = prepare(kernel, smem); e != cudaSuccess) return cuda_check(c, e, "apply");
  if (!c->vloc) return fail(c, NHMF_ERR_STATE, "apply: no element-local buffer (set_linearization first)");
  if (c->g.E > 0x7fffffffLL || (long long)c->g.M * c->g.M > 0x7fffffffLL)
    return fail(c, NHMF_ERR_ARG, "apply: the FP32 element-local path needs fewer than 2^31 elements");
  nhmf_ctx::Rec rec{NHMF_KIND_APPLY, 2, nullptr, nullptr};
  if (c->profiling) {
    cudaEventCreate(&rec.a);
    cudaEventCreate(&rec.b);
    cudaEventRecord(rec.a, s);
  }
  a.col = c->g.all;
  a.vloc = c->vloc;
  kernel<<<(unsigned)((c->g.E + NE - 1) / NE), threads, smem, s>>>(a);
  const dim3 gather_grid((unsigned)(((long long)c->g.M * c->g.M + 255) / 256), (unsigned)c->g.M);
  k_gather_local<P><<<gather_grid, 256, 0, s>>>(c->vloc, du, v, c->g.N, c->g.M, a.bc);
  if (c->profiling) {
    cudaEventRecord(rec.b, s);
    c->prof.push_back(rec);
  }
  return cuda_check(c, cudaGetLastError(), "apply");
}

template <typename T>
nhmf_status fix_rows(nhmf_ctx* c, const T* src, T* out, int mode, T value, cudaStream_t s) {
  if (c->prm.bc == NHMF_BC_NONE) return NHMF_OK;
  const long long M2 = (long long)c->g.M * c->g.M;
  k_fix_constrained<T><<<(unsigned)((M2 + 255) / 256), 256, 0, s>>>(c->prm.bc, c->g.M, c->g.M3, src, out, mode, value);
  return cuda_check(c, cudaGetLastError(), "dirichlet rows");
}

template <int P, typename T, int STRAT>
nhmf_status apply_p(nhmf_ctx* c, const void* du, void* v, bool raw, cudaStream_t s) {
  using S = typename Store<T>::type;
  constexpr int n3 = (P + 1) * (P + 1) * (P + 1), NE = LaunchCfg<P, T, STRAT>::NE, NI = NE * n3;
  OpArgs a = base_args(c);
  if (raw) a.bc = NHMF_BC_NONE;  // unconstrained operator K: no masking, no identity rows
  a.u64 = c->u_at ? c->u_at : c->ubar;
  a.u32 = c->ubar32;
  a.du = du;
  a.v = v;
  a.cache = std::is_same<T, df64>::value ? (const void*)c->cachedf
            : (sizeof(T) == 8 ? (const void*)c->cache64 : (const void*)c->cache32);
  a.cachesp_in = c->cachesp;
  const size_t slots = kTabSlots + (STRAT == NHMF_ON_THE_FLY ? 15 : 12) * (size_t)NI;  // spatial: as cached
  const size_t smem = slots * sizeof(T);
  // the energy model is a compile-time parameter of the on-the-fly point code (a runtime
  // branch would charge the split model's registers to every model)
  constexpr int SPLIT = STRAT == NHMF_ON_THE_FLY ? NHMF_MODEL_SPLIT : NHMF_MODEL_COMPRESSIBLE;
  const bool split = STRAT == NHMF_ON_THE_FLY && c->prm.model == NHMF_MODEL_SPLIT;
  if constexpr (std::is_same<T, float>::value) {
    // FP32: one launch over all elements with element-local results, then the node gather
    // (which also writes the Dirichlet rows): no memset, no colour classes
    const float* du32 = static_cast<const float*>(du);
    float* v32 = static_cast<float*>(v);
    if constexpr (P <= kRegMaxP) {
      if (c->reg32) {
        // the compressible on-the-fly kernel's point values and slice kinematics (see k_apply_reg)
        constexpr size_t n3 = (P + 1) * (P + 1) * (P + 1), n2 = (P + 1) * (P + 1);
        const size_t kin_smem = (3 * n3 + 10 * n2) * kRegThreads * sizeof(float);
        if (split)
          return run_local<P>(c, k_apply_reg<P, STRAT, SPLIT>, a, kRegThreads, kRegThreads, 0, du32, v32, s);
        return run_local<P>(c, k_apply_reg<P, STRAT, NHMF_MODEL_COMPRESSIBLE>, a, kRegThreads, kRegThreads,
                            STRAT == NHMF_ON_THE_FLY ? kin_smem : 0, du32, v32, s);
      }
    }
    auto* k = split ? k_apply<P, T, STRAT, SPLIT> : k_apply<P, T, STRAT, NHMF_MODEL_COMPRESSIBLE>;
    return run_local<P>(c, k, a, NE, LaunchCfg<P, T, STRAT>::THREADS, smem, du32, v32, s);
  }
  if (cudaError_t e = cudaMemsetAsync(v, 0, sizeof(S) * 3 * c->g.M3, s); e != cudaSuccess)
    return cuda_check(c, e, "apply memset");
  nhmf_status st;
  {
    auto* k = split ? k_apply<P, T, STRAT, SPLIT> : k_apply<P, T, STRAT, NHMF_MODEL_COMPRESSIBLE>;
    st = run_colours(c, k, a, NE, LaunchCfg<P, T, STRAT>::THREADS, smem, s, "apply", NHMF_KIND_APPLY);
  }
  if (st != NHMF_OK || raw) return st;
  return fix_rows<S>(c, static_cast<const S*>(du), static_cast<S*>(v), 0, S(0), s);
}

template <int P>
nhmf_status apply_dispatch_p(nhmf_ctx* c, int prec, int strat, const void* du, void* v, bool raw, cudaStream_t s) {
  if (prec == NHMF_DF64) {
    if (strat != NHMF_CACHED) return fail(c, NHMF_ERR_ARG, "df64 apply: cached strategy only");
    return apply_p<P, df64, NHMF_CACHED>(c, du, v, raw, s);
  }
  if (prec == NHMF_FP64) {
    if (strat == NHMF_SPATIAL) return apply_p<P, double, NHMF_SPATIAL>(c, du, v, raw, s);
    return strat == NHMF_CACHED ? apply_p<P, double, NHMF_CACHED>(c, du, v, raw, s)
                                : apply_p<P, double, NHMF_ON_THE_FLY>(c, du, v, raw, s);
  }
  return strat == NHMF_CACHED ? apply_p<P, float, NHMF_CACHED>(c, du, v, raw, s)
                              : apply_p<P, float, NHMF_ON_THE_FLY>(c, du, v, raw, s);
}

template <int P>
nhmf_status cache_p(nhmf_ctx* c, cudaStream_t s) {
  constexpr int n3 = (P + 1) * (P + 1) * (P + 1), NE = Cfg<P, double>::NE, NI = NE * n3;
  OpArgs a = base_args(c);
  a.u64 = c->ubar;
  a.cache64_out = c->cache64;
  a.cache32_out = c->cache32;
  a.cachedf_out = c->cachedf;
  a.cachesp_out = c->cachesp;
  const size_t smem = (kTabSlots + 6 * (size_t)NI) * sizeof(double);
  return run_colours(c, k_cache<P>, a, NE, Cfg<P, double>::THREADS, smem, s, "cache build", NHMF_KIND_CACHE);
}

template <int P>
nhmf_status residual_p(nhmf_ctx* c, const double* u, double* r, cudaStream_t s) {
  constexpr int n3 = (P + 1) * (P + 1) * (P + 1), NE = LaunchCfg<P, double, 0>::NE, NI = NE * n3;
  OpArgs a = base_args(c);
  a.u64 = u;
  a.v = r;
  const size_t smem = (kTabSlots + 12 * (size_t)NI) * sizeof(double);
  if (cudaError_t e = cudaMemsetAsync(r, 0, sizeof(double) * 3 * c->g.M3, s); e != cudaSuccess)
    return cuda_check(c, e, "residual memset");
  nhmf_status st =
      run_colours(c, k_residual<P>, a, NE, LaunchCfg<P, double, 0>::THREADS, smem, s, "residual", NHMF_KIND_RESIDUAL);
  if (st != NHMF_OK) return st;
  return fix_rows<double>(c, nullptr, r, 1, 0.0, s);
}

template <int P>
nhmf_status diagonal_p(nhmf_ctx* c, double* d, cudaStream_t s) {
  constexpr int n3 = (P + 1) * (P + 1) * (P + 1), NE = DiagCfg<P>::NE, NI = NE * n3;
  OpArgs a = base_args(c);
  a.u64 = c->ubar;
  a.v = d;
  const size_t smem = (kTabSlots + 3 * kMaxN * kMaxN + 1 + 29 * (size_t)NI) * sizeof(double);
  if (cudaError_t e = cudaMemsetAsync(d, 0, sizeof(double) * 3 * c->g.M3, s); e != cudaSuccess)
    return cuda_check(c, e, "diagonal memset");
  nhmf_status st = run_colours(c, k_diagonal<P>, a, NE, Cfg<P, double>::THREADS, smem, s, "diagonal", NHMF_KIND_DIAGONAL);
  if (st != NHMF_OK) return st;
  return fix_rows<double>(c, nullptr, d, 1, 1.0, s);
}

}  // namespace

nhmf_status launch_apply(nhmf_ctx* c, int prec, int strat, const void* du, void* v, cudaStream_t s, bool raw) {
  switch (c->g.p) {
    case 1: return apply_dispatch_p<1>(c, prec, strat, du, v, raw, s);
    case 2: return apply_dispatch_p<2>(c, prec, strat, du, v, raw, s);
    case 3: return apply_dispatch_p<3>(c, prec, strat, du, v, raw, s);
    case 4: return apply_dispatch_p<4>(c, prec, strat, du, v, raw, s);
  }
  return fail(c, NHMF_ERR_ARG, "degree out of range");
}

nhmf_status launch_cache_build(nhmf_ctx* c, cudaStream_t s) {
  switch (c->g.p) {
    case 1: return cache_p<1>(c, s);
    case 2: return cache_p<2>(c, s);
    case 3: return cache_p<3>(c, s);
    case 4: return cache_p<4>(c, s);
  }
  return fail(c, NHMF_ERR_ARG, "degree out of range");
}

nhmf_status launch_residual(nhmf_ctx* c, const double* u, double* r, cudaStream_t s) {
  switch (c->g.p) {
    case 1: return residual_p<1>(c, u, r, s);
    case 2: return residual_p<2>(c, u, r, s);
    case 3: return residual_p<3>(c, u, r, s);
    case 4: return residual_p<4>(c, u, r, s);
  }
  return fail(c, NHMF_ERR_ARG, "degree out of range");
}

nhmf_status launch_diagonal(nhmf_ctx* c, double* d, cudaStream_t s) {
  switch (c->g.p) {
    case 1: return diagonal_p<1>(c, d, s);
    case 2: return diagonal_p<2>(c, d, s);
    case 3: return diagonal_p<3>(c, d, s);
    case 4: return diagonal_p<4>(c, d, s);
  }
  return fail(c, NHMF_ERR_ARG, "degree out of range");
}

nhmf_status fix_rows64(nhmf_ctx* c, const double* src, double* out, int mode, double value, cudaStream_t s) {
  return fix_rows<double>(c, src, out, mode, value, s);
}

nhmf_status fix_rows32(nhmf_ctx* c, const float* src, float* out, int mode, float value, cudaStream_t s) {
  return fix_rows<float>(c, src, out, mode, value, s);
}

nhmf_status launch_to_fp32(const double* x, float* y, long long n, cudaStream_t s) {
  k_to_fp32<<<1216, 256, 0, s>>>(x, y, n);
  return cudaGetLastError() == cudaSuccess ? NHMF_OK : NHMF_ERR_CUDA;
}

}  // namespace nhmf
