/*
 * Plain sum-factorised tangent application on the CPU, FP64 (oracle; test infrastructure and
 * the timed CPU baseline only -- the product path never links it).
 *
 * It computes the same operator as oracle/fem.py (the direct route with an explicit L) and is
 * checked against it in tests/test_oracle_sumfact.py; it exists to be timed on the host cores
 * beside the GPU library.
 *
 * Algorithm 1 of the paper, element by element:
 *   gather the element's nodal values of u and du (du zeroed on constrained DoFs);
 *   sum factorisation (Section 2.4): values and reference gradients at the (p+1)^3 Gauss
 *     points by 1D passes with B[q][i] = l_i(x_q) and D[q][i] = l_i'(x_q) per direction,
 *     Grad = (1/h) grad_ref on the affine cube;
 *   point code: F = I + Grad u, J = det F, F^-1, ln J, and the linearised first Piola stress
 *     of Eq. hypref (the contraction L : Grad du of Eq. L written out):
 *       dP = mu dH + (mu - 2 lambda ln J) F^-T dH^T F^-T + 2 lambda tr(F^-1 dH) F^-T;
 *     the cached strategy (partial assembly, Section 3.2.2) reads F^-1 and ln J per point from
 *     a table built once by sf_cache;
 *   transposed sum factorisation: W_{c,a} = sum_q sum_d dP_{cd} dphi_a/dX_d w_q h^3;
 *   scatter-add into v.
 * Dirichlet DoFs: v = du there (identity rows and columns, as oracle/fem.py).
 *
 * Threads: OpenMP over the elements of one of the eight colour classes at a time (elements
 * (cx + 2 i, cy + 2 j, cz + 2 k)); elements of one class share no node, so the scatter has no
 * races and the result does not depend on the thread count.
 *
 * Layout: vectors [3][M^3], node (i, j, k) -> i + M (j + M k); 1D tables row-major [q][i];
 * cache [E][(p+1)^3][10] in natural element order (F^-1 row-major, then ln J).
 */
#include <math.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NMAX 5
#define N3MAX (NMAX * NMAX * NMAX)

typedef struct {
  int N, p, n, M, bc;
  long long M3;
  double mu, lam, h;
  const double *B, *D, *w;
} problem;

static int constrained(const problem* P, int c, int i, int k) {
  if (P->bc == 1) return i == 0;
  if (P->bc == 2) return k == 0 || (c == 2 && k == P->M - 1);
  return 0;
}

/* out = A applied along direction dir (0 x, 1 y, 2 z) of the n^3 block in (x fastest):
 * out[.., r, ..] = sum_m A(r, m) in[.., m, ..], A(r, m) = A[r n + m], or A[m n + r] if tr.
 * The helpers below are inlined into one copy per degree (see sf_apply), so that n is a
 * compile-time constant there and the loops have fixed trip counts. */
#define INLINE static inline __attribute__((always_inline))
INLINE void pass(const int n, const double* A, int tr, int dir, const double* in, double* out) {
  const int s = dir == 0 ? 1 : (dir == 1 ? n : n * n);   /* stride along the pass */
  const int s1 = dir == 0 ? n : 1, s2 = dir == 2 ? n : n * n;  /* strides of the other two */
  for (int b2 = 0; b2 < n; ++b2)
    for (int b1 = 0; b1 < n; ++b1) {
      const int base = b1 * s1 + b2 * s2;
      for (int r = 0; r < n; ++r) {
        double acc = 0.0;
        for (int m = 0; m < n; ++m) acc += (tr ? A[m * n + r] : A[r * n + m]) * in[base + m * s];
        out[base + r * s] = acc;
      }
    }
}

/* Reference gradient at the Gauss points of one scalar field f (nodal values):
 * g[d][q] = D along d, B along the other two directions. */
INLINE void grad_ref(const problem* P, const int n, const double* f, double g[3][N3MAX]) {
  double xB[N3MAX], xD[N3MAX], yBB[N3MAX], yBD[N3MAX], yDB[N3MAX];
  pass(n, P->B, 0, 0, f, xB);
  pass(n, P->D, 0, 0, f, xD);
  pass(n, P->B, 0, 1, xB, yBB);
  pass(n, P->D, 0, 1, xB, yBD);
  pass(n, P->B, 0, 1, xD, yDB);
  pass(n, P->B, 0, 2, yDB, g[0]);
  pass(n, P->B, 0, 2, yBD, g[1]);
  pass(n, P->D, 0, 2, yBB, g[2]);
}

/* Transposed: out[a] = sum_q sum_d G[d][q] (D along d, B elsewhere)(q, a). */
INLINE void grad_ref_T(const problem* P, const int n, double G[3][N3MAX], double* out) {
  const int n3 = n * n * n;
  double s0[N3MAX], s1[N3MAX], s2[N3MAX], t0[N3MAX], t1[N3MAX], t2[N3MAX], o0[N3MAX], o1[N3MAX];
  pass(n, P->B, 1, 2, G[0], s0);
  pass(n, P->B, 1, 2, G[1], s1);
  pass(n, P->D, 1, 2, G[2], s2);
  pass(n, P->B, 1, 1, s0, t0);
  pass(n, P->D, 1, 1, s1, t1);
  pass(n, P->B, 1, 1, s2, t2);
  for (int t = 0; t < n3; ++t) t1[t] += t2[t];
  pass(n, P->D, 1, 0, t0, o0);
  pass(n, P->B, 1, 0, t1, o1);
  for (int t = 0; t < n3; ++t) out[t] = o0[t] + o1[t];
}

/* F^-1 and ln J of F = I + H (row-major 3x3); returns J. */
INLINE double kinematics(const double H[9], double Fi[9], double* lnJ) {
  double F[9];
  for (int k = 0; k < 9; ++k) F[k] = H[k] + (k % 4 == 0 ? 1.0 : 0.0);
  const double J = F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
                   F[2] * (F[3] * F[7] - F[4] * F[6]);
  Fi[0] = (F[4] * F[8] - F[5] * F[7]) / J;
  Fi[1] = (F[2] * F[7] - F[1] * F[8]) / J;
  Fi[2] = (F[1] * F[5] - F[2] * F[4]) / J;
  Fi[3] = (F[5] * F[6] - F[3] * F[8]) / J;
  Fi[4] = (F[0] * F[8] - F[2] * F[6]) / J;
  Fi[5] = (F[2] * F[3] - F[0] * F[5]) / J;
  Fi[6] = (F[3] * F[7] - F[4] * F[6]) / J;
  Fi[7] = (F[1] * F[6] - F[0] * F[7]) / J;
  Fi[8] = (F[0] * F[4] - F[1] * F[3]) / J;
  *lnJ = J > 0.0 ? log(J) : 0.0;
  return J;
}

/* dP = mu dH + (mu - 2 lambda ln J) F^-T dH^T F^-T + 2 lambda tr(F^-1 dH) F^-T. */
INLINE void linearised_piola(double mu, double lam, const double Fi[9], double lnJ, const double dH[9], double dP[9]) {
  double K[9], Q[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) K[3 * i + j] = Fi[3 * i] * dH[j] + Fi[3 * i + 1] * dH[3 + j] + Fi[3 * i + 2] * dH[6 + j];
  const double trK = K[0] + K[4] + K[8];
  for (int i = 0; i < 3; ++i)   /* Q = K F^-1 = F^-1 dH F^-1, and (F^-T dH^T F^-T)_iJ = Q_Ji */
    for (int j = 0; j < 3; ++j) Q[3 * i + j] = K[3 * i] * Fi[j] + K[3 * i + 1] * Fi[3 + j] + K[3 * i + 2] * Fi[6 + j];
  for (int i = 0; i < 3; ++i)
    for (int J = 0; J < 3; ++J)
      dP[3 * i + J] = mu * dH[3 * i + J] + (mu - 2.0 * lam * lnJ) * Q[3 * J + i] + 2.0 * lam * trK * Fi[3 * J + i];
}

INLINE long long node_of(const problem* P, const int n, int ex, int ey, int ez, int a) {
  const int i = P->p * ex + a % n, j = P->p * ey + (a / n) % n, k = P->p * ez + a / (n * n);
  return i + (long long)P->M * (j + (long long)P->M * k);
}

/* One element's contribution added into v; returns 0, or 1 if det F <= 0 at a point. */
INLINE int element_apply(const problem* P, const int n, int ex, int ey, int ez, const double* u,
                         const double* du, const double* cache, double* v) {
  const int n3 = n * n * n;
  const double invh = 1.0 / P->h, h3 = P->h * P->h * P->h;
  double ue[3][N3MAX], due[3][N3MAX], gu[3][3][N3MAX], gdu[3][3][N3MAX], G[3][3][N3MAX], out[N3MAX];
  int bad = 0;
  for (int a = 0; a < n3; ++a) {
    const long long nd = node_of(P, n, ex, ey, ez, a);
    const int i = P->p * ex + a % n, k = P->p * ez + a / (n * n);
    for (int c = 0; c < 3; ++c) {
      if (!cache) ue[c][a] = u[c * P->M3 + nd];
      due[c][a] = constrained(P, c, i, k) ? 0.0 : du[c * P->M3 + nd];
    }
  }
  for (int c = 0; c < 3; ++c) {
    if (!cache) grad_ref(P, n, ue[c], gu[c]);
    grad_ref(P, n, due[c], gdu[c]);
  }
  const long long e = ex + (long long)P->N * (ey + (long long)P->N * ez);
  for (int q = 0; q < n3; ++q) {
    double Fi[9], lnJ, dH[9], dP[9];
    if (cache) {
      const double* cq = cache + (e * n3 + q) * 10;
      for (int k = 0; k < 9; ++k) Fi[k] = cq[k];
      lnJ = cq[9];
    } else {
      double H[9];
      for (int c = 0; c < 3; ++c)
        for (int d = 0; d < 3; ++d) H[3 * c + d] = gu[c][d][q] * invh;
      if (!(kinematics(H, Fi, &lnJ) > 0.0)) bad = 1;
    }
    for (int c = 0; c < 3; ++c)
      for (int d = 0; d < 3; ++d) dH[3 * c + d] = gdu[c][d][q] * invh;
    linearised_piola(P->mu, P->lam, Fi, lnJ, dH, dP);
    const double wq = P->w[q % n] * P->w[(q / n) % n] * P->w[q / (n * n)] * h3 * invh;
    for (int c = 0; c < 3; ++c)
      for (int d = 0; d < 3; ++d) G[c][d][q] = dP[3 * c + d] * wq;
  }
  for (int c = 0; c < 3; ++c) {
    grad_ref_T(P, n, G[c], out);
    for (int a = 0; a < n3; ++a) v[c * P->M3 + node_of(P, n, ex, ey, ez, a)] += out[a];
  }
  return bad;
}

static void setup(problem* P, int N, int p, double mu, double lam, int bc, const double* B, const double* D,
                  const double* w) {
  P->N = N;
  P->p = p;
  P->n = p + 1;
  P->M = p * N + 1;
  P->M3 = (long long)P->M * P->M * P->M;
  P->bc = bc;
  P->mu = mu;
  P->lam = lam;
  P->h = 1.0 / N;
  P->B = B;
  P->D = D;
  P->w = w;
}

/* Threads an OpenMP parallel region would use (1 without OpenMP). */
int sf_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* v = A(u) du (cache == NULL: on the fly from u; else the cached strategy, u unused).
 * Returns 0, 1 if det F <= 0 at some point, -1 for bad arguments. */
int sf_apply(int N, int p, double mu, double lam, int bc, const double* B, const double* D, const double* w,
             const double* u, const double* du, const double* cache, double* v) {
  if (N < 1 || p < 1 || p > NMAX - 1 || !du || !v || (!u && !cache)) return -1;
  problem P;
  setup(&P, N, p, mu, lam, bc, B, D, w);
  memset(v, 0, sizeof(double) * 3 * P.M3);
  int bad = 0;
  for (int col = 0; col < 8; ++col) {
    const int cx = col & 1, cy = (col >> 1) & 1, cz = col >> 2;
    const int nx = (N - cx + 1) / 2, ny = (N - cy + 1) / 2, nz = (N - cz + 1) / 2;
    const long long cnt = (long long)nx * ny * nz;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (long long t = 0; t < cnt; ++t) {
      const int ex = cx + 2 * (int)(t % nx), ey = cy + 2 * (int)((t / nx) % ny), ez = cz + 2 * (int)(t / ((long long)nx * ny));
      switch (P.n) {  /* one inlined copy of the element routine per degree */
        case 2: bad |= element_apply(&P, 2, ex, ey, ez, u, du, cache, v); break;
        case 3: bad |= element_apply(&P, 3, ex, ey, ez, u, du, cache, v); break;
        case 4: bad |= element_apply(&P, 4, ex, ey, ez, u, du, cache, v); break;
        default: bad |= element_apply(&P, 5, ex, ey, ez, u, du, cache, v); break;
      }
    }
  }
  for (int c = 0; c < 3; ++c)
    for (long long nd = 0; nd < P.M3; ++nd) {
      const int i = (int)(nd % P.M), k = (int)(nd / ((long long)P.M * P.M));
      if (constrained(&P, c, i, k)) v[c * P.M3 + nd] = du[c * P.M3 + nd];
    }
  return bad;
}

/* The cached strategy's table at the linearisation point u: per point F^-1 (9) and ln J.
 * Returns 0, 1 if det F <= 0 at some point, -1 for bad arguments. */
int sf_cache(int N, int p, const double* B, const double* D, const double* u, double* cache) {
  if (N < 1 || p < 1 || p > NMAX - 1 || !u || !cache) return -1;
  problem P;
  setup(&P, N, p, 1.0, 0.0, 0, B, D, NULL);
  const int n = P.n, n3 = n * n * n;
  const long long E = (long long)N * N * N;
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (long long e = 0; e < E; ++e) {
    const int ex = (int)(e % N), ey = (int)((e / N) % N), ez = (int)(e / ((long long)N * N));
    double ue[3][N3MAX], gu[3][3][N3MAX];
    for (int a = 0; a < n3; ++a)
      for (int c = 0; c < 3; ++c) ue[c][a] = u[c * P.M3 + node_of(&P, n, ex, ey, ez, a)];
    for (int c = 0; c < 3; ++c) grad_ref(&P, n, ue[c], gu[c]);
    for (int q = 0; q < n3; ++q) {
      double H[9], lnJ;
      double* cq = cache + (e * n3 + q) * 10;
      for (int c = 0; c < 3; ++c)
        for (int d = 0; d < 3; ++d) H[3 * c + d] = gu[c][d][q] * N;
      if (!(kinematics(H, cq, &lnJ) > 0.0)) bad = 1;
      cq[9] = lnJ;
    }
  }
  return bad;
}
