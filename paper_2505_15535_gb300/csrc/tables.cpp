// 1D tables of the Q_p element: GLL nodes, Gauss-Legendre rule, Lagrange basis values and
// derivatives (Section 2.2: Q_p elements; Section 2.4: (p+1)^3 Gauss points per cell).
// Computed in FP64 on the host by Newton iteration on Legendre polynomials.
#include <cmath>

#include "internal.h"

namespace nhmf {
namespace {

// Legendre P_k(t) and P_k'(t) by the three-term recurrence.
void legendre(int k, double t, double* P, double* dP) {
  double p0 = 1.0, p1 = t;
  if (k == 0) { *P = 1.0; *dP = 0.0; return; }
  for (int m = 2; m <= k; ++m) {
    double p2 = ((2 * m - 1) * t * p1 - (m - 1) * p0) / m;
    p0 = p1;
    p1 = p2;
  }
  *P = p1;
  *dP = (std::fabs(t) < 1.0) ? k * (t * p1 - p0) / (t * t - 1.0) : 0.5 * k * (k + 1) * std::pow(t, k + 1);
}

// Gauss-Legendre points/weights on [-1, 1]: roots of P_n, w = 2 / ((1 - t^2) P_n'(t)^2).
void gauss(int n, double* t, double* w) {
  for (int i = 0; i < n; ++i) {
    double x = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(n, x, &P, &dP);
      double dx = P / dP;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    double P, dP;
    legendre(n, x, &P, &dP);
    t[n - 1 - i] = x;
    w[n - 1 - i] = 2.0 / ((1.0 - x * x) * dP * dP);
  }
}

// GLL nodes on [-1, 1]: +-1 and the roots of P_p' (Newton on P_p' with P_p'' from the
// Legendre ODE (1 - t^2) P'' = 2 t P' - p (p + 1) P), started at Chebyshev-Lobatto points.
void gll(int p, double* t) {
  t[0] = -1.0;
  t[p] = 1.0;
  for (int j = 1; j < p; ++j) {
    double x = -std::cos(M_PI * j / p);
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(p, x, &P, &dP);
      double d2P = (2.0 * x * dP - p * (p + 1) * P) / (1.0 - x * x);
      double dx = dP / d2P;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    t[j] = x;
  }
}

double lagrange(const double* z, int n, int i, double x) {
  double v = 1.0;
  for (int j = 0; j < n; ++j)
    if (j != i) v *= (x - z[j]) / (z[i] - z[j]);
  return v;
}

double lagrange_deriv(const double* z, int n, int i, double x) {
  double s = 0.0;
  for (int m = 0; m < n; ++m) {
    if (m == i) continue;
    double v = 1.0 / (z[i] - z[m]);
    for (int j = 0; j < n; ++j)
      if (j != i && j != m) v *= (x - z[j]) / (z[i] - z[j]);
    s += v;
  }
  return s;
}

}  // namespace

void build_tables(int p, Tables1D* T) {
  const int n = p + 1;
  T->n = n;
  double t[kMaxN], w[kMaxN], z[kMaxN];
  gauss(n, t, w);
  gll(p, z);
  for (int i = 0; i < n; ++i) {
    T->xq[i] = 0.5 * (t[i] + 1.0);
    T->w[i] = 0.5 * w[i];
    T->nodes[i] = 0.5 * (z[i] + 1.0);
  }
  for (int q = 0; q < n; ++q)
    for (int i = 0; i < n; ++i) {
      T->B[q][i] = lagrange(T->nodes, n, i, T->xq[q]);
      T->D[q][i] = lagrange_deriv(T->nodes, n, i, T->xq[q]);
      T->Dc[q][i] = lagrange_deriv(T->xq, n, i, T->xq[q]);
    }
}

}  // namespace nhmf
