// 1D rules and tables of the discretization (Section 2): Lagrange basis on the
// Legendre-Gauss-Lobatto nodes, (p+1)-point Gauss-Legendre quadrature, and the
// sum-factorisation matrices built from them (Section 4).
//
// The points are computed by Newton's method on the Legendre recurrence
// (Gauss points: roots of P_n; GL interior nodes: roots of P'_{n-1}), on
// [-1,1] and mapped to the reference interval [0,1].
#include <cmath>
#include <cstring>
#include <mutex>

#include "sipg_internal.h"

namespace sipg {

namespace {

// P_k(x) and P_k'(x) by the three-term recurrence.
void legendre(int k, double x, double &p, double &dp) {
  double p0 = 1.0, p1 = x;
  if (k == 0) {
    p = 1.0;
    dp = 0.0;
    return;
  }
  for (int j = 2; j <= k; ++j) {
    const double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
    p0 = p1;
    p1 = p2;
  }
  p = p1;
  dp = k * (x * p1 - p0) / (x * x - 1.0);
}

std::vector<double> gauss_points(int n, std::vector<double> &w) {
  std::vector<double> x(n);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(n, z, p, dp);
      const double dz = p / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p, dp;
    legendre(n, z, p, dp);
    x[n - 1 - i] = z;
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
  for (int i = 0; i < n; ++i) {   // exact symmetry, then map to [0,1]
    const double xs = 0.5 * (x[i] - x[n - 1 - i]);
    const double ws = 0.5 * (w[i] + w[n - 1 - i]);
    x[i] = xs;
    w[i] = ws;
  }
  for (int i = 0; i < n; ++i) {
    x[i] = 0.5 * (x[i] + 1.0);
    w[i] *= 0.5;
  }
  return x;
}

std::vector<double> gauss_lobatto_points(int n) {
  const int k = n - 1;   // degree; interior nodes are roots of P_k'
  std::vector<double> x(n);
  x[0] = -1.0;
  x[n - 1] = 1.0;
  for (int i = 1; i < n - 1; ++i) {
    double z = -std::cos(M_PI * i / k);
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(k, z, p, dp);
      const double d2p = (2.0 * z * dp - k * (k + 1.0) * p) / (1.0 - z * z);
      const double dz = dp / d2p;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
  }
  std::vector<double> y(n);
  for (int i = 0; i < n; ++i) y[i] = 0.5 * (0.5 * (x[i] - x[n - 1 - i]) + 1.0);
  y[0] = 0.0;
  y[n - 1] = 1.0;
  return y;
}

void fill_rules(Rules1D &r, int n) {
  r.n = n;
  r.gl = gauss_lobatto_points(n);
  r.xq = gauss_points(n, r.wq);
  r.S.assign(n * n, 0);
  r.Sd.assign(n * n, 0);
  r.D.assign(n * n, 0);
  for (int q = 0; q < n; ++q) {
    const auto v = lagrange_values(r.gl, r.xq[q]);
    const auto dv = lagrange_derivs(r.gl, r.xq[q]);
    const auto dG = lagrange_derivs(r.xq, r.xq[q]);
    for (int i = 0; i < n; ++i) {
      r.S[q * n + i] = v[i];
      r.Sd[q * n + i] = dv[i];
      r.D[q * n + i] = dG[i];
    }
  }
  r.l0 = lagrange_values(r.xq, 0.0);
  r.l1 = lagrange_values(r.xq, 1.0);
  r.lp0 = lagrange_derivs(r.gl, 0.0);
  r.lp1 = lagrange_derivs(r.gl, 1.0);
}

// Even-odd blocks of a matrix with M[i][j] = par * M[n-1-i][n-1-j].
void even_odd(const std::vector<double> &M, int n, int par, double *E, double *O) {
  const int h = n / 2, hc = (n + 1) / 2;
  for (int i = 0; i < 25; ++i) E[i] = 0;
  for (int i = 0; i < 20; ++i) O[i] = 0;
  for (int i = 0; i < hc; ++i) {
    for (int j = 0; j < h; ++j) {
      E[i * 5 + j] = 0.5 * (M[i * n + j] + M[i * n + n - 1 - j]);
      O[i * 4 + j] = 0.5 * (M[i * n + j] - M[i * n + n - 1 - j]);
    }
    if (n & 1) E[i * 5 + h] = M[i * n + h];
  }
  (void)par;
}

}  // namespace

void gauss_rule(int n, std::vector<double> &x, std::vector<double> &w) { x = gauss_points(n, w); }

std::vector<double> lagrange_values(const std::vector<double> &nodes, double x) {
  const int n = (int)nodes.size();
  std::vector<double> v(n, 1.0);
  for (int j = 0; j < n; ++j)
    for (int m = 0; m < n; ++m)
      if (m != j) v[j] *= (x - nodes[m]) / (nodes[j] - nodes[m]);
  return v;
}

std::vector<double> lagrange_derivs(const std::vector<double> &nodes, double x) {
  const int n = (int)nodes.size();
  std::vector<double> d(n, 0.0);
  for (int j = 0; j < n; ++j)
    for (int m = 0; m < n; ++m) {
      if (m == j) continue;
      double t = 1.0 / (nodes[j] - nodes[m]);
      for (int r = 0; r < n; ++r)
        if (r != j && r != m) t *= (x - nodes[r]) / (nodes[j] - nodes[r]);
      d[j] += t;
    }
  return d;
}

const Rules1D &rules(int n) {
  static Rules1D table[kMaxN + 1];
  static std::once_flag once;
  std::call_once(once, [] {
    for (int m = 2; m <= kMaxN; ++m) fill_rules(table[m], m);
  });
  return table[n];
}

template <typename T>
void build_tables(Tables<T> &t) {
  std::memset(&t, 0, sizeof(t));
  for (int n = 2; n <= kMaxN; ++n) {
    const Rules1D &r = rules(n);
    std::vector<double> St(n * n), Dt(n * n);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        St[i * n + j] = r.S[j * n + i];
        Dt[i * n + j] = r.D[j * n + i];
      }
    if (n <= 4)
      for (int i = 0; i < n * n; ++i) {
        t.S[n][i] = (T)r.S[i];
        t.St[n][i] = (T)St[i];
        t.D[n][i] = (T)r.D[i];
        t.Dt[n][i] = (T)Dt[i];
      }
    double E[25], O[20];
    auto put = [&](const std::vector<double> &M, int par, T *e, T *o) {
      even_odd(M, n, par, E, O);
      for (int i = 0; i < 25; ++i) e[i] = (T)E[i];
      for (int i = 0; i < 20; ++i) o[i] = (T)O[i];
    };
    put(r.S, +1, t.SE[n], t.SO[n]);
    put(St, +1, t.StE[n], t.StO[n]);
    put(r.D, -1, t.DE[n], t.DO[n]);
    put(Dt, -1, t.DtE[n], t.DtO[n]);
    std::vector<double> M1(n * n, 0.0), K1(n * n, 0.0);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j)
        for (int q = 0; q < n; ++q) {
          M1[i * n + j] += r.wq[q] * r.S[q * n + i] * r.S[q * n + j];
          K1[i * n + j] += r.wq[q] * r.Sd[q * n + i] * r.Sd[q * n + j];
        }
    if (n <= 4)
      for (int i = 0; i < n * n; ++i) {
        t.M1[n][i] = (T)M1[i];
        t.K1[n][i] = (T)K1[i];
      }
    put(M1, +1, t.M1E[n], t.M1O[n]);
    put(K1, +1, t.K1E[n], t.K1O[n]);
    std::vector<double> KG(n * n, 0.0);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j)
        for (int q = 0; q < n; ++q) KG[i * n + j] += r.D[q * n + i] * r.wq[q] * r.D[q * n + j];
    if (n <= 4)
      for (int i = 0; i < n * n; ++i) t.KG[n][i] = (T)KG[i];
    put(KG, +1, t.KGE[n], t.KGO[n]);
    for (int q = 0; q < n; ++q) {
      t.l0[n][q] = (T)r.l0[q];
      t.l1[n][q] = (T)r.l1[q];
      double d0 = 0, d1 = 0;   // (D^T l)[q] = sum_j D[j][q] l[j]
      for (int j = 0; j < n; ++j) {
        d0 += r.D[j * n + q] * r.l0[j];
        d1 += r.D[j * n + q] * r.l1[j];
      }
      t.dl0[n][q] = (T)d0;
      t.dl1[n][q] = (T)d1;
    }
  }
}
template void build_tables<double>(Tables<double> &);
template void build_tables<float>(Tables<float> &);

}  // namespace sipg
