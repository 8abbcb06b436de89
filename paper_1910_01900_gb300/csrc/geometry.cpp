// Host-side setup of the discretization data (Section 2; Section 4 "geometry
// terms"): the element mapping x(xi), the metric w |det J| J^-1 J^-T at the
// cell Gauss points, the face data (area element, J^-1 n of each side), the
// penalty tau_e, the manufactured right-hand side and the dense coarse
// matrix.  All of it is setup work (Section 3.1 excludes setup cost).
#include <omp.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <stdexcept>

#include "geometry.h"

namespace sipg {

namespace {

inline double det3(const double J[9]) {
  return J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) +
         J[2] * (J[3] * J[7] - J[4] * J[6]);
}
inline void inv3(const double J[9], double det, double Ji[9]) {
  const double id = 1.0 / det;
  Ji[0] = (J[4] * J[8] - J[5] * J[7]) * id;
  Ji[1] = (J[2] * J[7] - J[1] * J[8]) * id;
  Ji[2] = (J[1] * J[5] - J[2] * J[4]) * id;
  Ji[3] = (J[5] * J[6] - J[3] * J[8]) * id;
  Ji[4] = (J[0] * J[8] - J[2] * J[6]) * id;
  Ji[5] = (J[2] * J[3] - J[0] * J[5]) * id;
  Ji[6] = (J[3] * J[7] - J[4] * J[6]) * id;
  Ji[7] = (J[1] * J[6] - J[0] * J[7]) * id;
  Ji[8] = (J[0] * J[4] - J[1] * J[3]) * id;
}

}  // namespace

Mapping::Mapping(const MeshDesc &m) : mesh(m) {
  for (int d = 0; d < 3; ++d) h[d] = (m.hi[d] - m.lo[d]) / m.m[d];
  if (m.deform) {
    // degree-3 mapping support points: the GL nodes of degree 3
    const Rules1D &r = rules(4);
    mnodes = r.gl;
  }
}

std::array<double, 3> Mapping::analytic(const std::array<double, 3> &X) const {
  if (!mesh.deform) return X;
  double s = 1.0;
  for (int j = 0; j < 3; ++j) s *= std::sin(M_PI * (X[j] - mesh.lo[j]) / (mesh.hi[j] - mesh.lo[j]));
  return {X[0] + mesh.amp * s, X[1] + mesh.amp * s, X[2] + mesh.amp * s};
}

void Mapping::cell_ijk(int64_t e, int ijk[3]) const {
  ijk[0] = (int)(e % mesh.m[0]);
  ijk[1] = (int)((e / mesh.m[0]) % mesh.m[1]);
  ijk[2] = (int)(e / ((int64_t)mesh.m[0] * mesh.m[1]));
}

PointTable Mapping::table(const std::vector<std::array<double, 3>> &pts) const {
  PointTable t;
  t.P = (int)pts.size();
  if (!mesh.deform) {
    t.pts = pts;
    return t;
  }
  const int q = (int)mnodes.size(), Q3 = q * q * q;
  t.V.assign((size_t)t.P * Q3, 0);
  t.G.assign((size_t)3 * t.P * Q3, 0);
  for (int p = 0; p < t.P; ++p) {
    std::vector<double> v[3], dv[3];
    for (int d = 0; d < 3; ++d) {
      v[d] = lagrange_values(mnodes, pts[p][d]);
      dv[d] = lagrange_derivs(mnodes, pts[p][d]);
    }
    for (int k = 0; k < q; ++k)
      for (int j = 0; j < q; ++j)
        for (int i = 0; i < q; ++i) {
          const int mm = i + q * (j + q * k);
          t.V[(size_t)p * Q3 + mm] = v[0][i] * v[1][j] * v[2][k];
          t.G[((size_t)0 * t.P + p) * Q3 + mm] = dv[0][i] * v[1][j] * v[2][k];
          t.G[((size_t)1 * t.P + p) * Q3 + mm] = v[0][i] * dv[1][j] * v[2][k];
          t.G[((size_t)2 * t.P + p) * Q3 + mm] = v[0][i] * v[1][j] * dv[2][k];
        }
  }
  t.pts = pts;
  return t;
}

void Mapping::eval(int64_t e, const PointTable &t, double *x, double *J) const {
  int ijk[3];
  cell_ijk(e, ijk);
  if (!mesh.deform) {
    for (int p = 0; p < t.P; ++p) {
      for (int a = 0; a < 3; ++a) {
        if (x) x[p * 3 + a] = mesh.lo[a] + (ijk[a] + t.pts[p][a]) * h[a];
        for (int b = 0; b < 3; ++b) J[p * 9 + a * 3 + b] = (a == b) ? h[a] : 0.0;
      }
    }
    return;
  }
  const int q = (int)mnodes.size(), Q3 = q * q * q;
  std::vector<std::array<double, 3>> Phi(Q3);
  for (int k = 0; k < q; ++k)
    for (int j = 0; j < q; ++j)
      for (int i = 0; i < q; ++i) {
        std::array<double, 3> X = {mesh.lo[0] + (ijk[0] + mnodes[i]) * h[0],
                                   mesh.lo[1] + (ijk[1] + mnodes[j]) * h[1],
                                   mesh.lo[2] + (ijk[2] + mnodes[k]) * h[2]};
        Phi[i + q * (j + q * k)] = analytic(X);
      }
  for (int p = 0; p < t.P; ++p) {
    double xx[3] = {0, 0, 0}, JJ[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    const double *V = &t.V[(size_t)p * Q3];
    const double *G0 = &t.G[((size_t)0 * t.P + p) * Q3];
    const double *G1 = &t.G[((size_t)1 * t.P + p) * Q3];
    const double *G2 = &t.G[((size_t)2 * t.P + p) * Q3];
    for (int mm = 0; mm < Q3; ++mm) {
      for (int a = 0; a < 3; ++a) {
        const double f = Phi[mm][a];
        xx[a] += V[mm] * f;
        JJ[a * 3 + 0] += G0[mm] * f;
        JJ[a * 3 + 1] += G1[mm] * f;
        JJ[a * 3 + 2] += G2[mm] * f;
      }
    }
    if (x)
      for (int a = 0; a < 3; ++a) x[p * 3 + a] = xx[a];
    for (int i = 0; i < 9; ++i) J[p * 9 + i] = JJ[i];
  }
}

static std::vector<std::array<double, 3>> cell_points(const Rules1D &r) {
  const int n = r.n;
  std::vector<std::array<double, 3>> pts(n * n * n);
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) pts[i + n * (j + n * k)] = {r.xq[i], r.xq[j], r.xq[k]};
  return pts;
}

// Face points of the face normal to d; side 0: xi_d = 0, side 1: xi_d = 1.
static std::vector<std::array<double, 3>> face_points(const Rules1D &r, int d, int side) {
  const int n = r.n;
  const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
  std::vector<std::array<double, 3>> pts(n * n);
  for (int b = 0; b < n; ++b)
    for (int a = 0; a < n; ++a) {
      std::array<double, 3> p;
      p[d] = side ? 1.0 : 0.0;
      p[t1] = r.xq[a];
      p[t2] = r.xq[b];
      pts[a + n * b] = p;
    }
  return pts;
}

void cell_geometry(const Mapping &map, int n, std::vector<double> &metric, std::vector<double> &wcart) {
  const Rules1D &r = rules(n);
  const int N3 = n * n * n;
  const MeshDesc &m = map.mesh;
  wcart.assign(3 * N3, 0.0);
  const double vol = map.h[0] * map.h[1] * map.h[2];
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) {
        const int p = i + n * (j + n * k);
        const double w = r.wq[i] * r.wq[j] * r.wq[k];
        for (int d = 0; d < 3; ++d) wcart[d * N3 + p] = w * vol / (map.h[d] * map.h[d]);
      }
  metric.clear();
  if (!m.deform) return;
  const int64_t E = (int64_t)m.m[0] * m.m[1] * m.m[2];
  metric.assign((size_t)E * 6 * N3, 0.0);
  const PointTable t = map.table(cell_points(r));
#pragma omp parallel
  {
    std::vector<double> J((size_t)9 * N3);
#pragma omp for schedule(static)
    for (int64_t e = 0; e < E; ++e) {
      map.eval(e, t, nullptr, J.data());
      double *M = &metric[(size_t)e * 6 * N3];
      for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
          for (int i = 0; i < n; ++i) {
            const int p = i + n * (j + n * k);
            const double *Jp = &J[(size_t)p * 9];
            const double det = det3(Jp);
            double Ji[9];
            inv3(Jp, det, Ji);
            const double jxw = std::fabs(det) * r.wq[i] * r.wq[j] * r.wq[k];
            // G = jxw J^-1 J^-T ; G_ab = jxw sum_c Ji[a][c] Ji[b][c]
            auto G = [&](int a, int b) {
              return jxw * (Ji[a * 3] * Ji[b * 3] + Ji[a * 3 + 1] * Ji[b * 3 + 1] + Ji[a * 3 + 2] * Ji[b * 3 + 2]);
            };
            M[0 * N3 + p] = G(0, 0);
            M[1 * N3 + p] = G(1, 1);
            M[2 * N3 + p] = G(2, 2);
            M[3 * N3 + p] = G(0, 1);
            M[4 * N3 + p] = G(0, 2);
            M[5 * N3 + p] = G(1, 2);
          }
    }
  }
}

void face_geometry(const Mapping &map, int n, std::vector<double> fdA[3], std::vector<double> fc[3],
                   std::vector<double> &fwcart) {
  const Rules1D &r = rules(n);
  const int N2 = n * n;
  const MeshDesc &m = map.mesh;
  fwcart.assign(3 * N2, 0.0);
  for (int d = 0; d < 3; ++d) {
    const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
    for (int b = 0; b < n; ++b)
      for (int a = 0; a < n; ++a) fwcart[d * N2 + a + n * b] = r.wq[a] * r.wq[b] * map.h[t1] * map.h[t2];
  }
  for (int d = 0; d < 3; ++d) {
    fdA[d].clear();
    fc[d].clear();
  }
  if (!m.deform) return;
  for (int d = 0; d < 3; ++d) {
    const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
    const int64_t nfp = (int64_t)m.m[t1] * m.m[t2];
    const int64_t F = (int64_t)(m.m[d] + 1) * nfp;
    fdA[d].assign((size_t)F * N2, 0.0);
    fc[d].assign((size_t)F * 2 * 3 * N2, 0.0);
    const PointTable tL = map.table(face_points(r, d, 1));   // lower cell: xi_d = 1
    const PointTable tU = map.table(face_points(r, d, 0));   // upper cell: xi_d = 0
#pragma omp parallel
    {
      std::vector<double> JL((size_t)9 * N2), JU((size_t)9 * N2);
#pragma omp for schedule(static)
      for (int64_t f = 0; f < F; ++f) {
        const int plane = (int)(f / nfp);
        const int64_t rem = f - (int64_t)plane * nfp;
        const int it1 = (int)(rem % m.m[t1]), it2 = (int)(rem / m.m[t1]);
        int ijk[3];
        ijk[t1] = it1;
        ijk[t2] = it2;
        const bool hasL = plane > 0, hasU = plane < m.m[d];
        int64_t eL = -1, eU = -1;
        if (hasL) {
          ijk[d] = plane - 1;
          eL = ijk[0] + (int64_t)m.m[0] * (ijk[1] + (int64_t)m.m[1] * ijk[2]);
          map.eval(eL, tL, nullptr, JL.data());
        }
        if (hasU) {
          ijk[d] = plane;
          eU = ijk[0] + (int64_t)m.m[0] * (ijk[1] + (int64_t)m.m[1] * ijk[2]);
          map.eval(eU, tU, nullptr, JU.data());
        }
        for (int l = 0; l < N2; ++l) {
          const int a = l % n, b = l / n;
          const double w = r.wq[a] * r.wq[b];
          const double *Jp = hasL ? &JL[(size_t)l * 9] : &JU[(size_t)l * 9];
          const double det = det3(Jp);
          double Ji[9];
          inv3(Jp, det, Ji);
          // J^-T e_d = row d of J^-1
          double raw[3] = {Ji[d * 3 + 0], Ji[d * 3 + 1], Ji[d * 3 + 2]};
          const double nr = std::sqrt(raw[0] * raw[0] + raw[1] * raw[1] + raw[2] * raw[2]);
          const double sgn = hasL ? 1.0 : -1.0;
          double nv[3] = {sgn * raw[0] / nr, sgn * raw[1] / nr, sgn * raw[2] / nr};   // out of L (or U)
          fdA[d][(size_t)f * N2 + l] = std::fabs(det) * nr * w;
          if (hasL) {   // role 0: lower cell, own outward normal = nv
            for (int c = 0; c < 3; ++c)
              fc[d][(((size_t)f * 2 + 0) * 3 + c) * N2 + l] = Ji[c * 3] * nv[0] + Ji[c * 3 + 1] * nv[1] + Ji[c * 3 + 2] * nv[2];
          }
          if (hasU) {   // role 1: upper cell, own outward normal = -nv (interior) or nv (lower boundary)
            const double *Ju = &JU[(size_t)l * 9];
            double Jui[9];
            inv3(Ju, det3(Ju), Jui);
            const double s2 = hasL ? -1.0 : 1.0;
            for (int c = 0; c < 3; ++c)
              fc[d][(((size_t)f * 2 + 1) * 3 + c) * N2 + l] =
                  s2 * (Jui[c * 3] * nv[0] + Jui[c * 3 + 1] * nv[1] + Jui[c * 3 + 2] * nv[2]);
          }
        }
      }
    }
  }
}

void penalty(const Mapping &map, int n, double factor, std::vector<double> &tau) {
  const Rules1D &r = rules(n);
  const MeshDesc &m = map.mesh;
  const int64_t E = (int64_t)m.m[0] * m.m[1] * m.m[2];
  const int N3 = n * n * n, N2 = n * n;
  tau.assign(E, 0.0);
  const PointTable tc = map.table(cell_points(r));
  PointTable tf[3][2];
  for (int d = 0; d < 3; ++d)
    for (int s = 0; s < 2; ++s) tf[d][s] = map.table(face_points(r, d, s));
#pragma omp parallel
  {
    std::vector<double> J((size_t)9 * N3);
#pragma omp for schedule(static)
    for (int64_t e = 0; e < E; ++e) {
      int ijk[3];
      map.cell_ijk(e, ijk);
      map.eval(e, tc, nullptr, J.data());
      double vol = 0;
      for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
          for (int i = 0; i < n; ++i) {
            const int p = i + n * (j + n * k);
            vol += std::fabs(det3(&J[(size_t)p * 9])) * r.wq[i] * r.wq[j] * r.wq[k];
          }
      double a_int = 0, a_bd = 0;
      for (int d = 0; d < 3; ++d)
        for (int s = 0; s < 2; ++s) {
          map.eval(e, tf[d][s], nullptr, J.data());
          double area = 0;
          for (int l = 0; l < N2; ++l) {
            const double *Jp = &J[(size_t)l * 9];
            const double det = det3(Jp);
            double Ji[9];
            inv3(Jp, det, Ji);
            const double nr = std::sqrt(Ji[d * 3] * Ji[d * 3] + Ji[d * 3 + 1] * Ji[d * 3 + 1] + Ji[d * 3 + 2] * Ji[d * 3 + 2]);
            area += std::fabs(det) * nr * r.wq[l % n] * r.wq[l / n];
          }
          const bool bd = s ? (ijk[d] == m.m[d] - 1) : (ijk[d] == 0);
          (bd ? a_bd : a_int) += area;
        }
      tau[e] = factor * (double)n * n * (0.5 * a_int + a_bd) / vol;
    }
  }
}

void manufactured_rhs(const Mapping &map, int n, const std::vector<double> &tau, std::vector<double> &b) {
  const Rules1D &r = rules(n);
  const MeshDesc &m = map.mesh;
  const int64_t E = (int64_t)m.m[0] * m.m[1] * m.m[2];
  const int N3 = n * n * n, N2 = n * n;
  b.assign((size_t)E * N3, 0.0);
  double L[3];
  for (int d = 0; d < 3; ++d) L[d] = m.hi[d] - m.lo[d];
  auto u = [&](const double *x) {
    double s = 1;
    for (int j = 0; j < 3; ++j) s *= std::sin(M_PI * (x[j] - m.lo[j]) / L[j]);
    return s;
  };
  const double lapc = M_PI * M_PI * (1 / (L[0] * L[0]) + 1 / (L[1] * L[1]) + 1 / (L[2] * L[2]));
  const PointTable tc = map.table(cell_points(r));
  PointTable tf[3][2];
  for (int d = 0; d < 3; ++d)
    for (int s = 0; s < 2; ++s) tf[d][s] = map.table(face_points(r, d, s));
  (void)tau;
#pragma omp parallel
  {
    std::vector<double> J((size_t)9 * N3), X((size_t)3 * N3), F(N3);
#pragma omp for schedule(static)
    for (int64_t e = 0; e < E; ++e) {
      int ijk[3];
      map.cell_ijk(e, ijk);
      map.eval(e, tc, X.data(), J.data());
      for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
          for (int i = 0; i < n; ++i) {
            const int p = i + n * (j + n * k);
            F[p] = lapc * u(&X[(size_t)p * 3]) * std::fabs(det3(&J[(size_t)p * 9])) * r.wq[i] * r.wq[j] * r.wq[k];
          }
      double *be = &b[(size_t)e * N3];
      for (int c = 0; c < n; ++c)
        for (int bb = 0; bb < n; ++bb)
          for (int a = 0; a < n; ++a) {
            double s = 0;
            for (int k = 0; k < n; ++k)
              for (int j = 0; j < n; ++j)
                for (int i = 0; i < n; ++i)
                  s += r.S[i * n + a] * r.S[j * n + bb] * r.S[k * n + c] * F[i + n * (j + n * k)];
            be[a + n * (bb + n * c)] = s;
          }
      // Neumann sides: + int N_i h with h = du/dn (u and its tangential
      // derivatives vanish there only on Dirichlet sides; g = u = 0 on the box)
      for (int d = 0; d < 3; ++d)
        for (int s = 0; s < 2; ++s) {
          const bool bd = s ? (ijk[d] == m.m[d] - 1) : (ijk[d] == 0);
          if (!bd || m.bc[2 * d + s] != 1) continue;
          map.eval(e, tf[d][s], X.data(), J.data());
          const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
          for (int l = 0; l < N2; ++l) {
            const double *x = &X[(size_t)l * 3];
            double prod = 1;
            for (int j = 0; j < 3; ++j)
              if (j != d) prod *= std::sin(M_PI * (x[j] - m.lo[j]) / L[j]);
            // du/dx_d at x_d = lo (cos 0 = 1) or hi (cos pi = -1); outward normal -e_d or +e_d
            const double hval = -(M_PI / L[d]) * prod;
            const double *Jp = &J[(size_t)l * 9];
            const double det = det3(Jp);
            double Ji[9];
            inv3(Jp, det, Ji);
            const double nr = std::sqrt(Ji[d * 3] * Ji[d * 3] + Ji[d * 3 + 1] * Ji[d * 3 + 1] + Ji[d * 3 + 2] * Ji[d * 3 + 2]);
            const double dA = std::fabs(det) * nr * r.wq[l % n] * r.wq[l / n];
            const int a = l % n, bq = l / n;
            // face basis: node index along d is 0 (s=0) or n-1 (s=1)
            for (int i2 = 0; i2 < n; ++i2)
              for (int i1 = 0; i1 < n; ++i1) {
                int ii[3];
                ii[d] = s ? n - 1 : 0;
                ii[t1] = i1;
                ii[t2] = i2;
                be[ii[0] + n * (ii[1] + n * ii[2])] += r.S[a * n + i1] * r.S[bq * n + i2] * hval * dA;
              }
          }
        }
    }
  }
}

double l2_error_manufactured(const Mapping &map, int n, const double *x) {
  // || u_h - u ||_L2 with an (n+2)-point Gauss rule per direction; u_h from the
  // nodal values x (DG order), u = prod_j sin(pi (x_j - lo_j) / L_j)
  const MeshDesc &m = map.mesh;
  const int nq = n + 2;
  struct {
    std::vector<double> xq, wq;
  } rq;
  gauss_rule(nq, rq.xq, rq.wq);
  const Rules1D &rn = rules(n);
  std::vector<double> S((size_t)nq * n);
  for (int q = 0; q < nq; ++q) {
    const auto v = lagrange_values(rn.gl, rq.xq[q]);
    for (int i = 0; i < n; ++i) S[(size_t)q * n + i] = v[i];
  }
  std::vector<std::array<double, 3>> pts((size_t)nq * nq * nq);
  for (int k = 0; k < nq; ++k)
    for (int j = 0; j < nq; ++j)
      for (int i = 0; i < nq; ++i) pts[i + nq * (j + nq * k)] = {rq.xq[i], rq.xq[j], rq.xq[k]};
  const PointTable t = map.table(pts);
  const int64_t E = (int64_t)m.m[0] * m.m[1] * m.m[2];
  const int n3 = n * n * n, q3 = nq * nq * nq;
  double L[3];
  for (int d = 0; d < 3; ++d) L[d] = m.hi[d] - m.lo[d];
  double total = 0;
#pragma omp parallel reduction(+ : total)
  {
    std::vector<double> J((size_t)9 * q3), X((size_t)3 * q3), a((size_t)nq * n * n), b((size_t)nq * nq * n);
#pragma omp for schedule(static)
    for (int64_t e = 0; e < E; ++e) {
      map.eval(e, t, X.data(), J.data());
      const double *xe = x + (size_t)e * n3;
      for (int k = 0; k < n; ++k)   // x direction: a[k][j][qx]
        for (int j = 0; j < n; ++j)
          for (int qx = 0; qx < nq; ++qx) {
            double s2 = 0;
            for (int i = 0; i < n; ++i) s2 += S[(size_t)qx * n + i] * xe[i + n * (j + n * k)];
            a[(size_t)(k * n + j) * nq + qx] = s2;
          }
      for (int k = 0; k < n; ++k)   // y direction: b[k][qy][qx]
        for (int qy = 0; qy < nq; ++qy)
          for (int qx = 0; qx < nq; ++qx) {
            double s2 = 0;
            for (int j = 0; j < n; ++j) s2 += S[(size_t)qy * n + j] * a[(size_t)(k * n + j) * nq + qx];
            b[(size_t)(k * nq + qy) * nq + qx] = s2;
          }
      for (int qz = 0; qz < nq; ++qz)
        for (int qy = 0; qy < nq; ++qy)
          for (int qx = 0; qx < nq; ++qx) {
            double uh = 0;
            for (int k = 0; k < n; ++k) uh += S[(size_t)qz * n + k] * b[(size_t)(k * nq + qy) * nq + qx];
            const int p = qx + nq * (qy + nq * qz);
            double u = 1;
            for (int d = 0; d < 3; ++d) u *= std::sin(M_PI * (X[(size_t)p * 3 + d] - m.lo[d]) / L[d]);
            const double w = rq.wq[qx] * rq.wq[qy] * rq.wq[qz] * std::fabs(det3(&J[(size_t)p * 9]));
            total += (uh - u) * (uh - u) * w;
          }
    }
  }
  return std::sqrt(total);
}

namespace {

// Q1 stiffness matrix of cell e with the 2-point Gauss rule and the cell's
// mapping: K[i][j] = sum_q w_q |det J| grad N_i . grad N_j, local node i =
// ix + 2 iy + 4 iz; gidx[i] = its node in the (m+1)^3 grid (x fastest).
void q1_cell_matrix(const Mapping &map, const PointTable &tc, const Rules1D &r, int64_t e, double K[8][8],
                    int gidx[8]) {
  const MeshDesc &m = map.mesh;
  const int grid[3] = {m.m[0] + 1, m.m[1] + 1, m.m[2] + 1};
  double J[9 * 8];
  int ijk[3];
  map.cell_ijk(e, ijk);
  map.eval(e, tc, nullptr, J);
  for (int i = 0; i < 8; ++i)
    for (int j = 0; j < 8; ++j) K[i][j] = 0.0;
  for (int qz = 0; qz < 2; ++qz)
    for (int qy = 0; qy < 2; ++qy)
      for (int qx = 0; qx < 2; ++qx) {
        const int p = qx + 2 * (qy + 2 * qz);
        const double *Jp = &J[p * 9];
        const double det = det3(Jp);
        double Ji[9];
        inv3(Jp, det, Ji);
        const double jxw = std::fabs(det) * r.wq[qx] * r.wq[qy] * r.wq[qz];
        double gr[8][3];
        for (int i = 0; i < 8; ++i) {
          const int ix = i & 1, iy = (i >> 1) & 1, iz = i >> 2;
          const double g0 = r.Sd[qx * 2 + ix] * r.S[qy * 2 + iy] * r.S[qz * 2 + iz];
          const double g1 = r.S[qx * 2 + ix] * r.Sd[qy * 2 + iy] * r.S[qz * 2 + iz];
          const double g2 = r.S[qx * 2 + ix] * r.S[qy * 2 + iy] * r.Sd[qz * 2 + iz];
          for (int a = 0; a < 3; ++a) gr[i][a] = Ji[0 * 3 + a] * g0 + Ji[1 * 3 + a] * g1 + Ji[2 * 3 + a] * g2;
        }
        for (int i = 0; i < 8; ++i)
          for (int j = 0; j < 8; ++j) K[i][j] += jxw * (gr[i][0] * gr[j][0] + gr[i][1] * gr[j][1] + gr[i][2] * gr[j][2]);
      }
  for (int i = 0; i < 8; ++i) {
    const int ix = i & 1, iy = (i >> 1) & 1, iz = i >> 2;
    gidx[i] = (ijk[0] + ix) + grid[0] * ((ijk[1] + iy) + grid[1] * (ijk[2] + iz));
  }
}

// nodes of the (m+1)^3 grid on a Dirichlet side (strongly constrained)
std::vector<char> q1_constrained(const MeshDesc &m, const int bc[6]) {
  const int grid[3] = {m.m[0] + 1, m.m[1] + 1, m.m[2] + 1};
  const int N = grid[0] * grid[1] * grid[2];
  std::vector<char> c(N, 0);
  for (int g = 0; g < N; ++g) {
    const int gx = g % grid[0], gy = (g / grid[0]) % grid[1], gz = g / (grid[0] * grid[1]);
    c[g] = (gx == 0 && bc[0] == 0) || (gx == grid[0] - 1 && bc[1] == 0) || (gy == 0 && bc[2] == 0) ||
           (gy == grid[1] - 1 && bc[3] == 0) || (gz == 0 && bc[4] == 0) || (gz == grid[2] - 1 && bc[5] == 0);
  }
  return c;
}

}  // namespace

void coarse_matrix(const Mapping &map, const int bc[6], std::vector<double> &A, int &N) {
  const MeshDesc &m = map.mesh;
  const int grid[3] = {m.m[0] + 1, m.m[1] + 1, m.m[2] + 1};
  N = grid[0] * grid[1] * grid[2];
  A.assign((size_t)N * N, 0.0);
  const Rules1D &r = rules(2);
  const PointTable tc = map.table(cell_points(r));
  const int64_t E = (int64_t)m.m[0] * m.m[1] * m.m[2];
  for (int64_t e = 0; e < E; ++e) {
    double K[8][8];
    int gidx[8];
    q1_cell_matrix(map, tc, r, e, K, gidx);
    for (int i = 0; i < 8; ++i)
      for (int j = 0; j < 8; ++j) A[(size_t)gidx[i] * N + gidx[j]] += K[i][j];
  }
  const std::vector<char> cons = q1_constrained(m, bc);
  for (int g = 0; g < N; ++g) {
    if (!cons[g]) continue;
    for (int j = 0; j < N; ++j) {
      A[(size_t)g * N + j] = 0;
      A[(size_t)j * N + g] = 0;
    }
    A[(size_t)g * N + g] = 1.0;
  }
}

void coarse_matrix_csr(const Mapping &map, const int bc[6], Csr &A) {
  const MeshDesc &m = map.mesh;
  const int grid[3] = {m.m[0] + 1, m.m[1] + 1, m.m[2] + 1};
  const int N = grid[0] * grid[1] * grid[2];
  const Rules1D &r = rules(2);
  const PointTable tc = map.table(cell_points(r));
  const int64_t E = (int64_t)m.m[0] * m.m[1] * m.m[2];
  const std::vector<char> cons = q1_constrained(m, bc);
  // the 27-point pattern of every node (neighbours within one grid step),
  // columns ascending; values summed cell by cell in cell order
  A.n = N;
  A.ncols = N;
  A.ptr.assign(N + 1, 0);
  auto nb = [&](int g, int d) {   // neighbour offset d = (dx+1) + 3 (dy+1) + 9 (dz+1), -1 if outside
    const int gx = g % grid[0], gy = (g / grid[0]) % grid[1], gz = g / (grid[0] * grid[1]);
    const int x = gx + d % 3 - 1, y = gy + (d / 3) % 3 - 1, z = gz + d / 9 - 1;
    if (x < 0 || y < 0 || z < 0 || x >= grid[0] || y >= grid[1] || z >= grid[2]) return -1;
    return x + grid[0] * (y + grid[1] * z);
  };
  for (int g = 0; g < N; ++g) {
    int cnt = 0;
    if (cons[g]) cnt = 1;
    else
      for (int d = 0; d < 27; ++d) {
        const int h = nb(g, d);
        if (h >= 0 && (h == g || !cons[h])) ++cnt;
      }
    A.ptr[g + 1] = A.ptr[g] + cnt;
  }
  A.idx.assign(A.ptr[N], 0);
  A.val.assign(A.ptr[N], 0.0);
  for (int g = 0; g < N; ++g) {
    int o = A.ptr[g];
    if (cons[g]) {
      A.idx[o] = g;
      A.val[o] = 1.0;
      continue;
    }
    for (int d = 0; d < 27; ++d) {   // d ascending = column ascending
      const int h = nb(g, d);
      if (h >= 0 && (h == g || !cons[h])) A.idx[o++] = h;
    }
  }
  auto slot = [&](int row, int col) -> double * {
    for (int o = A.ptr[row]; o < A.ptr[row + 1]; ++o)
      if (A.idx[o] == col) return &A.val[o];
    return nullptr;
  };
  for (int64_t e = 0; e < E; ++e) {
    double K[8][8];
    int gidx[8];
    q1_cell_matrix(map, tc, r, e, K, gidx);
    for (int i = 0; i < 8; ++i) {
      if (cons[gidx[i]]) continue;
      for (int j = 0; j < 8; ++j) {
        if (cons[gidx[j]]) continue;
        *slot(gidx[i], gidx[j]) += K[i][j];
      }
    }
  }
}

bool cholesky_inverse(std::vector<double> &A, int N) {
  // A = L L^T (L in the lower triangle), then A^-1 = L^-T L^-1
  std::vector<double> Lm(A);
  for (int j = 0; j < N; ++j) {
    double s = Lm[(size_t)j * N + j];
    for (int k = 0; k < j; ++k) s -= Lm[(size_t)j * N + k] * Lm[(size_t)j * N + k];
    if (!(s > 0)) return false;
    const double d = std::sqrt(s);
    Lm[(size_t)j * N + j] = d;
#pragma omp parallel for schedule(static)
    for (int i = j + 1; i < N; ++i) {
      double t = Lm[(size_t)i * N + j];
      for (int k = 0; k < j; ++k) t -= Lm[(size_t)i * N + k] * Lm[(size_t)j * N + k];
      Lm[(size_t)i * N + j] = t / d;
    }
  }
  // W = L^-1 (lower triangular), column by column
  std::vector<double> W((size_t)N * N, 0.0);
#pragma omp parallel for schedule(dynamic)
  for (int c = 0; c < N; ++c) {
    W[(size_t)c * N + c] = 1.0 / Lm[(size_t)c * N + c];
    for (int i = c + 1; i < N; ++i) {
      double t = 0;
      for (int k = c; k < i; ++k) t -= Lm[(size_t)i * N + k] * W[(size_t)k * N + c];
      W[(size_t)i * N + c] = t / Lm[(size_t)i * N + i];
    }
  }
  // A^-1 = W^T W
#pragma omp parallel for schedule(dynamic)
  for (int i = 0; i < N; ++i)
    for (int j = 0; j <= i; ++j) {
      double t = 0;
      for (int k = i; k < N; ++k) t += W[(size_t)k * N + i] * W[(size_t)k * N + j];
      A[(size_t)i * N + j] = t;
      A[(size_t)j * N + i] = t;
    }
  return true;
}

double tridiag_max_eig(const std::vector<double> &diag, const std::vector<double> &off) {
  // Sturm-sequence bisection for the largest eigenvalue of a symmetric tridiagonal
  const int m = (int)diag.size();
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < m; ++i) {
    const double r = (i > 0 ? std::fabs(off[i - 1]) : 0) + (i + 1 < m ? std::fabs(off[i]) : 0);
    lo = std::min(lo, diag[i] - r);
    hi = std::max(hi, diag[i] + r);
  }
  auto count_below = [&](double x) {   // eigenvalues < x
    int c = 0;
    double q = diag[0] - x;
    if (q < 0) ++c;
    for (int i = 1; i < m; ++i) {
      const double qq = (q == 0) ? 1e-300 : q;
      q = diag[i] - x - off[i - 1] * off[i - 1] / qq;
      if (q < 0) ++c;
    }
    return c;
  };
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (count_below(mid) == m) hi = mid;
    else lo = mid;
  }
  return 0.5 * (lo + hi);
}

uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

double uniform_pm1(uint64_t seed, uint64_t i) {
  const uint64_t z = splitmix64(seed ^ i);
  return 2.0 * ((double)(z >> 11) * 0x1.0p-53) - 1.0;
}

}  // namespace sipg
