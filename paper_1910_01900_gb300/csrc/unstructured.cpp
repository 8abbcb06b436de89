// Unstructured hexahedral meshes (Section 2; Section 5.3: the paper's nozzle
// and lung meshes are unstructured hexahedra with Dirichlet and Neumann
// boundary parts): host setup of the DG level's connectivity and geometry.
//
// Cell map: the trilinear interpolant of the cell's 8 vertices (local vertex
// i + 2 j + 4 k at reference corner (i, j, k)); with a deformation, the
// analytic map x + amp prod_j sin(pi (x_j - lo_j)/(hi_j - lo_j)) of that
// image interpolated by the degree-3 tensor Lagrange polynomial on the cell's
// GL(3) points.  Both are held as the 64 degree-3 support values per cell
// (a trilinear map is reproduced exactly at degree 3).
//
// Connectivity: local face f = 2 d + s is the face xi_d = s; two cells are
// neighbours through the face whose four vertex ids they share.  The
// orientation of the shared face is read off those ids: the map from the own
// face corners (c1, c2) (tangential directions t1 < t2) to the neighbour's is
// one of the eight symmetries of the square, coded as bit 0 swap the two
// directions, bit 1 reverse the first, bit 2 reverse the second; Gauss points
// transform by the same symmetry (the 1D Gauss points are symmetric).
//
// Geometry per cell and local face (own side): area element times weights
// dA = |det J| |J^-T e_d| w, own outward unit normal n and J^-1 n; per cell
// the metric w |det J| J^-1 J^-T at the Gauss points and the penalty tau_e of
// Section 2 from the cell's own face areas and volume.
#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <string>
#include <vector>

#include "geometry.h"

namespace sipg {

namespace {

inline double det3u(const double J[9]) {
  return J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) + J[2] * (J[3] * J[7] - J[4] * J[6]);
}

inline void inv3u(const double J[9], double det, double Ji[9]) {
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

// degree-3 basis values and reference gradients at points: V[p][64], G[3][p][64]
struct Q3Table {
  int P = 0;
  std::vector<double> V, G;
};

Q3Table q3_table(const std::vector<double> &gl4, const std::vector<std::array<double, 3>> &pts) {
  Q3Table t;
  t.P = (int)pts.size();
  t.V.assign((size_t)t.P * 64, 0.0);
  t.G.assign((size_t)3 * t.P * 64, 0.0);
  for (int p = 0; p < t.P; ++p) {
    std::vector<double> v[3], dv[3];
    for (int a = 0; a < 3; ++a) {
      v[a] = lagrange_values(gl4, pts[p][a]);
      dv[a] = lagrange_derivs(gl4, pts[p][a]);
    }
    for (int k = 0; k < 4; ++k)
      for (int j = 0; j < 4; ++j)
        for (int i = 0; i < 4; ++i) {
          const int m = i + 4 * (j + 4 * k);
          t.V[(size_t)p * 64 + m] = v[0][i] * v[1][j] * v[2][k];
          t.G[((size_t)0 * t.P + p) * 64 + m] = dv[0][i] * v[1][j] * v[2][k];
          t.G[((size_t)1 * t.P + p) * 64 + m] = v[0][i] * dv[1][j] * v[2][k];
          t.G[((size_t)2 * t.P + p) * 64 + m] = v[0][i] * v[1][j] * dv[2][k];
        }
  }
  return t;
}

// Jacobians J[p][a][b] = dx_a/dxi_b of one cell from its 64 support values X[m][3]
void q3_jacobians(const Q3Table &t, const double *X, double *J) {
  for (int p = 0; p < t.P; ++p) {
    double JJ[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int m = 0; m < 64; ++m)
      for (int b = 0; b < 3; ++b) {
        const double g = t.G[((size_t)b * t.P + p) * 64 + m];
        for (int a = 0; a < 3; ++a) JJ[a * 3 + b] += g * X[m * 3 + a];
      }
    for (int i = 0; i < 9; ++i) J[(size_t)p * 9 + i] = JJ[i];
  }
}

// local vertex at face f's corner (c1, c2) over its tangential directions t1 < t2
int corner_vertex(int f, int c1, int c2) {
  const int d = f / 2, s = f % 2;
  const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
  return (s << d) | (c1 << t1) | (c2 << t2);
}

// the symmetry of the square that code applies to a point (q1, q2) of an n x n grid
void apply_code(int code, int n, int q1, int q2, int &p1, int &p2) {
  int a = (code & 1) ? q2 : q1, b = (code & 1) ? q1 : q2;
  if (code & 2) a = n - 1 - a;
  if (code & 4) b = n - 1 - b;
  p1 = a;
  p2 = b;
}

}  // namespace

bool build_unstructured(const UMeshIn &in, int n, double penalty_factor, UGeometry &g, std::string &err) {
  const int E = in.ncells, NV = in.nverts;
  if (E < 1 || NV < 8 || !in.vertices || !in.cells) {
    err = "unstructured mesh: need vertices (>= 8) and cells (>= 1)";
    return false;
  }
  for (int64_t i = 0; i < (int64_t)E * 8; ++i)
    if (in.cells[i] < 0 || in.cells[i] >= NV) {
      err = "unstructured mesh: vertex id out of range";
      return false;
    }
  if (in.face_bc)
    for (int64_t i = 0; i < (int64_t)E * 6; ++i)
      if (in.face_bc[i] != 0 && in.face_bc[i] != 1) {
        err = "unstructured mesh: face_bc must be 0 (Dirichlet) or 1 (Neumann)";
        return false;
      }
  const Rules1D &r = rules(n);
  const std::vector<double> &gl4 = rules(4).gl;
  const int N2 = n * n, N3 = N2 * n;
  // degree-3 support values of every cell
  std::vector<double> X((size_t)E * 64 * 3);
  for (int e = 0; e < E; ++e)
    for (int k = 0; k < 4; ++k)
      for (int j = 0; j < 4; ++j)
        for (int i = 0; i < 4; ++i) {
          const double xi[3] = {gl4[i], gl4[j], gl4[k]};
          double p[3] = {0, 0, 0};
          for (int v = 0; v < 8; ++v) {
            double w = 1.0;
            for (int a = 0; a < 3; ++a) w *= ((v >> a) & 1) ? xi[a] : 1.0 - xi[a];
            const double *P = &in.vertices[(size_t)in.cells[(size_t)e * 8 + v] * 3];
            for (int a = 0; a < 3; ++a) p[a] += w * P[a];
          }
          if (in.deform) {
            double s = 1.0;
            for (int a = 0; a < 3; ++a) s *= std::sin(M_PI * (p[a] - in.lo[a]) / (in.hi[a] - in.lo[a]));
            for (int a = 0; a < 3; ++a) p[a] += in.amp * s;
          }
          double *o = &X[((size_t)e * 64 + i + 4 * (j + 4 * k)) * 3];
          for (int a = 0; a < 3; ++a) o[a] = p[a];
        }
  // connectivity through sorted vertex quadruples
  std::map<std::array<int, 4>, std::vector<std::pair<int, int>>> faces;
  for (int e = 0; e < E; ++e)
    for (int f = 0; f < 6; ++f) {
      std::array<int, 4> key;
      int q = 0;
      for (int c2 = 0; c2 < 2; ++c2)
        for (int c1 = 0; c1 < 2; ++c1) key[q++] = in.cells[(size_t)e * 8 + corner_vertex(f, c1, c2)];
      std::sort(key.begin(), key.end());
      faces[key].push_back({e, f});
    }
  g.ufn.assign((size_t)E * 6 * 2, 0);
  for (int e = 0; e < E; ++e)
    for (int f = 0; f < 6; ++f) {
      const int bc = in.face_bc ? in.face_bc[(size_t)e * 6 + f] : 0;
      g.ufn[((size_t)e * 6 + f) * 2] = bc == 0 ? -1 : -2;
      g.ufn[((size_t)e * 6 + f) * 2 + 1] = 0;
    }
  for (auto &kv : faces) {
    if (kv.second.size() == 1) continue;
    if (kv.second.size() > 2) {
      err = "unstructured mesh: a face is shared by more than two cells";
      return false;
    }
    for (int side = 0; side < 2; ++side) {
      const int e = kv.second[side].first, f = kv.second[side].second;
      const int en = kv.second[1 - side].first, fn = kv.second[1 - side].second;
      if (e == en) {
        err = "unstructured mesh: a cell shares a face with itself";
        return false;
      }
      // corner map own (c1, c2) -> neighbour corner holding the same vertex id
      int img[2][2][2];
      for (int c2 = 0; c2 < 2; ++c2)
        for (int c1 = 0; c1 < 2; ++c1) {
          const int vid = in.cells[(size_t)e * 8 + corner_vertex(f, c1, c2)];
          bool found = false;
          for (int d2 = 0; d2 < 2 && !found; ++d2)
            for (int d1 = 0; d1 < 2 && !found; ++d1)
              if (in.cells[(size_t)en * 8 + corner_vertex(fn, d1, d2)] == vid) {
                img[c1][c2][0] = d1;
                img[c1][c2][1] = d2;
                found = true;
              }
          if (!found) {
            err = "unstructured mesh: inconsistent face";
            return false;
          }
        }
      int code = -1;
      for (int k = 0; k < 8 && code < 0; ++k) {
        bool ok = true;
        for (int c2 = 0; c2 < 2; ++c2)
          for (int c1 = 0; c1 < 2; ++c1) {
            int p1, p2;
            apply_code(k, 2, c1, c2, p1, p2);
            ok = ok && p1 == img[c1][c2][0] && p2 == img[c1][c2][1];
          }
        if (ok) code = k;
      }
      if (code < 0) {
        err = "unstructured mesh: face corners do not match a symmetry of the square";
        return false;
      }
      g.ufn[((size_t)e * 6 + f) * 2] = en;
      g.ufn[((size_t)e * 6 + f) * 2 + 1] = fn | (code << 3);
    }
  }
  // geometry
  std::vector<std::array<double, 3>> cpts(N3);
  for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
      for (int i = 0; i < n; ++i) cpts[i + n * (j + n * k)] = {r.xq[i], r.xq[j], r.xq[k]};
  const Q3Table tc = q3_table(gl4, cpts);
  std::vector<Q3Table> tf(6);
  for (int f = 0; f < 6; ++f) {
    const int d = f / 2, s = f % 2;
    const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
    std::vector<std::array<double, 3>> fp(N2);
    for (int b = 0; b < n; ++b)
      for (int a = 0; a < n; ++a) {
        std::array<double, 3> p;
        p[d] = (double)s;
        p[t1] = r.xq[a];
        p[t2] = r.xq[b];
        fp[a + n * b] = p;
      }
    tf[f] = q3_table(gl4, fp);
  }
  g.metric.assign((size_t)E * 6 * N3, 0.0);
  g.fdA.assign((size_t)E * 6 * N2, 0.0);
  g.fc.assign((size_t)E * 6 * 3 * N2, 0.0);
  g.tau.assign(E, 0.0);
  bool bad = false;
#pragma omp parallel
  {
    std::vector<double> J((size_t)9 * std::max(N3, N2));
#pragma omp for schedule(static)
    for (int e = 0; e < E; ++e) {
      const double *Xe = &X[(size_t)e * 64 * 3];
      q3_jacobians(tc, Xe, J.data());
      double vol = 0;
      double *M = &g.metric[(size_t)e * 6 * N3];
      for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
          for (int i = 0; i < n; ++i) {
            const int p = i + n * (j + n * k);
            const double *Jp = &J[(size_t)p * 9];
            const double det = det3u(Jp);
            if (!(std::fabs(det) > 0)) bad = true;
            double Ji[9];
            inv3u(Jp, det, Ji);
            const double jxw = std::fabs(det) * r.wq[i] * r.wq[j] * r.wq[k];
            vol += jxw;
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
      double a_int = 0, a_bd = 0;
      for (int f = 0; f < 6; ++f) {
        const int d = f / 2, s = f % 2;
        q3_jacobians(tf[f], Xe, J.data());
        double area = 0;
        for (int l = 0; l < N2; ++l) {
          const double *Jp = &J[(size_t)l * 9];
          const double det = det3u(Jp);
          double Ji[9];
          inv3u(Jp, det, Ji);
          const double sg = s ? 1.0 : -1.0;   // outward reference normal (2 s - 1) e_d
          const double raw[3] = {sg * Ji[d * 3], sg * Ji[d * 3 + 1], sg * Ji[d * 3 + 2]};
          const double nr = std::sqrt(raw[0] * raw[0] + raw[1] * raw[1] + raw[2] * raw[2]);
          const double nv[3] = {raw[0] / nr, raw[1] / nr, raw[2] / nr};
          const double dA = std::fabs(det) * nr * r.wq[l % n] * r.wq[l / n];
          g.fdA[((size_t)e * 6 + f) * N2 + l] = dA;
          for (int b = 0; b < 3; ++b)
            g.fc[(((size_t)e * 6 + f) * 3 + b) * N2 + l] = Ji[b * 3] * nv[0] + Ji[b * 3 + 1] * nv[1] + Ji[b * 3 + 2] * nv[2];
          area += dA;
        }
        if (g.ufn[((size_t)e * 6 + f) * 2] >= 0) a_int += area;
        else a_bd += area;
      }
      g.tau[e] = penalty_factor * (double)n * n * (0.5 * a_int + a_bd) / vol;
    }
  }
  if (bad) {
    err = "unstructured mesh: a cell map is singular at a quadrature point";
    return false;
  }
  return true;
}

}  // namespace sipg
