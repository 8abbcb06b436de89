// Host-side setup of the discretization data; see geometry.cpp.
#pragma once
#include <array>
#include <string>
#include <vector>

#include "sipg_internal.h"

namespace sipg {

struct MeshDesc {
  int m[3];
  double lo[3], hi[3];
  int deform;
  double amp;
  int bc[6];
};

// Reference points and, for curved cells, the mapping basis evaluated there.
struct PointTable {
  int P = 0;
  std::vector<std::array<double, 3>> pts;
  std::vector<double> V, G;   // [P][64], [3][P][64]
};

// x(xi) of every cell: affine, or the degree-3 tensor Lagrange interpolant of
// the analytic deformation on the cell's GL(3) points.
struct Mapping {
  MeshDesc mesh;
  double h[3];
  std::vector<double> mnodes;
  explicit Mapping(const MeshDesc &m);
  std::array<double, 3> analytic(const std::array<double, 3> &X) const;
  void cell_ijk(int64_t e, int ijk[3]) const;
  PointTable table(const std::vector<std::array<double, 3>> &pts) const;
  // physical points x[P][3] (may be null) and Jacobians J[P][3][3] = dx_a/dxi_b
  void eval(int64_t e, const PointTable &t, double *x, double *J) const;
};

void cell_geometry(const Mapping &map, int n, std::vector<double> &metric, std::vector<double> &wcart);
void face_geometry(const Mapping &map, int n, std::vector<double> fdA[3], std::vector<double> fc[3],
                   std::vector<double> &fwcart);
void penalty(const Mapping &map, int n, double factor, std::vector<double> &tau);
void manufactured_rhs(const Mapping &map, int n, const std::vector<double> &tau, std::vector<double> &b);
double l2_error_manufactured(const Mapping &map, int n, const double *x_host);
void coarse_matrix(const Mapping &map, const int bc[6], std::vector<double> &A, int &N);

// Compressed sparse rows (columns ascending within a row), FP64.
struct Csr {
  int n = 0, ncols = 0;
  std::vector<int> ptr, idx;
  std::vector<double> val;
};
// The same FE_1 matrix as coarse_matrix in CSR: the 27-point pattern, constrained
// rows identity and constrained columns left out.
void coarse_matrix_csr(const Mapping &map, const int bc[6], Csr &A);
bool cholesky_inverse(std::vector<double> &A, int N);

// Unstructured hexahedral mesh (host arrays; see unstructured.cpp).
struct UMeshIn {
  int nverts = 0, ncells = 0;
  const double *vertices = nullptr;   // [nverts][3]
  const int *cells = nullptr;         // [ncells][8], local vertex i + 2 j + 4 k at corner (i, j, k)
  const int *face_bc = nullptr;       // [ncells][6] or null (all Dirichlet)
  int deform = 0;
  double amp = 0.1, lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
};
// DG-level data of an unstructured mesh: metric [cell][6][n^3], fdA
// [cell][6][n^2], fc [cell][6][3][n^2], tau [cell], ufn [cell][6][2] (see
// DGArgs::ufn).
struct UGeometry {
  std::vector<double> metric, fdA, fc, tau;
  std::vector<int> ufn;
};
bool build_unstructured(const UMeshIn &in, int n, double penalty_factor, UGeometry &g, std::string &err);
double tridiag_max_eig(const std::vector<double> &diag, const std::vector<double> &off);
uint64_t splitmix64(uint64_t x);
double uniform_pm1(uint64_t seed, uint64_t i);

}  // namespace sipg
