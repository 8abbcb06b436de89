// Coarse-grid solver: conjugate gradients preconditioned by one V-cycle of a
// smoothed-aggregation algebraic multigrid, to a relative tolerance
// (Section 3.3, "Coarse-grid solver"; the paper uses Trilinos ML with an
// ILU(0) smoother and a direct solve on its last level).
//
// Setup (host, FP64, from the FE_1 matrix of the coarsest mesh in CSR):
//   strength   j != i strong for i when |a_ij| > theta sqrt(a_ii a_jj)
//   aggregates three passes in node order: (1) a free node whose strong
//              neighbours are all free roots an aggregate with them; (2) a
//              free node joins the aggregate (after pass 1) of its strongest
//              aggregated neighbour, the smallest index among couplings
//              within a relative 1e-12 of the largest; (3) a free node roots an
//              aggregate with its free strong neighbours.  Nodes without
//              strong neighbours (the identity rows of Dirichlet nodes) stay
//              out of every aggregate.
//   prolongator P = (I - omega D^-1 A) P~, P~ = 1/sqrt(|aggregate|) on each
//              aggregate's nodes, omega = 4 / (3 max_i sum_j |a_ij| / a_ii)
//   Galerkin   A_c = P^T A P, until the matrix has at most kCoarseMax rows or
//              aggregation stops shrinking it; the last level gets the
//              explicit inverse of its Cholesky factor.
//   smoother   Chebyshev-Jacobi (Algorithm 3, the geometric levels' smoother)
//              of degree 3 before and after the coarse correction, on
//              [cheb_lo, cheb_hi] lambda, lambda from 10 Jacobi-PCG Lanczos
//              steps: the AMG smoothing of the paper's lung runs (Table Lung);
//              its other runs use an ILU(0) sweep, a sequential smoother whose
//              data-parallel counterpart is the polynomial one.
//
// Solve (device, FP64): CG from x = 0 until ||r|| <= rtol ||b|| or maxit
// iterations.  The iteration count is fixed at launch so that the whole solve
// can be captured in the V-cycle's CUDA graph: every kernel of an iteration
// first reads a device flag that the residual-norm reduction sets once the
// tolerance is met, and returns at once when it is set.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <stdexcept>
#include <string>
#include <vector>

#include "geometry.h"
#include "sipg_internal.h"

namespace sipg {

namespace {

constexpr double kTheta = 0.02;
constexpr double kTie = 1e-12;
constexpr int kCoarseMax = 500;
constexpr int kMaxLevels = 10;
constexpr int kEigIters = 10;
constexpr int kSmoothDeg = 3;
constexpr int kRedBlocksA = 64, kRedThreadsA = 256;
constexpr int kRowsPerBlock = 8;   // one warp per row

// ---------------------------------------------------------------- host CSR

void spmv_host(const Csr &A, const double *x, double *y) {
  for (int i = 0; i < A.n; ++i) {
    double s = 0;
    for (int o = A.ptr[i]; o < A.ptr[i + 1]; ++o) s += A.val[o] * x[A.idx[o]];
    y[i] = s;
  }
}

double diag_of(const Csr &A, int i) {
  for (int o = A.ptr[i]; o < A.ptr[i + 1]; ++o)
    if (A.idx[o] == i) return A.val[o];
  return 0.0;
}

// C = A B (rows of A times B, columns ascending)
Csr spgemm(const Csr &A, const Csr &B) {
  Csr C;
  C.n = A.n;
  C.ncols = B.ncols;
  C.ptr.assign(A.n + 1, 0);
  std::vector<double> acc(B.ncols, 0.0);
  std::vector<int> mark(B.ncols, -1), cols;
  for (int i = 0; i < A.n; ++i) {
    cols.clear();
    for (int o = A.ptr[i]; o < A.ptr[i + 1]; ++o) {
      const int k = A.idx[o];
      const double a = A.val[o];
      for (int q = B.ptr[k]; q < B.ptr[k + 1]; ++q) {
        const int j = B.idx[q];
        if (mark[j] != i) {
          mark[j] = i;
          acc[j] = 0.0;
          cols.push_back(j);
        }
        acc[j] += a * B.val[q];
      }
    }
    std::sort(cols.begin(), cols.end());
    for (int j : cols) {
      C.idx.push_back(j);
      C.val.push_back(acc[j]);
    }
    C.ptr[i + 1] = (int)C.idx.size();
  }
  return C;
}

Csr transpose(const Csr &A) {
  Csr T;
  T.n = A.ncols;
  T.ncols = A.n;
  T.ptr.assign(T.n + 1, 0);
  for (int j : A.idx) ++T.ptr[j + 1];
  for (int i = 0; i < T.n; ++i) T.ptr[i + 1] += T.ptr[i];
  T.idx.resize(A.idx.size());
  T.val.resize(A.val.size());
  std::vector<int> fill(T.ptr.begin(), T.ptr.end() - 1);
  for (int i = 0; i < A.n; ++i)   // rows ascending: columns of T come out ascending
    for (int o = A.ptr[i]; o < A.ptr[i + 1]; ++o) {
      const int w = fill[A.idx[o]]++;
      T.idx[w] = i;
      T.val[w] = A.val[o];
    }
  return T;
}

// aggregate of every node (-1: no strong neighbour) and the aggregate count
int aggregate(const Csr &A, std::vector<int> &agg) {
  const int n = A.n;
  std::vector<double> d(n);
  for (int i = 0; i < n; ++i) d[i] = diag_of(A, i);
  // strong neighbours, columns ascending (CSR order), with |a_ij|
  std::vector<int> sptr(n + 1, 0), sidx;
  std::vector<double> sw;
  for (int i = 0; i < n; ++i) {
    for (int o = A.ptr[i]; o < A.ptr[i + 1]; ++o) {
      const int j = A.idx[o];
      if (j == i) continue;
      const double a = std::fabs(A.val[o]);
      if (a > kTheta * std::sqrt(std::fabs(d[i] * d[j]))) {
        sidx.push_back(j);
        sw.push_back(a);
      }
    }
    sptr[i + 1] = (int)sidx.size();
  }
  agg.assign(n, -1);
  int na = 0;
  auto isolated = [&](int i) { return sptr[i] == sptr[i + 1]; };
  for (int i = 0; i < n; ++i) {   // pass 1
    if (isolated(i) || agg[i] >= 0) continue;
    bool free = true;
    for (int o = sptr[i]; o < sptr[i + 1] && free; ++o) free = agg[sidx[o]] < 0;
    if (!free) continue;
    agg[i] = na;
    for (int o = sptr[i]; o < sptr[i + 1]; ++o) agg[sidx[o]] = na;
    ++na;
  }
  const std::vector<int> after1(agg);
  for (int i = 0; i < n; ++i) {   // pass 2, against the pass-1 aggregates
    if (isolated(i) || after1[i] >= 0) continue;
    double top = -1;
    for (int o = sptr[i]; o < sptr[i + 1]; ++o)
      if (after1[sidx[o]] >= 0) top = std::max(top, sw[o]);
    if (top < 0) continue;
    for (int o = sptr[i]; o < sptr[i + 1]; ++o)
      if (after1[sidx[o]] >= 0 && sw[o] >= top * (1.0 - kTie)) {
        agg[i] = after1[sidx[o]];
        break;
      }
  }
  for (int i = 0; i < n; ++i) {   // pass 3
    if (isolated(i) || agg[i] >= 0) continue;
    agg[i] = na;
    for (int o = sptr[i]; o < sptr[i + 1]; ++o)
      if (agg[sidx[o]] < 0) agg[sidx[o]] = na;
    ++na;
  }
  return na;
}

// P = (I - omega D^-1 A) P~ (the smoothed prolongator)
Csr smoothed_prolongator(const Csr &A, const std::vector<int> &agg, int na) {
  const int n = A.n;
  std::vector<int> size(na, 0);
  for (int a : agg)
    if (a >= 0) ++size[a];
  Csr Pt;
  Pt.n = n;
  Pt.ncols = na;
  Pt.ptr.assign(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    if (agg[i] >= 0) {
      Pt.idx.push_back(agg[i]);
      Pt.val.push_back(1.0 / std::sqrt((double)size[agg[i]]));
    }
    Pt.ptr[i + 1] = (int)Pt.idx.size();
  }
  std::vector<double> dinv(n);
  double rho = 0;
  for (int i = 0; i < n; ++i) {
    dinv[i] = 1.0 / diag_of(A, i);
    double s = 0;
    for (int o = A.ptr[i]; o < A.ptr[i + 1]; ++o) s += std::fabs(A.val[o]);
    rho = std::max(rho, s * std::fabs(dinv[i]));
  }
  const double omega = 4.0 / (3.0 * rho);
  Csr AP = spgemm(A, Pt);
  Csr P;
  P.n = n;
  P.ncols = na;
  P.ptr.assign(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    const double f = omega * dinv[i];
    int q = Pt.ptr[i];   // at most one tentative entry per row
    for (int o = AP.ptr[i]; o < AP.ptr[i + 1]; ++o) {
      const int j = AP.idx[o];
      double v = -f * AP.val[o];
      if (q < Pt.ptr[i + 1] && Pt.idx[q] == j) {
        v += Pt.val[q];
        ++q;
      }
      P.idx.push_back(j);
      P.val.push_back(v);
    }
    if (q < Pt.ptr[i + 1]) {   // a tentative entry outside A P's pattern (not for a connected node)
      P.idx.push_back(Pt.idx[q]);
      P.val.push_back(Pt.val[q]);
      std::vector<std::pair<int, double>> row;
      for (int o = P.ptr[i]; o < (int)P.idx.size(); ++o) row.push_back({P.idx[o], P.val[o]});
      std::sort(row.begin(), row.end());
      for (size_t t = 0; t < row.size(); ++t) {
        P.idx[P.ptr[i] + t] = row[t].first;
        P.val[P.ptr[i] + t] = row[t].second;
      }
    }
    P.ptr[i + 1] = (int)P.idx.size();
  }
  return P;
}

// lambda_max of D^-1 A: 10 Jacobi-PCG steps from SplitMix64 uniform(-1,1)
// values (seed 1910), the Lanczos tridiagonal of the CG coefficients
double estimate_lambda_host(const Csr &A) {
  const int n = A.n;
  std::vector<double> r(n), z(n), p(n), Ap(n), dinv(n);
  for (int i = 0; i < n; ++i) {
    r[i] = uniform_pm1(1910, (uint64_t)i);
    dinv[i] = 1.0 / diag_of(A, i);
    z[i] = dinv[i] * r[i];
    p[i] = z[i];
  }
  auto dot = [&](const std::vector<double> &a, const std::vector<double> &b) {
    double s = 0;
    for (int i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
  };
  double rz = dot(r, z);
  const double rz0 = rz;
  std::vector<double> alphas, betas;
  for (int it = 0; it < kEigIters; ++it) {
    spmv_host(A, p.data(), Ap.data());
    const double alpha = rz / dot(p, Ap);
    for (int i = 0; i < n; ++i) {
      r[i] -= alpha * Ap[i];
      z[i] = dinv[i] * r[i];
    }
    const double rz_new = dot(r, z);
    alphas.push_back(alpha);
    if (!(rz_new > 1e-28 * rz0)) break;
    const double beta = rz_new / rz;
    betas.push_back(beta);
    for (int i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    rz = rz_new;
  }
  const int m = (int)alphas.size();
  std::vector<double> dg(m), off(m > 1 ? m - 1 : 0);
  for (int j = 0; j < m; ++j) {
    dg[j] = 1.0 / alphas[j] + (j > 0 ? betas[j - 1] / alphas[j - 1] : 0.0);
    if (j + 1 < m) off[j] = std::sqrt(betas[j]) / alphas[j];
  }
  return tridiag_max_eig(dg, off);
}

// ---------------------------------------------------------------- device

struct DevCsr {
  int n = 0;
  int *ptr = nullptr, *idx = nullptr;
  double *val = nullptr;
};

__device__ __forceinline__ bool stopped(const int *done) { return done && *done; }

// One warp per row: y = (A x)_i, then by mode
//   0: out = y                 2: out = b - y
//   1: out = c3 dinv (b - y) + c1 x + c2 xp  (a Chebyshev step, A square)
//   3: out = b + y             (prolongation added to b; out may alias b)
__global__ void csr_kernel(const int *__restrict__ ptr, const int *__restrict__ idx, const double *__restrict__ val,
                           int n, const double *x, const double *b, const double *xp, const double *dinv, double c1,
                           double c2, double c3, int mode, double *out, const int *done) {
  if (stopped(done)) return;
  const int row = blockIdx.x * kRowsPerBlock + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= n) return;
  double s = 0;
  for (int o = ptr[row] + lane; o < ptr[row + 1]; o += 32) s = fma(val[o], x[idx[o]], s);
#pragma unroll
  for (int w = 16; w > 0; w >>= 1) s += __shfl_xor_sync(0xffffffffu, s, w);
  if (lane != 0) return;
  double z;
  if (mode == 0) z = s;
  else if (mode == 2) z = b[row] - s;
  else if (mode == 3) z = b[row] + s;
  else {
    z = c3 * dinv[row] * (b[row] - s);
    z = fma(c1, x[row], z);
    if (xp) z = fma(c2, xp[row], z);
  }
  out[row] = z;
}

// x = c dinv b (the first Chebyshev step from x = 0)
__global__ void amg_xdb_kernel(double *x, double c, const double *dinv, const double *b, int n, const int *done) {
  if (stopped(done)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = c * dinv[i] * b[i];
}

// x = Ainv b on the last level (one warp per row)
__global__ void amg_gemv_kernel(const double *__restrict__ Ainv, const double *__restrict__ b, double *x, int n,
                                const int *done) {
  if (stopped(done)) return;
  const int row = blockIdx.x * kRowsPerBlock + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= n) return;
  double s = 0;
  for (int j = lane; j < n; j += 32) s = fma(Ainv[(size_t)row * n + j], b[j], s);
#pragma unroll
  for (int w = 16; w > 0; w >>= 1) s += __shfl_xor_sync(0xffffffffu, s, w);
  if (lane == 0) x[row] = s;
}

// Two-stage deterministic reduction (fixed grid, the last block sums the
// partials in block order).  Scalar slots sc[]: 0 ||b||^2, 1 r.z (new),
// 2 r.z (old), 3 p.q, 4 r.r; flag[0] = done, flag[1] = iterations taken.
__device__ void amg_reduce(double a, double *partials, unsigned *counter, double *out, int op, double *sc, int *flag,
                           double rtol2) {
  __shared__ double sh[kRedThreadsA];
  __shared__ bool last;
  sh[threadIdx.x] = a;
  __syncthreads();
  for (int w = kRedThreadsA / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = sh[0];
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s = 0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += kRedThreadsA) s += ((volatile double *)partials)[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = kRedThreadsA / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *out = sh[0];
    if (op == 1) flag[0] = !(sh[0] > 0);                          // ||b|| = 0: nothing to do
    if (op == 2) {                                                 // after an update: converged?
      flag[1] += 1;
      if (sh[0] <= rtol2 * sc[0]) flag[0] = 1;
    }
    *counter = 0;
  }
}

// op 1: x = 0, r = b, ||b||^2 -> sc[0]; flag = (b == 0), iterations = 0
__global__ void amg_init_kernel(double *x, double *r, const double *b, int n, double *partials, unsigned *counter,
                                double *sc, int *flag) {
  if (blockIdx.x == 0 && threadIdx.x == 0) flag[1] = 0;
  double a = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    x[i] = 0.0;
    r[i] = b[i];
    a = fma(b[i], b[i], a);
  }
  amg_reduce(a, partials, counter, sc + 0, 1, sc, flag, 0.0);
}

// dot x.y -> *out (skipped once converged)
__global__ void amg_dot_kernel(const double *x, const double *y, int n, double *partials, unsigned *counter,
                               double *out, double *sc, int *flag) {
  if (flag[0]) return;
  double a = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a = fma(x[i], y[i], a);
  amg_reduce(a, partials, counter, out, 0, sc, flag, 0.0);
}

// p = z + beta p, beta = rz_new / rz_old (p = z on the first iteration)
__global__ void amg_update_p_kernel(double *p, const double *z, int n, const double *sc, int first, const int *flag) {
  if (flag[0]) return;
  const double beta = first ? 0.0 : sc[1] / sc[2];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    p[i] = first ? z[i] : fma(beta, p[i], z[i]);
}

// x += alpha p, r -= alpha q (alpha = rz / pq), ||r||^2 -> sc[4], the
// convergence flag and the iteration count; rz moves to the "old" slot
__global__ void amg_update_xr_kernel(double *x, double *r, const double *p, const double *q, int n, double *partials,
                                     unsigned *counter, double *sc, int *flag, double rtol2) {
  if (flag[0]) return;
  const double alpha = sc[3] > 0 ? sc[1] / sc[3] : 0.0;
  double a = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = fma(-alpha, q[i], r[i]);
    r[i] = ri;
    a = fma(ri, ri, a);
  }
  amg_reduce(a, partials, counter, sc + 4, 2, sc, flag, rtol2);
}

__global__ void amg_shift_kernel(double *sc, const int *flag) {
  if (flag[0]) return;
  sc[2] = sc[1];
}

__global__ void amg_copy_kernel(double *dst, const double *src, int n, const int *flag) {
  if (flag[0]) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[i];
}

template <typename T>
T *dcopy(const std::vector<T> &h) {
  T *d = nullptr;
  if (h.empty()) return nullptr;
  if (cudaMalloc(&d, h.size() * sizeof(T)) != cudaSuccess) throw std::runtime_error("cudaMalloc failed (AMG setup)");
  if (cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
    throw std::runtime_error("cudaMemcpy failed (AMG setup)");
  return d;
}

template <typename T>
T *dzeros(size_t n) {
  T *d = nullptr;
  if (cudaMalloc(&d, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess)
    throw std::runtime_error("cudaMalloc failed (AMG setup)");
  cudaMemset(d, 0, std::max<size_t>(n, 1) * sizeof(T));
  return d;
}

DevCsr upload(const Csr &A) {
  DevCsr d;
  d.n = A.n;
  d.ptr = dcopy(A.ptr);
  d.idx = dcopy(A.idx);
  d.val = dcopy(A.val);
  return d;
}

}  // namespace

struct AmgCoarse {
  struct Lev {
    int n = 0, nc = 0;
    DevCsr A, P, R;
    double *dinv = nullptr, *b = nullptr, *x = nullptr, *xt = nullptr, *r = nullptr;
    double lam = 0;
  };
  std::vector<Lev> lv;
  int nlast = 0;
  double *Ainv = nullptr;
  double rtol = 1e-3, cheb_lo = 0.06, cheb_hi = 1.2;
  int maxit = 10;
  double *cr = nullptr, *cp = nullptr, *cq = nullptr;   // CG vectors (residual, direction, A p)
  double *sc = nullptr, *partials = nullptr;
  unsigned *counter = nullptr;
  int *flag = nullptr;
  std::vector<void *> owned;
};

namespace {

void launch_csr(const DevCsr &A, const double *x, const double *b, const double *xp, const double *dinv, double c1,
                double c2, double c3, int mode, double *out, const int *done, cudaStream_t s) {
  if (A.n == 0) return;
  csr_kernel<<<(A.n + kRowsPerBlock - 1) / kRowsPerBlock, 32 * kRowsPerBlock, 0, s>>>(
      A.ptr, A.idx, A.val, A.n, x, b, xp, dinv, c1, c2, c3, mode, out, done);
  note_launch();
}

// Chebyshev (Algorithm 3) on level l: from x = 0 (zero_start) or from the
// current x; the result ends in *x (buffers swapped as the steps proceed)
void amg_chebyshev(AmgCoarse &M, int l, double *&x, double *&xt, bool zero_start, const int *done, cudaStream_t s) {
  AmgCoarse::Lev &L = M.lv[l];
  const double lhi = M.cheb_hi * L.lam, llo = M.cheb_lo * L.lam;
  const double theta = 0.5 * (lhi + llo), delta = 0.5 * (lhi - llo);
  bool have_prev;
  if (zero_start) {
    amg_xdb_kernel<<<(L.n + 255) / 256, 256, 0, s>>>(x, 1.0 / theta, L.dinv, L.b, L.n, done);
    note_launch();
    have_prev = false;
  } else {
    launch_csr(L.A, x, L.b, nullptr, L.dinv, 1.0, 0.0, 1.0 / theta, 1, xt, done, s);
    std::swap(x, xt);
    have_prev = true;
  }
  double rho_prev = delta / theta;
  for (int j = 1; j < kSmoothDeg; ++j) {
    const double rho = 1.0 / (2.0 * theta / delta - rho_prev);
    const double sigma = rho * rho_prev, th = 2.0 * rho / delta;
    launch_csr(L.A, x, L.b, have_prev ? xt : nullptr, L.dinv, 1.0 + sigma, -sigma, th, 1, xt, done, s);
    std::swap(x, xt);
    have_prev = true;
    rho_prev = rho;
  }
}

// one V-cycle from x = 0 on level l with right-hand side lv[l].b; returns x
double *amg_cycle(AmgCoarse &M, int l, const int *done, cudaStream_t s) {
  AmgCoarse::Lev &L = M.lv[l];
  if (l == (int)M.lv.size() - 1) {
    amg_gemv_kernel<<<(L.n + kRowsPerBlock - 1) / kRowsPerBlock, 32 * kRowsPerBlock, 0, s>>>(M.Ainv, L.b, L.x, L.n,
                                                                                             done);
    note_launch();
    return L.x;
  }
  double *x = L.x, *xt = L.xt;
  amg_chebyshev(M, l, x, xt, true, done, s);
  launch_csr(L.A, x, L.b, nullptr, nullptr, 0, 0, 0, 2, L.r, done, s);
  launch_csr(L.R, L.r, nullptr, nullptr, nullptr, 0, 0, 0, 0, M.lv[l + 1].b, done, s);
  const double *xc = amg_cycle(M, l + 1, done, s);
  launch_csr(L.P, xc, x, nullptr, nullptr, 0, 0, 0, 3, x, done, s);
  amg_chebyshev(M, l, x, xt, false, done, s);
  return x;
}

}  // namespace

AmgCoarse *amg_create(const Csr &A0, double rtol, int maxit, double cheb_lo, double cheb_hi, std::string *err) {
  AmgCoarse *M = new AmgCoarse();
  try {
    M->rtol = rtol;
    M->maxit = maxit;
    M->cheb_lo = cheb_lo;
    M->cheb_hi = cheb_hi;
    std::vector<Csr> As{A0}, Ps, Rs;
    while (As.back().n > kCoarseMax && (int)As.size() < kMaxLevels) {
      std::vector<int> agg;
      const int na = aggregate(As.back(), agg);
      if (na == 0 || na >= As.back().n / 1.5) break;
      Csr P = smoothed_prolongator(As.back(), agg, na);
      Csr R = transpose(P);
      Csr Ac = spgemm(R, spgemm(As.back(), P));
      Ps.push_back(P);
      Rs.push_back(R);
      As.push_back(Ac);
    }
    const int nl = (int)As.size();
    M->lv.resize(nl);
    for (int l = 0; l < nl; ++l) {
      AmgCoarse::Lev &L = M->lv[l];
      const Csr &A = As[l];
      L.n = A.n;
      std::vector<double> dinv(A.n);
      for (int i = 0; i < A.n; ++i) dinv[i] = 1.0 / diag_of(A, i);
      L.b = dzeros<double>(A.n);
      L.x = dzeros<double>(A.n);
      if (l + 1 < nl) {
        L.A = upload(A);
        L.P = upload(Ps[l]);
        L.R = upload(Rs[l]);
        L.nc = Ps[l].ncols;
        L.dinv = dcopy(dinv);
        L.xt = dzeros<double>(A.n);
        L.r = dzeros<double>(A.n);
        L.lam = estimate_lambda_host(A);
      }
    }
    // the last level: the explicit inverse from its Cholesky factor
    const Csr &Al = As.back();
    const int N = Al.n;
    std::vector<double> D((size_t)N * N, 0.0);
    for (int i = 0; i < N; ++i)
      for (int o = Al.ptr[i]; o < Al.ptr[i + 1]; ++o) D[(size_t)i * N + Al.idx[o]] = Al.val[o];
    if (!cholesky_inverse(D, N)) throw std::runtime_error("AMG: last-level matrix is not positive definite");
    M->nlast = N;
    M->Ainv = dcopy(D);
    const int n0 = A0.n;
    M->cr = dzeros<double>(n0);
    M->cp = dzeros<double>(n0);
    M->cq = dzeros<double>(n0);
    M->sc = dzeros<double>(8);
    M->partials = dzeros<double>(kRedBlocksA);
    M->counter = dzeros<unsigned>(1);
    M->flag = dzeros<int>(2);
  } catch (std::exception &e) {
    if (err) *err = e.what();
    amg_destroy(M);
    return nullptr;
  }
  return M;
}

void amg_destroy(AmgCoarse *M) {
  if (!M) return;
  auto f = [](void *p) {
    if (p) cudaFree(p);
  };
  for (auto &L : M->lv) {
    for (DevCsr *c : {&L.A, &L.P, &L.R}) {
      f(c->ptr);
      f(c->idx);
      f(c->val);
    }
    f(L.dinv);
    f(L.b);
    f(L.x);
    f(L.xt);
    f(L.r);
  }
  f(M->Ainv);
  f(M->cr);
  f(M->cp);
  f(M->cq);
  f(M->sc);
  f(M->partials);
  f(M->counter);
  f(M->flag);
  delete M;
}

int amg_level_sizes(const AmgCoarse *M, int *sizes, int max) {
  const int nl = (int)M->lv.size();
  for (int l = 0; l < nl && l < max; ++l) sizes[l] = M->lv[l].n;
  return nl;
}

cudaError_t amg_vcycle(AmgCoarse *M, const double *b, double *x, cudaStream_t s) {
  AmgCoarse::Lev &L0 = M->lv[0];
  cudaMemcpyAsync(L0.b, b, L0.n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  const double *z = amg_cycle(*M, 0, nullptr, s);
  cudaMemcpyAsync(x, z, L0.n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  return cudaGetLastError();
}

// CG (Algorithm 1) preconditioned by one V-cycle, from x = 0, until ||r|| <=
// rtol ||b|| (or maxit iterations); b and x are FP64 device vectors of n0.
cudaError_t amg_solve(AmgCoarse *M, const double *b, double *x, cudaStream_t s) {
  AmgCoarse::Lev &L0 = M->lv[0];
  const int n = L0.n;
  const double rtol2 = M->rtol * M->rtol;
  int *flag = M->flag;
  double *sc = M->sc;
  const int gb = (n + 255) / 256, gr = std::min(kRedBlocksA, gb);
  amg_init_kernel<<<gr, kRedThreadsA, 0, s>>>(x, M->cr, b, n, M->partials, M->counter, sc, flag);
  note_launch();
  for (int it = 0; it < M->maxit; ++it) {
    amg_copy_kernel<<<gb, 256, 0, s>>>(L0.b, M->cr, n, flag);   // the cycle's right-hand side
    note_launch();
    const double *z = amg_cycle(*M, 0, flag, s);
    amg_dot_kernel<<<gr, kRedThreadsA, 0, s>>>(M->cr, z, n, M->partials, M->counter, sc + 1, sc, flag);
    note_launch();
    amg_update_p_kernel<<<gb, 256, 0, s>>>(M->cp, z, n, sc, it == 0, flag);
    note_launch();
    launch_csr(L0.A, M->cp, nullptr, nullptr, nullptr, 0, 0, 0, 0, M->cq, flag, s);
    amg_dot_kernel<<<gr, kRedThreadsA, 0, s>>>(M->cp, M->cq, n, M->partials, M->counter, sc + 3, sc, flag);
    note_launch();
    amg_update_xr_kernel<<<gr, kRedThreadsA, 0, s>>>(x, M->cr, M->cp, M->cq, n, M->partials, M->counter, sc, flag,
                                                     rtol2);
    note_launch();
    amg_shift_kernel<<<1, 1, 0, s>>>(sc, flag);
    note_launch();
  }
  return cudaGetLastError();
}

cudaError_t amg_last_iterations(AmgCoarse *M, int *iterations, cudaStream_t s) {
  int h[2] = {0, 0};
  cudaError_t e = cudaMemcpyAsync(h, M->flag, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  *iterations = h[1];
  return e;
}

}  // namespace sipg
