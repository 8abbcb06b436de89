// Continuous FE levels of the cph hierarchy (Section 2, Eq. WeakFormFE;
// Section 3.2 transfers), both precisions.
//
// FE operator: a cell pass evaluates (grad v, grad u) on every cell by sum
// factorisation (same interpolation/derivative sweeps as the DG cell term)
// after gathering the cell's nodes from the global grid (constrained
// Dirichlet nodes read as zero), and writes the cell-local result into an
// element buffer.  A node pass then sums, for every global node, the
// contributions of the (at most 8) cells that share it -- the transpose of
// the gather -- and applies the fused epilogue.  No atomics: every output is
// written by exactly one thread, in a fixed summation order.
//
// The same node pass, fed with a DG vector as the element buffer, is the
// c-restriction (sum of the duplicated DG nodes, Section 3.2 c-coarsening).
#include <algorithm>

#include "sumfac.cuh"

namespace sipg {

template <>
void upload_tables_fe<double>(const Tables<double> &t) { upload_tables_tu(t); }
template <>
void upload_tables_fe<float>(const Tables<float> &t) { upload_tables_tu(t); }

// (x, y, z) of point i of an nx x ny x nz grid in 32-bit arithmetic (the
// launchers keep every grid below 2^32 points): the 64-bit divisions they
// replace cost more than the loads of the small node passes
__device__ __forceinline__ void grid_coords(const long i, const int nx, const int ny, int g[3]) {
  const unsigned u = (unsigned)i, r = u / (unsigned)nx;
  g[0] = (int)(u - r * (unsigned)nx);
  g[1] = (int)(r % (unsigned)ny);
  g[2] = (int)(r / (unsigned)ny);
}

__device__ __forceinline__ bool node_constrained(const int g[3], const int grid[3], const int bc[6]) {
  return (g[0] == 0 && bc[0] == 0) || (g[0] == grid[0] - 1 && bc[1] == 0) ||
         (g[1] == 0 && bc[2] == 0) || (g[1] == grid[1] - 1 && bc[3] == 0) ||
         (g[2] == 0 && bc[4] == 0) || (g[2] == grid[2] - 1 && bc[5] == 0);
}

// The cell pass on cells cell0 .. cell0 + ncta - 1 of one vector (input ug,
// element buffer ebv), one line of N points per thread, N^2 threads per cell
// (threads beyond ncta N^2 only join the barriers).
template <typename T, int N, bool CURVED>
__device__ __forceinline__ void fe_cell_body(const FEArgs<T> &a, const T *__restrict__ ug, T *__restrict__ ebv,
                                             const int cell0, const int ncta, T *sm) {
  constexpr int N2 = N * N, N3 = N2 * N, TT = Tile<N>::T3;
  const int NT = blockDim.x;
  const int tid = threadIdx.x, cl = tid / N2, l = tid - cl * N2;
  const bool act = cl < ncta;
  T *su = sm + cl * Tile<N>::CS;
  // each thread gathers its z-line of the cell's nodes straight into
  // registers (constrained Dirichlet nodes read as zero); the first sweep
  // runs on them before anything goes to shared memory
  T xl[N];
  if (act) {
    constexpr int P = N - 1;
    const int cell = cell0 + cl;
    const int cx = cell % a.m[0], rr = cell / a.m[0], cy = rr % a.m[1], cz = rr / a.m[1];
    int g[3] = {cx * P + l % N, cy * P + l / N, 0};
    const size_t b0 = g[0] + (size_t)a.grid[0] * g[1], sz = (size_t)a.grid[0] * a.grid[1];
#pragma unroll
    for (int q = 0; q < N; ++q) {
      g[2] = cz * P + q;
      xl[q] = node_constrained(g, a.grid, a.bc) ? T(0) : ug[b0 + sz * g[2]];
    }
  }
  if constexpr (!CURVED) {
    // An axis-aligned box cell: its matrix is the sum over d of alpha_d times
    // the tensor product of the 1D stiffness matrix K1 in direction d and the
    // 1D mass matrix M1 in the other two (both under the Gauss rule, as the
    // interpolate / differentiate / weight / transpose sweeps of the general
    // path compute it), so y = ax K1 M1 M1 u + ay M1 K1 M1 u + az M1 M1 K1 u
    // takes 7 1D products instead of 12: along z a = M1 u, b = K1 u; along y
    // c = M1 a, f = ay K1 a + az M1 b; along x y = ax K1 c + M1 f.
    T *t0 = su, *t1 = su + TT;
    int base, stride;
    if (act) {
      line_of<N>(2, l, base, stride);
      T y[N];
      apply_mat<T, N, MK1>(xl, y);
      store_line<T, N>(t1, base, stride, y);
      apply_mat<T, N, MM1>(xl, y);
      store_line<T, N>(t0, base, stride, y);
    }
    __syncthreads();
    if (act) {
      line_of<N>(1, l, base, stride);
      T x[N], y[N], k[N];
      load_line<T, N>(t0, base, stride, x);
      apply_mat<T, N, MM1>(x, y);
      store_line<T, N>(t0, base, stride, y);
      apply_mat<T, N, MK1>(x, k);
      load_line<T, N>(t1, base, stride, x);
      apply_mat<T, N, MM1>(x, y);
#pragma unroll
      for (int q = 0; q < N; ++q) y[q] = fma(a.alpha[1], k[q], a.alpha[2] * y[q]);
      store_line<T, N>(t1, base, stride, y);
    }
    __syncthreads();
    if (!act) return;
    line_of<N>(0, l, base, stride);
    T x[N], y[N], k[N];
    load_line<T, N>(t0, base, stride, x);
    apply_mat<T, N, MK1>(x, k);
    load_line<T, N>(t1, base, stride, x);
    apply_mat<T, N, MM1>(x, y);
    T *eb = ebv + (size_t)(cell0 + cl) * N3 + N * l;   // the x-line of points (q, l % N, l / N)
#pragma unroll
    for (int q = 0; q < N; ++q) eb[q] = fma(a.alpha[0], k[q], y[q]);
    return;
  }
  if (act) {   // interpolation along z from the registers, then x and y in place
    int base, stride;
    line_of<N>(2, l, base, stride);
    T y[N];
    apply_mat<T, N, MS>(xl, y);
    store_line<T, N>(su, base, stride, y);
  }
  __syncthreads();
#pragma unroll 1
  for (int d = 0; d < 2; ++d) {
    if (act) sweep_inplace<T, N, MS>(su, d, l);
    __syncthreads();
  }
  if (act) {
#pragma unroll 1
    for (int d = 0; d < 3; ++d) {
      int base, stride;
      line_of<N>(d, l, base, stride);
      T x[N], y[N];
      load_line<T, N>(su, base, stride, x);
      apply_mat<T, N, MD>(x, y);
      store_line<T, N>(su + (1 + d) * TT, base, stride, y);
    }
  }
  __syncthreads();
  for (int i = tid; i < ncta * N3; i += NT) {
    const int c = i / N3, p = i - c * N3;
    T *s = sm + c * Tile<N>::CS + TT + Tile<N>::idx(p);
    const T g0 = s[0], g1 = s[TT], g2 = s[2 * TT];
    if constexpr (!CURVED) {
      s[0] = g0 * a.wcart[p];
      s[TT] = g1 * a.wcart[N3 + p];
      s[2 * TT] = g2 * a.wcart[2 * N3 + p];
    } else {
      const T *M = a.metric + (size_t)(cell0 + c) * 6 * N3 + p;
      const T xx = M[0], yy = M[N3], zz = M[2 * N3], xy = M[3 * N3], xz = M[4 * N3], yz = M[5 * N3];
      s[0] = xx * g0 + xy * g1 + xz * g2;
      s[TT] = xy * g0 + yy * g1 + yz * g2;
      s[2 * TT] = xz * g0 + yz * g1 + zz * g2;
    }
  }
  __syncthreads();
#pragma unroll 1
  for (int d = 0; d < 3; ++d) {
    if (act) {
      int base, stride;
      line_of<N>(d, l, base, stride);
      T x[N], y[N];
      load_line<T, N>(su + (1 + d) * TT, base, stride, x);
      apply_mat<T, N, MDt>(x, y);
      if (d == 0) {
        store_line<T, N>(su, base, stride, y);
      } else {
#pragma unroll
        for (int q = 0; q < N; ++q) su[base + q * stride] += y[q];
      }
    }
    __syncthreads();
  }
#pragma unroll 1
  for (int d = 0; d < 2; ++d) {
    if (act) sweep_inplace<T, N, MSt>(su, d, l);
    __syncthreads();
  }
  if (!act) return;
  T x[N], y[N];
  {
    int base, stride;
    line_of<N>(2, l, base, stride);
    load_line<T, N>(su, base, stride, x);
  }
  apply_mat<T, N, MSt>(x, y);
  T *eb = ebv + (size_t)(cell0 + cl) * N3 + l;
#pragma unroll
  for (int q = 0; q < N; ++q) eb[q * N2] = y[q];
}

// cb cells per thread block (a launch parameter, cb N^2 threads); MULTI:
// several vectors, block b = cell group b / nv of vector b % nv (compiled
// apart from the single-vector kernel, whose offsets would cost registers)
template <typename T, int N, bool CURVED, bool MULTI>
__global__ void __launch_bounds__(kCellThreads) fe_cell_kernel(const FEArgs<T> a, const int cb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sm = reinterpret_cast<T *>(smem_raw);
  // block -> (cell group, vector); the vectors of one group are neighbours
  const int grp = MULTI ? blockIdx.x / a.nv : blockIdx.x, vec = MULTI ? blockIdx.x - grp * a.nv : 0;
  const int cell0 = grp * cb;
  fe_cell_body<T, N, CURVED>(a, MULTI ? a.u + vec * a.vs : a.u, MULTI ? a.ebuf + vec * a.es : a.ebuf, cell0,
                             min(cb, a.ncells - cell0), sm);
}

// Cell-local diagonal of the FE operator (setup, FP64): one thread per (cell, node).
template <int N, bool CURVED>
__global__ void fe_diag_cells_kernel(const FEArgs<double> a, const double *S, const double *Sd) {
  constexpr int N2 = N * N, N3 = N2 * N;
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)a.ncells * N3) return;
  const int cell = (int)(idx / N3), i = (int)(idx - (long)cell * N3);
  const int ix = i % N, iy = (i / N) % N, iz = i / N2;
  double sum = 0;
  for (int qz = 0; qz < N; ++qz)
    for (int qy = 0; qy < N; ++qy)
      for (int qx = 0; qx < N; ++qx) {
        const int p = qx + N * qy + N2 * qz;
        const double sx = S[qx * N + ix], sy = S[qy * N + iy], sz = S[qz * N + iz];
        const double g0 = Sd[qx * N + ix] * sy * sz, g1 = sx * Sd[qy * N + iy] * sz, g2 = sx * sy * Sd[qz * N + iz];
        if (!CURVED) {
          sum += a.wcart[p] * g0 * g0 + a.wcart[N3 + p] * g1 * g1 + a.wcart[2 * N3 + p] * g2 * g2;
        } else {
          const double *M = a.metric + (size_t)cell * 6 * N3 + p;
          sum += M[0] * g0 * g0 + M[N3] * g1 * g1 + M[2 * N3] * g2 * g2 +
                 2.0 * (M[3 * N3] * g0 * g1 + M[4 * N3] * g0 * g2 + M[5 * N3] * g1 * g2);
        }
      }
  a.ebuf[idx] = sum;
}

// ------------------------------------------------- assembled low-degree levels
// On FE levels of degree p <= 2 the operator is applied from an assembled
// stencil instead of by sum factorisation: those levels are small and their
// matrix-free apply (a cell pass with a dozen barriers plus a node pass) is
// bound by latency, not by arithmetic or bytes.  The stencil holds, for every
// node g and offset o in [-p, p]^3, the matrix entry A[g][g + o] = the sum of
// the element-matrix entries of the cells containing both nodes, with the
// same quadrature and metric as the matrix-free cell pass (so both give the
// same operator up to rounding); constrained rows are identity rows and
// constrained columns are zero, as in the matrix-free pass.

// Element matrices K[cell][i][j] = sum_q grad phi_i^T M_q grad phi_j (setup, FP64).
template <int N, bool CURVED>
__global__ void fe_elem_matrix_kernel(const FEArgs<double> a, const double *S, const double *Sd, double *K) {
  constexpr int N2 = N * N, N3 = N2 * N;
  const int cell = blockIdx.x;
  for (int ij = threadIdx.x; ij < N3 * N3; ij += blockDim.x) {
    const int i = ij / N3, j = ij - i * N3;
    const int ii[3] = {i % N, (i / N) % N, i / N2}, jj[3] = {j % N, (j / N) % N, j / N2};
    double sum = 0;
    for (int qz = 0; qz < N; ++qz)
      for (int qy = 0; qy < N; ++qy)
        for (int qx = 0; qx < N; ++qx) {
          const int q = qx + N * qy + N2 * qz;
          const double si[3] = {S[qx * N + ii[0]], S[qy * N + ii[1]], S[qz * N + ii[2]]};
          const double sj[3] = {S[qx * N + jj[0]], S[qy * N + jj[1]], S[qz * N + jj[2]]};
          const double gi[3] = {Sd[qx * N + ii[0]] * si[1] * si[2], si[0] * Sd[qy * N + ii[1]] * si[2],
                                si[0] * si[1] * Sd[qz * N + ii[2]]};
          const double gj[3] = {Sd[qx * N + jj[0]] * sj[1] * sj[2], sj[0] * Sd[qy * N + jj[1]] * sj[2],
                                sj[0] * sj[1] * Sd[qz * N + jj[2]]};
          if (!CURVED) {
            sum += a.wcart[q] * gi[0] * gj[0] + a.wcart[N3 + q] * gi[1] * gj[1] + a.wcart[2 * N3 + q] * gi[2] * gj[2];
          } else {
            const double *M = a.metric + (size_t)cell * 6 * N3 + q;
            const double xx = M[0], yy = M[N3], zz = M[2 * N3], xy = M[3 * N3], xz = M[4 * N3], yz = M[5 * N3];
            sum += gi[0] * (xx * gj[0] + xy * gj[1] + xz * gj[2]) + gi[1] * (xy * gj[0] + yy * gj[1] + yz * gj[2]) +
                   gi[2] * (xz * gj[0] + yz * gj[1] + zz * gj[2]);
          }
        }
    K[(size_t)cell * N3 * N3 + ij] = sum;
  }
}

// Stencil of the level: coef[o][g], one thread per (node, offset) (setup, FP64).
__global__ void fe_stencil_assemble_kernel(const FEArgs<double> a, const double *__restrict__ K,
                                           double *__restrict__ coef) {
  const int p = a.deg, n = p + 1, n3 = n * n * n, w = 2 * p + 1;
  const long ng = (long)a.grid[0] * a.grid[1] * a.grid[2];
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ng * w * w * w) return;
  const int o = (int)(idx / ng);
  const long gid = idx - (long)o * ng;
  int g[3];
  grid_coords(gid, a.grid[0], a.grid[1], g);
  const int off[3] = {o % w - p, (o / w) % w - p, o / (w * w) - p};
  if (node_constrained(g, a.grid, a.bc)) {
    coef[idx] = (off[0] == 0 && off[1] == 0 && off[2] == 0) ? 1.0 : 0.0;
    return;
  }
  int h[3];
  for (int d = 0; d < 3; ++d) h[d] = g[d] + off[d];
  for (int d = 0; d < 3; ++d)
    if (h[d] < 0 || h[d] >= a.grid[d]) {
      coef[idx] = 0.0;
      return;
    }
  if (node_constrained(h, a.grid, a.bc)) {
    coef[idx] = 0.0;
    return;
  }
  // cells containing both nodes: per direction c with c p <= min, max <= c p + p
  int cs[3][2], cn[3];
  for (int d = 0; d < 3; ++d) {
    cn[d] = 0;
    const int lo = min(g[d], h[d]), hi = max(g[d], h[d]);
    for (int c = lo / p - 1; c <= lo / p; ++c)
      if (c >= 0 && c < a.m[d] && c * p <= lo && hi <= c * p + p) cs[d][cn[d]++] = c;
  }
  double sum = 0;
  for (int z = 0; z < cn[2]; ++z)
    for (int y = 0; y < cn[1]; ++y)
      for (int x = 0; x < cn[0]; ++x) {
        const int c[3] = {cs[0][x], cs[1][y], cs[2][z]};
        const size_t cell = c[0] + (size_t)a.m[0] * (c[1] + (size_t)a.m[1] * c[2]);
        const int li = (g[0] - c[0] * p) + n * ((g[1] - c[1] * p) + n * (g[2] - c[2] * p));
        const int lj = (h[0] - c[0] * p) + n * ((h[1] - c[1] * p) + n * (h[2] - c[2] * p));
        sum += K[cell * n3 * n3 + (size_t)li * n3 + lj];
      }
  coef[idx] = sum;
}

// Stencil apply with the gather's epilogue (modes 0, 1, 2), vector
// blockIdx.y.  SL = 4 (P = 1) or 8 (P = 2, 3) consecutive lanes share a node:
// lane z < W sums the W^2 offsets of slab z of the (2P+1)^3 stencil (all its
// loads issued together), the node's lanes add their sums by shuffles and the
// first lane writes the row.  Neighbours outside the grid or on a Dirichlet
// plane are skipped (their coefficients are zero).  Spreading a row over
// lanes shortens each thread's chain of dependent loads: these levels are
// small and bound by latency.
template <typename T, int P>
__global__ void __launch_bounds__(256) fe_stencil_apply_kernel(const FEArgs<T> a, const T *__restrict__ coef) {
  constexpr int W = 2 * P + 1, SL = P == 1 ? 4 : 8;
  const long ng = (long)a.grid[0] * a.grid[1] * a.grid[2];
  const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int z = (int)(t % SL);
  const long gid = t / SL;
  const bool live = gid < ng && z < W;
  const int64_t vo = blockIdx.y * a.vs;
  const T *__restrict__ u = a.u + vo;
  T y = T(0);
  int g[3] = {0, 0, 0};
  if (gid < ng) {
    grid_coords(gid, a.grid[0], a.grid[1], g);
  }
  if (live) {
    auto ok = [&](int d, int k) {
      const int h = g[d] + k - P;
      return h >= 0 && h < a.grid[d] && !(h == 0 && a.bc[2 * d] == 0) && !(h == a.grid[d] - 1 && a.bc[2 * d + 1] == 0);
    };
    if (ok(2, z)) {
      const long sy = a.grid[0], sz = (long)a.grid[0] * a.grid[1];
      const long base = gid + (long)(z - P) * sz;
      T cf[W * W], uv[W * W];
      // loads first (a skipped neighbour reads the node itself), then the sum
#pragma unroll
      for (int yy = 0; yy < W; ++yy)
#pragma unroll
        for (int x = 0; x < W; ++x) {
          const int o = x + W * (yy + W * z);
          const bool take = ok(0, x) && ok(1, yy);
          cf[x + W * yy] = coef[(long)o * ng + gid];
          uv[x + W * yy] = u[take ? base + (x - P) + (yy - P) * sy : gid];
        }
#pragma unroll
      for (int yy = 0; yy < W; ++yy)
#pragma unroll
        for (int x = 0; x < W; ++x)
          y = (ok(0, x) && ok(1, yy)) ? fma(cf[x + W * yy], uv[x + W * yy], y) : y;
    }
  }
#pragma unroll
  for (int w = SL / 2; w > 0; w >>= 1) y += __shfl_xor_sync(0xffffffffu, y, w, SL);
  if (gid >= ng || z != 0) return;
  if (node_constrained(g, a.grid, a.bc)) y = u[gid];   // identity row
  const long gv = vo + gid;
  if (a.mode == 0) {
    a.out[gv] = y;
  } else if (a.mode == 2) {
    a.out[gv] = a.b[gv] - y;
  } else {
    T v = a.c3 * a.dinv[gid] * (a.b[gv] - y);
    if (a.x) v = fma(a.c1, a.x[gv], v);
    if (a.xp) v = fma(a.c2, a.xp[gv], v);
    a.out[gv] = v;
  }
}

// Node pass: out[g] = sum over the cells sharing node g of ebuf, then the epilogue.
template <typename T, int P>
__device__ __forceinline__ void fe_gather_node(const FEArgs<T> &a, const long gid, const int vec) {
  constexpr int n = P + 1, n2 = n * n, n3 = n2 * n;
  const T *__restrict__ ebuf = a.ebuf + vec * a.es;
  const int64_t vo = vec * a.vs;
  int g[3];
  grid_coords(gid, a.grid[0], a.grid[1], g);
  const bool cons = node_constrained(g, a.grid, a.bc);
  T y;
  if (cons) {
    y = (a.mode == 3 || a.mode == 5) ? T(0) : (a.mode == 4 ? T(1) : a.u[vo + gid]);
  } else {
    // per direction: the cell the node starts (its last cell for the last
    // node, where it sits on the upper face) and, when the node is on that
    // cell's lower face, the cell below, whose entry is this one's plus the
    // fixed step D_d (local index + P, cell index - one cell)
    int c[3], r[3];
    bool lo[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      c[d] = g[d] / P;
      r[d] = g[d] - c[d] * P;
      if (c[d] == a.m[d]) {
        c[d] -= 1;
        r[d] = P;
      }
      lo[d] = r[d] == 0 && c[d] > 0;
    }
    const long own = (c[0] + (long)a.m[0] * (c[1] + (long)a.m[1] * c[2])) * n3 + r[0] + n * r[1] + n2 * r[2];
    const long D0 = P - (long)n3, D1 = (long)P * n - (long)a.m[0] * n3,
               D2 = (long)P * n2 - (long)a.m[0] * a.m[1] * n3;
    // all eight loads issued unconditionally (a missing cell reads entry 0),
    // then summed in a fixed order over the cells that exist (the cell below
    // before the own one in every direction)
    T e[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int x = q & 1, yy = (q >> 1) & 1, z = q >> 2;
      const bool take = (x || lo[0]) && (yy || lo[1]) && (z || lo[2]);
      const long addr = own + (x ? 0 : D0) + (yy ? 0 : D1) + (z ? 0 : D2);
      e[q] = ebuf[take ? addr : 0];
    }
    y = T(0);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int x = q & 1, yy = (q >> 1) & 1, z = q >> 2;
      if ((x || lo[0]) && (yy || lo[1]) && (z || lo[2])) y += e[q];
    }
  }
  const long gv = vo + gid;
  if (a.mode == 0 || a.mode >= 3) {
    a.out[gv] = y;
    if (a.mode == 5) a.out2[gv] = a.c3 * a.dinv[gid] * y;   // launch_xdb's x = c D^-1 b
  } else if (a.mode == 2) {
    a.out[gv] = a.b[gv] - y;
  } else {
    T v = a.c3 * a.dinv[gid] * (a.b[gv] - y);
    if (a.x) v = fma(a.c1, a.x[gv], v);
    if (a.xp) v = fma(a.c2, a.xp[gv], v);
    a.out[gv] = v;
  }
}

// the node pass for the task's degree (1..8)
template <typename T>
__device__ __forceinline__ void fe_gather_node_any(const FEArgs<T> &a, const long gid, const int vec) {
  switch (a.deg) {
    case 1: fe_gather_node<T, 1>(a, gid, vec); break;
    case 2: fe_gather_node<T, 2>(a, gid, vec); break;
    case 3: fe_gather_node<T, 3>(a, gid, vec); break;
    case 4: fe_gather_node<T, 4>(a, gid, vec); break;
    case 5: fe_gather_node<T, 5>(a, gid, vec); break;
    case 6: fe_gather_node<T, 6>(a, gid, vec); break;
    case 7: fe_gather_node<T, 7>(a, gid, vec); break;
    default: fe_gather_node<T, 8>(a, gid, vec); break;
  }
}

template <typename T, int P>
__global__ void fe_gather_kernel(const FEArgs<T> a) {
  const long total = (long)a.grid[0] * a.grid[1] * a.grid[2];
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= total) return;
  fe_gather_node<T, P>(a, gid, blockIdx.y);   // vector blockIdx.y
}

// c-transfer prolongation: x_dg[cell][i] += x_fe[node(cell, i)]  (injection).
template <typename T>
__device__ __forceinline__ void c_prolongate_dof(const FEArgs<T> &a, const T *xc, T *xdg, const long idx) {
  const int n = a.deg + 1, n2 = n * n, n3 = n2 * n;
  // 32-bit index arithmetic (the launchers keep the DG vector below 2^32 values)
  const unsigned ui = (unsigned)idx, cu = ui / (unsigned)n3;
  const int cell = (int)cu, p = (int)(ui - cu * (unsigned)n3);
  const int g[3] = {(cell % a.m[0]) * a.deg + p % n, ((cell / a.m[0]) % a.m[1]) * a.deg + (p / n) % n,
                    (cell / (a.m[0] * a.m[1])) * a.deg + p / n2};
  if (node_constrained(g, a.grid, a.bc)) return;
  xdg[idx] += xc[g[0] + (size_t)a.grid[0] * (g[1] + (size_t)a.grid[1] * g[2])];
}

template <typename T>
__global__ void c_prolongate_add_kernel(const FEArgs<T> a, const T *xc, T *xdg, const int64_t dg_stride) {
  const int n = a.deg + 1;
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)a.ncells * n * n * n) return;
  c_prolongate_dof<T>(a, xc + blockIdx.y * a.vs, xdg + blockIdx.y * dg_stride, idx);   // vector blockIdx.y
}

// ------------------------------------------------ batched launches (many problems)
// One launch of a pass for the same level of several independent problems:
// block b runs item b, which names the problem (its task: the pass's
// arguments for that problem) and the cells or nodes it covers.  The bodies
// are the single-problem ones, so every problem's result is bit for bit the
// one its own launch gives.  A problem whose flexible-CG system has left the
// iteration (segs[p].active == 0) is skipped.

template <typename T, bool CURVED>
__global__ void __launch_bounds__(kBatchCellThreads) fe_cell_batched_kernel(const FETask<T> *__restrict__ tasks,
                                                                          const WorkItem *__restrict__ items,
                                                                          const Seg *__restrict__ segs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sm = reinterpret_cast<T *>(smem_raw);
  const WorkItem w = items[blockIdx.x];
  if (segs && !segs[w.p].active) return;
  const FETask<T> &P = tasks[w.p];
  switch (P.a.deg + 1) {
#define SIPG_FEB_CASE(NN) \
  case NN:                \
    fe_cell_body<T, NN, CURVED>(P.a, P.a.u, P.a.ebuf, w.cell0, w.ncta, sm); \
    break;
    SIPG_FEB_CASE(2)
    SIPG_FEB_CASE(3)
    SIPG_FEB_CASE(4)
    SIPG_FEB_CASE(5)
    SIPG_FEB_CASE(6)
    SIPG_FEB_CASE(7)
    SIPG_FEB_CASE(8)
    SIPG_FEB_CASE(9)
#undef SIPG_FEB_CASE
    default:
      break;
  }
}

// node passes (kind 0: gather with the task's mode and epilogue) and the
// c-prolongation (kind 1), kBatchNodeThreads outputs per item
template <typename T>
__global__ void __launch_bounds__(kBatchNodeThreads) fe_nodes_batched_kernel(const FETask<T> *__restrict__ tasks,
                                                                           const NodeItem *__restrict__ items,
                                                                           const Seg *__restrict__ segs, int kind) {
  const NodeItem w = items[blockIdx.x];
  if (segs && !segs[w.p].active) return;
  const FETask<T> &P = tasks[w.p];
  const long i = (long)w.blk * kBatchNodeThreads + threadIdx.x;
  if (kind == 0) {
    if (i < (long)P.a.grid[0] * P.a.grid[1] * P.a.grid[2]) fe_gather_node_any<T>(P.a, i, 0);
  } else {
    const int n = P.a.deg + 1;
    if (i < (long)P.a.ncells * n * n * n) c_prolongate_dof<T>(P.a, P.xc, P.xdg, i);
  }
}

// p/h prolongation, one thread per fine node: the coarse FE function is
// evaluated at the node through the owning fine cell, x_f += P x_c.  The
// coarse function is continuous, so every cell sharing the node gives the
// same value and the multiplicity-weighted scatter of Section 3.2 reduces to
// one evaluation.  P1 holds the 1D interpolation matrices l^c_j(x^f_i)
// ([child][nf][nc]; child 0 only for the p-transfer).
// NC: coarse points per direction at compile time (unrolled, all loads in
// flight together), 0 = runtime
// COH: xc and xf were written earlier in the same launch by other blocks of
// a cluster (the fused tail below): read them through L2
template <bool COH, typename T>
__device__ __forceinline__ T ldv(const T *p) {
  if constexpr (COH) return __ldcg(p);
  else return *p;
}

template <typename T, int NC, bool COH>
__device__ __forceinline__ void fe_prolongate_node(const XferGeom &G, const T *__restrict__ P1, const T *xc, T *xf,
                                                   const long gid) {
  int g[3];
  grid_coords(gid, G.gf[0], G.gf[1], g);
  if (node_constrained(g, G.gf, G.bc)) return;
  const int nf = G.pf + 1, nc = NC > 0 ? NC : G.pc + 1;
  const T *row[3];
  int base[3];
  for (int d = 0; d < 3; ++d) {
    const int c = min(g[d] / G.pf, G.mf[d] - 1);
    const int r = g[d] - c * G.pf;
    int child = 0, cc = c;
    if (G.kind == 2) {
      child = c & 1;
      cc = c >> 1;
    }
    row[d] = P1 + ((size_t)child * nf + r) * nc;
    base[d] = cc * G.pc;
  }
  // factored tensor contraction: x, then y, then z (nc^3 + nc^2 + nc FMAs)
  T sum = T(0);
#pragma unroll
  for (int jz = 0; jz < (NC > 0 ? NC : nc); ++jz) {
    T sy = T(0);
#pragma unroll
    for (int jy = 0; jy < (NC > 0 ? NC : nc); ++jy) {
      const size_t off = (size_t)G.gc[0] * ((base[1] + jy) + (size_t)G.gc[1] * (base[2] + jz)) + base[0];
      T sx = T(0);
#pragma unroll
      for (int jx = 0; jx < (NC > 0 ? NC : nc); ++jx) sx = fma(row[0][jx], ldv<COH>(xc + off + jx), sx);
      sy = fma(row[1][jy], sx, sy);
    }
    sum = fma(row[2][jz], sy, sum);
  }
  xf[gid] = ldv<COH>(xf + gid) + sum;
}

template <typename T, int NC>
__global__ void fe_prolongate_add_kernel(const XferGeom G, const T *__restrict__ P1, const T *__restrict__ xc,
                                         T *__restrict__ xf) {
  const long total = (long)G.gf[0] * G.gf[1] * G.gf[2];
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= total) return;
  // vector blockIdx.y
  fe_prolongate_node<T, NC, false>(G, P1, xc + blockIdx.y * G.sc, xf + blockIdx.y * G.sf, gid);
}

// p/h restriction node by node for the two small transfers of the hierarchy
// (degree 2 -> 1 on one mesh, degree 1 across a 2:1 refinement): coarse node
// J sums the fine nodal values weighted by its coarse basis function at the
// fine nodes, r_c[J] = sum_i phi_J(x_i) r_f[i] over the unconstrained fine
// nodes i (R = P^T with the interpolation P of the prolongation), one launch
// instead of a cell pass and a node pass.  In both cases coarse node J sits
// at fine index 2 J per direction and its support there is 2J-1 .. 2J+1 (the
// fine nodes 2J +- 2 are the neighbouring coarse nodes, where phi_J = 0); the
// weights come from the prolongation's 1D tables.  27 loads per node, issued
// unconditionally (a missing entry reads fine node 2J) and summed by
// selection in a fixed order.
template <typename T, bool COH>
__device__ __forceinline__ void fe_restrict_node(const XferGeom &G, const T *__restrict__ P1, const T *rf, T *rc,
                                                 const long gid) {
  int J[3];
  grid_coords(gid, G.gc[0], G.gc[1], J);
  if (node_constrained(J, G.gc, G.bc)) {
    rc[gid] = T(0);
    return;
  }
  const int nf = G.pf + 1, nc = G.pc + 1;
  int idx[3][3];
  T w[3][3];
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      const int i = 2 * J[d] + e - 1;   // fine index
      const int C = e == 0 ? J[d] - 1 : (J[d] < G.mc[d] ? J[d] : J[d] - 1);   // coarse cell holding i and J
      const int a = J[d] - C;
      int ch = 0, b;
      if (G.kind == 2) {
        ch = min(i - 2 * C, 1);
        b = i - (2 * C + ch);
      } else {
        b = i - C * G.pf;
      }
      const bool ok = i >= 0 && i < G.gf[d] && C >= 0 && C < G.mc[d] && !(i == 0 && G.bc[2 * d] == 0) &&
                      !(i == G.gf[d] - 1 && G.bc[2 * d + 1] == 0);
      idx[d][e] = ok ? i : 2 * J[d];
      const size_t t = ok ? ((size_t)ch * nf + b) * nc + a : 0;   // in the table even when unused
      w[d][e] = ok ? P1[t] : T(0);
    }
  const long sy = G.gf[0], sz = (long)G.gf[0] * G.gf[1];
  T sum = T(0);
#pragma unroll
  for (int z = 0; z < 3; ++z)
#pragma unroll
    for (int y = 0; y < 3; ++y)
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        const T wt = w[0][x] * w[1][y] * w[2][z];
        const T v = ldv<COH>(rf + idx[0][x] + sy * idx[1][y] + sz * idx[2][z]);
        sum = wt != T(0) ? fma(wt, v, sum) : sum;
      }
  rc[gid] = sum;
}

template <typename T>
__global__ void fe_restrict_nodes_kernel(const XferGeom G, const T *__restrict__ P1, const T *__restrict__ rf,
                                         T *__restrict__ rc) {
  const long total = (long)G.gc[0] * G.gc[1] * G.gc[2];
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= total) return;
  // vector blockIdx.y
  fe_restrict_node<T, false>(G, P1, rf + blockIdx.y * G.sf, rc + blockIdx.y * G.sc, gid);
}

// p/h restriction, cell part, by sum factorisation: one thread block per
// coarse cell visits its fine cells (1 for p, 8 children for h); for each it
// loads the fine nodal values weighted by 1/multiplicity (the transposed,
// weighted scatter of Section 3.2; the weight is a product of per-direction
// factors 1 or 1/2, exact) and contracts them with the 1D matrix P1^T along x,
// y and z.  The coarse cell's local sums go to the element buffer; the node
// pass then sums the coarse cells sharing each coarse node.
template <typename T>
__global__ void fe_restrict_cells_kernel(const XferGeom G, const T *__restrict__ P1, const T *__restrict__ rf,
                                         T *__restrict__ ebuf) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sm = reinterpret_cast<T *>(smem_raw);
  const int nf = G.pf + 1, nc = G.pc + 1;
  const int nf3 = nf * nf * nf, nc3 = nc * nc * nc;
  T *A = sm;                        // nf^3
  T *B = A + nf3;                   // nf^2 nc   [iz][iy][jx]
  T *C = B + nf * nf * nc;          // nf nc^2   [iz][jy][jx]
  T *acc = C + nf * nc * nc;        // nc^3
  const int cc = blockIdx.x;
  rf += blockIdx.y * G.sf;   // vector blockIdx.y
  ebuf += blockIdx.y * G.se;
  const int cijk[3] = {cc % G.mc[0], (cc / G.mc[0]) % G.mc[1], cc / (G.mc[0] * G.mc[1])};
  const int nch = G.kind == 2 ? 2 : 1;
  for (int j = threadIdx.x; j < nc3; j += blockDim.x) acc[j] = T(0);
  for (int ch = 0; ch < nch * nch * nch; ++ch) {
    const int child[3] = {ch & (nch - 1), (ch / nch) & (nch - 1), ch / (nch * nch)};
    int fijk[3];
    for (int d = 0; d < 3; ++d) fijk[d] = G.kind == 2 ? 2 * cijk[d] + child[d] : cijk[d];
    __syncthreads();
    for (int i = threadIdx.x; i < nf3; i += blockDim.x) {
      const int ii[3] = {i % nf, (i / nf) % nf, i / (nf * nf)};
      int g[3];
      T w = T(1);
      for (int d = 0; d < 3; ++d) {
        g[d] = fijk[d] * G.pf + ii[d];
        if ((ii[d] == 0 && fijk[d] > 0) || (ii[d] == G.pf && fijk[d] < G.mf[d] - 1)) w *= T(0.5);
      }
      A[i] = node_constrained(g, G.gf, G.bc)
                 ? T(0)
                 : w * rf[g[0] + (size_t)G.gf[0] * (g[1] + (size_t)G.gf[1] * g[2])];
    }
    __syncthreads();
    const T *Px = P1 + (size_t)child[0] * nf * nc, *Py = P1 + (size_t)child[1] * nf * nc,
            *Pz = P1 + (size_t)child[2] * nf * nc;
    for (int o = threadIdx.x; o < nf * nf * nc; o += blockDim.x) {   // B[iz][iy][jx]
      const int jx = o % nc, r = o / nc;
      T s = T(0);
      for (int ix = 0; ix < nf; ++ix) s += Px[ix * nc + jx] * A[r * nf + ix];
      B[o] = s;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < nf * nc * nc; o += blockDim.x) {   // C[iz][jy][jx]
      const int jx = o % nc, jy = (o / nc) % nc, iz = o / (nc * nc);
      T s = T(0);
      for (int iy = 0; iy < nf; ++iy) s += Py[iy * nc + jy] * B[(iz * nf + iy) * nc + jx];
      C[o] = s;
    }
    __syncthreads();
    for (int o = threadIdx.x; o < nc3; o += blockDim.x) {   // acc[jz][jy][jx]
      const int jxy = o % (nc * nc), jz = o / (nc * nc);
      T s = T(0);
      for (int iz = 0; iz < nf; ++iz) s += Pz[iz * nc + jz] * C[iz * nc * nc + jxy];
      acc[o] += s;
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < nc3; j += blockDim.x) ebuf[(size_t)cc * nc3 + j] = acc[j];
}

// Transfers between DG levels (p on one mesh, or 2:1 h): the spaces share no
// nodes, so P is block diagonal over the fine cells with the parent's 1D
// interpolation matrices (no multiplicity weights).  One thread block per
// coarse cell and its fine cells (1 for p, 8 children for h), contracting
// along x, y, z in shared memory.  PROLONG: x_f += P x_c; else r_c = P^T r_f.
template <typename T, bool PROLONG>
__global__ void dg_transfer_kernel(const XferGeom G, const T *__restrict__ P1, const T *__restrict__ in,
                                   T *__restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sm = reinterpret_cast<T *>(smem_raw);
  const int nf = G.pf + 1, nc = G.pc + 1;
  const int nf3 = nf * nf * nf, nc3 = nc * nc * nc;
  const int big = nf3 > nc3 ? nf3 : nc3;
  T *A = sm, *B = A + big, *C = B + big, *acc = C + big;
  const int cc = blockIdx.x;
  in += blockIdx.y * (PROLONG ? G.sc : G.sf);   // vector blockIdx.y
  out += blockIdx.y * (PROLONG ? G.sf : G.sc);
  const int cijk[3] = {cc % G.mc[0], (cc / G.mc[0]) % G.mc[1], cc / (G.mc[0] * G.mc[1])};
  const int nch = G.kind == 4 ? 2 : 1;
  if (!PROLONG)
    for (int j = threadIdx.x; j < nc3; j += blockDim.x) acc[j] = T(0);
  else
    for (int j = threadIdx.x; j < nc3; j += blockDim.x) acc[j] = in[(size_t)cc * nc3 + j];
  for (int ch = 0; ch < nch * nch * nch; ++ch) {
    const int child[3] = {ch & (nch - 1), (ch / nch) & (nch - 1), ch / (nch * nch)};
    int fijk[3];
    for (int d = 0; d < 3; ++d) fijk[d] = G.kind == 4 ? 2 * cijk[d] + child[d] : cijk[d];
    const size_t fcell = fijk[0] + (size_t)G.mf[0] * (fijk[1] + (size_t)G.mf[1] * fijk[2]);
    const T *Px = P1 + (size_t)child[0] * nf * nc, *Py = P1 + (size_t)child[1] * nf * nc,
            *Pz = P1 + (size_t)child[2] * nf * nc;
    __syncthreads();
    if (PROLONG) {
      // B[jz][jy][ix] = sum_jx Px[ix][jx] acc[jz][jy][jx]; C[jz][iy][ix]; fine[iz][iy][ix]
      for (int o = threadIdx.x; o < nc * nc * nf; o += blockDim.x) {
        const int ix = o % nf, r = o / nf;
        T s = T(0);
        for (int jx = 0; jx < nc; ++jx) s += Px[ix * nc + jx] * acc[r * nc + jx];
        B[o] = s;
      }
      __syncthreads();
      for (int o = threadIdx.x; o < nc * nf * nf; o += blockDim.x) {
        const int ix = o % nf, iy = (o / nf) % nf, jz = o / (nf * nf);
        T s = T(0);
        for (int jy = 0; jy < nc; ++jy) s += Py[iy * nc + jy] * B[(jz * nc + jy) * nf + ix];
        C[o] = s;
      }
      __syncthreads();
      for (int o = threadIdx.x; o < nf3; o += blockDim.x) {
        const int ixy = o % (nf * nf), iz = o / (nf * nf);
        T s = T(0);
        for (int jz = 0; jz < nc; ++jz) s += Pz[iz * nc + jz] * C[jz * nf * nf + ixy];
        out[fcell * nf3 + o] += s;
      }
    } else {
      for (int i = threadIdx.x; i < nf3; i += blockDim.x) A[i] = in[fcell * nf3 + i];
      __syncthreads();
      for (int o = threadIdx.x; o < nf * nf * nc; o += blockDim.x) {   // B[iz][iy][jx]
        const int jx = o % nc, r = o / nc;
        T s = T(0);
        for (int ix = 0; ix < nf; ++ix) s += Px[ix * nc + jx] * A[r * nf + ix];
        B[o] = s;
      }
      __syncthreads();
      for (int o = threadIdx.x; o < nf * nc * nc; o += blockDim.x) {   // C[iz][jy][jx]
        const int jx = o % nc, jy = (o / nc) % nc, iz = o / (nc * nc);
        T s = T(0);
        for (int iy = 0; iy < nf; ++iy) s += Py[iy * nc + jy] * B[(iz * nf + iy) * nc + jx];
        C[o] = s;
      }
      __syncthreads();
      for (int o = threadIdx.x; o < nc3; o += blockDim.x) {
        const int jxy = o % (nc * nc), jz = o / (nc * nc);
        T s = T(0);
        for (int iz = 0; iz < nf; ++iz) s += Pz[iz * nc + jz] * C[iz * nc * nc + jxy];
        acc[o] += s;
      }
    }
  }
  if (!PROLONG) {
    __syncthreads();
    for (int j = threadIdx.x; j < nc3; j += blockDim.x) out[(size_t)cc * nc3 + j] = acc[j];
  }
}

// ---------------------------------------------------------------- launchers
template <typename T, int N, bool CURVED>
static cudaError_t run_fe_cells(const FEArgs<T> &a, cudaStream_t s, int cb) {
  if (cb <= 0) cb = default_cb(N);
  if (cb > max_cb(N, sizeof(T))) return cudaErrorInvalidValue;
  const size_t smem = (size_t)cb * Tile<N>::CS * sizeof(T);
  const int64_t grid = (int64_t)((a.ncells + cb - 1) / cb) * a.nv;
  if (grid == 0) return cudaSuccess;
  if (grid > 0x7fffffff) return cudaErrorInvalidValue;
  if (a.nv > 1)
    fe_cell_kernel<T, N, CURVED, true><<<(unsigned)grid, cb * N * N, smem, s>>>(a, cb);
  else
    fe_cell_kernel<T, N, CURVED, false><<<(unsigned)grid, cb * N * N, smem, s>>>(a, cb);
  note_launch();
  return cudaGetLastError();
}

template <typename T, int N, bool CURVED>
static cudaError_t occ_fe_cells(int cb, int *blocks) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, fe_cell_kernel<T, N, CURVED, false>, cb * N * N,
                                                       (size_t)cb * Tile<N>::CS * sizeof(T));
}

template <typename T, int N>
static cudaError_t prep_fe_n() {
  const int smem = max_cb(N, sizeof(T)) * Tile<N>::CS * (int)sizeof(T);
  cudaError_t e = cudaSuccess;
  for (cudaError_t r :
       {cudaFuncSetAttribute(fe_cell_kernel<T, N, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
        cudaFuncSetAttribute(fe_cell_kernel<T, N, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
        cudaFuncSetAttribute(fe_cell_kernel<T, N, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
        cudaFuncSetAttribute(fe_cell_kernel<T, N, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)})
    if (r != cudaSuccess) e = r;
  return e;
}

cudaError_t prepare_fe_kernels() {
  cudaError_t e = cudaSuccess;
  for (cudaError_t r : {prep_fe_n<double, 2>(), prep_fe_n<double, 3>(), prep_fe_n<double, 4>(), prep_fe_n<double, 5>(),
                        prep_fe_n<double, 6>(), prep_fe_n<double, 7>(), prep_fe_n<double, 8>(), prep_fe_n<double, 9>(),
                        prep_fe_n<float, 2>(), prep_fe_n<float, 3>(), prep_fe_n<float, 4>(), prep_fe_n<float, 5>(),
                        prep_fe_n<float, 6>(), prep_fe_n<float, 7>(), prep_fe_n<float, 8>(), prep_fe_n<float, 9>()})
    if (r != cudaSuccess) e = r;
  return e;
}

template <int N, bool CURVED>
static cudaError_t run_fe_diag(const FEArgs<double> &a, cudaStream_t s) {
  const Rules1D &r = rules(N);
  // tables are tiny: pass through a small device allocation owned by the call
  double *tabs = nullptr;
  cudaError_t e = cudaMallocAsync(&tabs, 2 * N * N * sizeof(double), s);
  if (e != cudaSuccess) return e;
  cudaMemcpyAsync(tabs, r.S.data(), N * N * sizeof(double), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(tabs + N * N, r.Sd.data(), N * N * sizeof(double), cudaMemcpyHostToDevice, s);
  const long total = (long)a.ncells * N * N * N;
  const int bs = 128;
  fe_diag_cells_kernel<N, CURVED><<<(int)((total + bs - 1) / bs), bs, 0, s>>>(a, tabs, tabs + N * N);
  note_launch();
  e = cudaGetLastError();
  cudaStreamSynchronize(s);
  cudaFreeAsync(tabs, s);
  return e;
}

template <typename T>
cudaError_t launch_fe_cells(int n, bool curved, const FEArgs<T> &a, bool diag_only, cudaStream_t s, int cb) {
#define SIPG_FE_CASE(NN)                                                                     \
  case NN:                                                                                   \
    if (diag_only) {                                                                         \
      if constexpr (sizeof(T) == 8)                                                          \
        return curved ? run_fe_diag<NN, true>(a, s) : run_fe_diag<NN, false>(a, s);          \
      return cudaErrorInvalidValue;                                                          \
    }                                                                                        \
    return curved ? run_fe_cells<T, NN, true>(a, s, cb) : run_fe_cells<T, NN, false>(a, s, cb);
  switch (n) {
    SIPG_FE_CASE(2)
    SIPG_FE_CASE(3)
    SIPG_FE_CASE(4)
    SIPG_FE_CASE(5)
    SIPG_FE_CASE(6)
    SIPG_FE_CASE(7)
    SIPG_FE_CASE(8)
    SIPG_FE_CASE(9)
    default:
      return cudaErrorInvalidValue;
  }
#undef SIPG_FE_CASE
}

template <int N, bool CURVED>
static cudaError_t run_fe_stencil_setup(const FEArgs<double> &a, double *coef, cudaStream_t s) {
  constexpr int N3 = N * N * N;
  const Rules1D &r = rules(N);
  double *tabs = nullptr, *K = nullptr;
  cudaError_t e = cudaMalloc(&tabs, 2 * N * N * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&K, std::max<size_t>(1, (size_t)a.ncells * N3 * N3) * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpyAsync(tabs, r.S.data(), N * N * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(tabs + N * N, r.Sd.data(), N * N * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && a.ncells > 0) {
    fe_elem_matrix_kernel<N, CURVED><<<a.ncells, 128, 0, s>>>(a, tabs, tabs + N * N, K);
    note_launch();
    const long w = 2 * (N - 1) + 1;
    const long total = (long)a.grid[0] * a.grid[1] * a.grid[2] * w * w * w;
    fe_stencil_assemble_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(a, K, coef);
    note_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(K);
  cudaFree(tabs);
  return e;
}

cudaError_t launch_fe_stencil_setup(bool curved, const FEArgs<double> &a, double *coef, cudaStream_t s) {
  switch (a.deg) {
    case 1:
      return curved ? run_fe_stencil_setup<2, true>(a, coef, s) : run_fe_stencil_setup<2, false>(a, coef, s);
    case 2:
      return curved ? run_fe_stencil_setup<3, true>(a, coef, s) : run_fe_stencil_setup<3, false>(a, coef, s);
    case 3:
      return curved ? run_fe_stencil_setup<4, true>(a, coef, s) : run_fe_stencil_setup<4, false>(a, coef, s);
    default:
      return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_fe_stencil_apply(const FEArgs<T> &a, const T *coef, cudaStream_t s) {
  const long total = (long)a.grid[0] * a.grid[1] * a.grid[2];
  const int bs = 256;
  if (total == 0) return cudaSuccess;
  if (total >= (1L << 32)) return cudaErrorInvalidValue;   // the kernel's 32-bit grid coordinates
  const long lanes = total * (a.deg == 1 ? 4 : 8);   // lanes per node (the kernel's SL)
  if ((lanes + bs - 1) / bs > 0x7fffffffL) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)((lanes + bs - 1) / bs), a.nv);
  if (a.deg == 1)
    fe_stencil_apply_kernel<T, 1><<<grid, bs, 0, s>>>(a, coef);
  else if (a.deg == 2)
    fe_stencil_apply_kernel<T, 2><<<grid, bs, 0, s>>>(a, coef);
  else if (a.deg == 3)
    fe_stencil_apply_kernel<T, 3><<<grid, bs, 0, s>>>(a, coef);
  else
    return cudaErrorInvalidValue;
  note_launch();
  return cudaGetLastError();
}

template <typename T>
int fe_max_cells_per_block(int n) {
  return max_cb(n, sizeof(T));
}

template <typename T>
cudaError_t fe_blocks_per_sm(int n, bool curved, int cb, int *blocks) {
#define SIPG_FE_OCC(NN) \
  case NN:              \
    return curved ? occ_fe_cells<T, NN, true>(cb, blocks) : occ_fe_cells<T, NN, false>(cb, blocks);
  switch (n) {
    SIPG_FE_OCC(2)
    SIPG_FE_OCC(3)
    SIPG_FE_OCC(4)
    SIPG_FE_OCC(5)
    SIPG_FE_OCC(6)
    SIPG_FE_OCC(7)
    SIPG_FE_OCC(8)
    SIPG_FE_OCC(9)
    default:
      return cudaErrorInvalidValue;
  }
#undef SIPG_FE_OCC
}

template <typename T>
cudaError_t launch_fe_gather(const FEArgs<T> &a, cudaStream_t s) {
  const long total = (long)a.grid[0] * a.grid[1] * a.grid[2];
  const int bs = 256;
  if (total == 0) return cudaSuccess;
  if (total >= (1L << 32) || a.deg < 1 || a.deg > 8) return cudaErrorInvalidValue;   // 32-bit coordinates
  const dim3 grid((unsigned)((total + bs - 1) / bs), a.nv);
  switch (a.deg) {
    case 1: fe_gather_kernel<T, 1><<<grid, bs, 0, s>>>(a); break;
    case 2: fe_gather_kernel<T, 2><<<grid, bs, 0, s>>>(a); break;
    case 3: fe_gather_kernel<T, 3><<<grid, bs, 0, s>>>(a); break;
    case 4: fe_gather_kernel<T, 4><<<grid, bs, 0, s>>>(a); break;
    case 5: fe_gather_kernel<T, 5><<<grid, bs, 0, s>>>(a); break;
    case 6: fe_gather_kernel<T, 6><<<grid, bs, 0, s>>>(a); break;
    case 7: fe_gather_kernel<T, 7><<<grid, bs, 0, s>>>(a); break;
    default: fe_gather_kernel<T, 8><<<grid, bs, 0, s>>>(a); break;
  }
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fe_cells_batched(bool curved, const FETask<T> *tasks, const WorkItem *items, int nitems,
                                    size_t smem, const Seg *segs, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  if (curved)
    fe_cell_batched_kernel<T, true><<<nitems, kBatchCellThreads, smem, s>>>(tasks, items, segs);
  else
    fe_cell_batched_kernel<T, false><<<nitems, kBatchCellThreads, smem, s>>>(tasks, items, segs);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fe_nodes_batched(const FETask<T> *tasks, const NodeItem *items, int nitems, const Seg *segs,
                                    int kind, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  fe_nodes_batched_kernel<T><<<nitems, kBatchNodeThreads, 0, s>>>(tasks, items, segs, kind);
  note_launch();
  return cudaGetLastError();
}

int tile_values(int n) { return cell_values(n); }

template <typename T>
cudaError_t prep_fe_cells_batched(size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(fe_cell_batched_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fe_cell_batched_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return e;
}

template <typename T>
cudaError_t launch_c_prolongate_add(const FEArgs<T> &a, const T *xc, T *xdg, cudaStream_t s, int64_t dg_stride) {
  const int n = a.deg + 1;
  const long total = (long)a.ncells * n * n * n;
  const int bs = 256;
  if (total == 0) return cudaSuccess;
  if (total >= (1L << 32)) return cudaErrorInvalidValue;   // the kernel's 32-bit index arithmetic
  c_prolongate_add_kernel<T><<<dim3((unsigned)((total + bs - 1) / bs), a.nv), bs, 0, s>>>(a, xc, xdg, dg_stride);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fe_prolongate_add(const XferGeom &g, const T *P1, const T *xc, T *xf, cudaStream_t s) {
  const long total = (long)g.gf[0] * g.gf[1] * g.gf[2];
  const int bs = 256;
  if (total == 0) return cudaSuccess;
  if (total >= (1L << 32)) return cudaErrorInvalidValue;   // the kernel's 32-bit grid coordinates
  const dim3 grid((unsigned)((total + bs - 1) / bs), g.nv);
  switch (g.pc + 1) {
    case 2:
      fe_prolongate_add_kernel<T, 2><<<grid, bs, 0, s>>>(g, P1, xc, xf);
      break;
    case 3:
      fe_prolongate_add_kernel<T, 3><<<grid, bs, 0, s>>>(g, P1, xc, xf);
      break;
    case 4:
      fe_prolongate_add_kernel<T, 4><<<grid, bs, 0, s>>>(g, P1, xc, xf);
      break;
    case 5:
      fe_prolongate_add_kernel<T, 5><<<grid, bs, 0, s>>>(g, P1, xc, xf);
      break;
    default:
      fe_prolongate_add_kernel<T, 0><<<grid, bs, 0, s>>>(g, P1, xc, xf);
  }
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fe_restrict_nodes(const XferGeom &g, const T *P1, const T *rf, T *rc, cudaStream_t s) {
  if (!fe_restrict_nodes_ok(g)) return cudaErrorInvalidValue;
  const long total = (long)g.gc[0] * g.gc[1] * g.gc[2];
  const int bs = 128;
  if (total == 0) return cudaSuccess;
  if (total >= (1L << 32)) return cudaErrorInvalidValue;   // the kernel's 32-bit grid coordinates
  fe_restrict_nodes_kernel<T><<<dim3((unsigned)((total + bs - 1) / bs), g.nv), bs, 0, s>>>(g, P1, rf, rc);
  note_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------- fused tail
// Below a few thousand nodes a V-cycle step is a few microseconds of launch
// and load latency for a few microseconds' worth of nothing; the tail runs
// all steps of its levels in one launch of one thread-block cluster, a
// cluster barrier (release/acquire at cluster scope) between the steps.
// Vectors written inside the launch are read through L2 (ldv<true>); the
// stencils, diagonals, transfer tables and the coarse inverse are read-only.

// all threads of the cluster: the writes before it are seen by the reads after
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;\n" ::: "memory");
}

// One row of a 27-point stencil apply and its epilogue, one thread per node:
// the three slab sums of fe_stencil_apply_kernel<T, 1> (slab z: its 9 offsets
// in the same order) combined in the order of its lane shuffles, lanes 0 and
// 2 first, then lane 1 with the idle lane 3's zero.  Written without
// branches: every load is issued (a neighbour outside the grid or on a
// Dirichlet plane reads the node itself) and the sums take their terms by
// selection.
template <typename T>
__device__ __forceinline__ void tail_stencil_node(const TailStep<T> &s, const int gid) {
  const int n[3] = {s.grid[0], s.grid[1], s.grid[2]};
  const long ng = (long)n[0] * n[1] * n[2];
  int g[3];
  grid_coords(gid, n[0], n[1], g);
  bool ok[3][3];   // neighbour at offset k - 1 along d exists and is free
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int h = g[d] + k - 1;
      ok[d][k] = (h >= 0) & (h < n[d]) & !((h == 0) & (s.bc[2 * d] == 0)) & !((h == n[d] - 1) & (s.bc[2 * d + 1] == 0));
    }
  const long sy = n[0], sz = (long)n[0] * n[1];
  const T *__restrict__ coef = s.coef;
  const T *u = s.u;
  T cf[27], uv[27];
#pragma unroll
  for (int z = 0; z < 3; ++z)
#pragma unroll
    for (int yy = 0; yy < 3; ++yy)
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        const int o = x + 3 * (yy + 3 * z);
        const bool take = ok[0][x] & ok[1][yy] & ok[2][z];
        cf[o] = coef[(long)o * ng + gid];
        uv[o] = ldv<true>(u + (take ? gid + (x - 1) + (yy - 1) * sy + (z - 1) * sz : gid));
      }
  // the epilogue's operands too, before the sums (an absent x or x_prev reads u)
  const bool cons = node_constrained(g, n, s.bc);
  const T ug = ldv<true>(u + gid);
  const T bv = ldv<true>(s.b + gid);
  const T dv = s.dinv[gid];
  const T xv = ldv<true>((s.x ? s.x : u) + gid), xpv = ldv<true>((s.xp ? s.xp : u) + gid);
  T part[3];
#pragma unroll
  for (int z = 0; z < 3; ++z) {
    T y = T(0);
#pragma unroll
    for (int yy = 0; yy < 3; ++yy)
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        const int o = x + 3 * (yy + 3 * z);
        y = (ok[0][x] & ok[1][yy]) ? fma(cf[o], uv[o], y) : y;
      }
    part[z] = ok[2][z] ? y : T(0);
  }
  T y = (part[0] + part[2]) + (part[1] + T(0));
  y = cons ? ug : y;   // identity row
  if (s.mode == 2) {
    s.out[gid] = bv - y;
  } else {
    T v = s.c3 * dv * (bv - y);
    if (s.x) v = fma(s.c1, xv, v);
    if (s.xp) v = fma(s.c2, xpv, v);
    s.out[gid] = v;
  }
}

// The program (nsteps steps) is copied to shared memory first; the grid is
// one cluster.  A step's items go out in chunks of 32 (one warp each), chunk q
// to block q mod C, so that a small level spreads over all the cluster's SMs
// instead of filling the first block.
template <typename T>
__global__ void __launch_bounds__(kTailThreads, 1) fe_tail_kernel(const TailStep<T> *__restrict__ prog,
                                                                  const int nsteps) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TailStep<T> *sp = reinterpret_cast<TailStep<T> *>(smem_raw);
  {
    const int4 *src = reinterpret_cast<const int4 *>(prog);
    int4 *dst = reinterpret_cast<int4 *>(smem_raw);
    const int words = nsteps * (int)(sizeof(TailStep<T>) / sizeof(int4));
    for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  const int nt = gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  const int q0 = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;   // the thread's first chunk
  const int first = q0 * 32 + lane;
#pragma unroll 1
  for (int k = 0; k < nsteps; ++k) {
    const TailStep<T> &s = sp[k];
    switch (s.op) {
      case kTailXdb:   // launch_xdb
#pragma unroll 1
        for (int i = first; i < s.n; i += nt) s.out[i] = s.c3 * s.dinv[i] * ldv<true>(s.b + i);
        break;
      case kTailStencil:
#pragma unroll 1
        for (int i = first; i < s.n; i += nt) tail_stencil_node<T>(s, i);
        break;
      case kTailRestrict:
#pragma unroll 1
        for (int i = first; i < s.n; i += nt) fe_restrict_node<T, true>(s.g, s.P1, s.u, s.out, i);
        break;
      case kTailCoarse: {   // launch_dense_gemv: one warp per row
#pragma unroll 1
        for (int row = q0; row < s.n; row += nt >> 5) {
          const double *ar = s.Ainv + (size_t)row * s.n;
          double acc = 0;
          for (int j = lane; j < s.n; j += 32) acc = fma(ar[j], (double)ldv<true>(s.b + j), acc);
          for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
          if (lane == 0) s.out[row] = (T)acc;
        }
        break;
      }
      default:   // kTailProlong
#pragma unroll 1
        for (int i = first; i < s.n; i += nt) fe_prolongate_node<T, 2, true>(s.g, s.P1, s.u, s.out, i);
    }
    cluster_barrier();
  }
}

template <typename T>
static cudaLaunchConfig_t tail_config(int nsteps, int cluster, cudaStream_t s, cudaLaunchAttribute *at) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)cluster);
  cfg.blockDim = dim3(kTailThreads);
  cfg.dynamicSmemBytes = (size_t)nsteps * sizeof(TailStep<T>);
  cfg.stream = s;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cfg;
}

template <typename T>
int fe_tail_cluster(int nsteps) {
  static_assert(sizeof(TailStep<T>) % sizeof(int4) == 0, "the program is copied in 16-byte words");
  if (nsteps <= 0 || nsteps > kTailMaxSteps) return 0;
  if (cudaFuncSetAttribute(fe_tail_kernel<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  for (const int cs : {16, 8}) {
    cudaLaunchAttribute at[1];
    const cudaLaunchConfig_t cfg = tail_config<T>(kTailMaxSteps, cs, nullptr, at);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, fe_tail_kernel<T>, &cfg) == cudaSuccess && n > 0) return cs;
    cudaGetLastError();
  }
  return 0;
}

template <typename T>
cudaError_t launch_fe_tail(const TailStep<T> *prog, int nsteps, int cluster, cudaStream_t s) {
  if (nsteps <= 0 || nsteps > kTailMaxSteps || (cluster != 8 && cluster != 16)) return cudaErrorInvalidValue;
  cudaLaunchAttribute at[1];
  const cudaLaunchConfig_t cfg = tail_config<T>(nsteps, cluster, s, at);
  const cudaError_t e = cudaLaunchKernelEx(&cfg, fe_tail_kernel<T>, prog, nsteps);
  note_launch();
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename T>
cudaError_t launch_fe_restrict_cells(const XferGeom &g, const T *P1, const T *rf, T *ebuf, cudaStream_t s) {
  const int nf = g.pf + 1, nc = g.pc + 1;
  const long ncc = (long)g.mc[0] * g.mc[1] * g.mc[2];
  const size_t smem = (size_t)(nf * nf * nf + nf * nf * nc + nf * nc * nc + nc * nc * nc) * sizeof(T);
  if (ncc == 0) return cudaSuccess;
  fe_restrict_cells_kernel<T><<<dim3((unsigned)ncc, g.nv), 128, smem, s>>>(g, P1, rf, ebuf);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_dg_transfer(const XferGeom &g, const T *P1, const T *in, T *out, bool prolong, cudaStream_t s) {
  const int nf = g.pf + 1, nc = g.pc + 1;
  const int big = std::max(nf * nf * nf, nc * nc * nc);
  const size_t smem = (size_t)(3 * big + nc * nc * nc) * sizeof(T);
  const long ncc = (long)g.mc[0] * g.mc[1] * g.mc[2];
  if (ncc == 0) return cudaSuccess;
  if (prolong)
    dg_transfer_kernel<T, true><<<dim3((unsigned)ncc, g.nv), 128, smem, s>>>(g, P1, in, out);
  else
    dg_transfer_kernel<T, false><<<dim3((unsigned)ncc, g.nv), 128, smem, s>>>(g, P1, in, out);
  note_launch();
  return cudaGetLastError();
}

#define SIPG_FE_INST(T)                                                                                   \
  template cudaError_t launch_fe_cells<T>(int, bool, const FEArgs<T> &, bool, cudaStream_t, int);       \
  template int fe_max_cells_per_block<T>(int);                                                          \
  template cudaError_t fe_blocks_per_sm<T>(int, bool, int, int *);                                      \
  template cudaError_t launch_fe_gather<T>(const FEArgs<T> &, cudaStream_t);                            \
  template cudaError_t launch_fe_stencil_apply<T>(const FEArgs<T> &, const T *, cudaStream_t);          \
  template cudaError_t launch_c_prolongate_add<T>(const FEArgs<T> &, const T *, T *, cudaStream_t, int64_t); \
  template cudaError_t launch_fe_cells_batched<T>(bool, const FETask<T> *, const WorkItem *, int, size_t,      \
                                                  const Seg *, cudaStream_t);                                  \
  template cudaError_t launch_fe_nodes_batched<T>(const FETask<T> *, const NodeItem *, int, const Seg *, int, \
                                                  cudaStream_t);                                               \
  template cudaError_t prep_fe_cells_batched<T>(size_t);                                                       \
  template cudaError_t launch_fe_prolongate_add<T>(const XferGeom &, const T *, const T *, T *,         \
                                                   cudaStream_t);                                       \
  template cudaError_t launch_fe_restrict_nodes<T>(const XferGeom &, const T *, const T *, T *,         \
                                                   cudaStream_t);                                       \
  template cudaError_t launch_fe_restrict_cells<T>(const XferGeom &, const T *, const T *, T *,         \
                                                   cudaStream_t);                                       \
  template cudaError_t launch_dg_transfer<T>(const XferGeom &, const T *, const T *, T *, bool, cudaStream_t); \
  template int fe_tail_cluster<T>(int);                                                                 \
  template cudaError_t launch_fe_tail<T>(const TailStep<T> *, int, int, cudaStream_t);
SIPG_FE_INST(double)
SIPG_FE_INST(float)

}  // namespace sipg
