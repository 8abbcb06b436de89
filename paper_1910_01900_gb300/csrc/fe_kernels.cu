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

__device__ __forceinline__ bool node_constrained(const int g[3], const int grid[3], const int bc[6]) {
  return (g[0] == 0 && bc[0] == 0) || (g[0] == grid[0] - 1 && bc[1] == 0) ||
         (g[1] == 0 && bc[2] == 0) || (g[1] == grid[1] - 1 && bc[3] == 0) ||
         (g[2] == 0 && bc[4] == 0) || (g[2] == grid[2] - 1 && bc[5] == 0);
}

template <typename T, int N, bool CURVED, int CB>
__global__ void __launch_bounds__(CB *N *N) fe_cell_kernel(const FEArgs<T> a) {
  constexpr int N2 = N * N, N3 = N2 * N, NT = CB * N2, TT = Tile<N>::T3;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sm = reinterpret_cast<T *>(smem_raw);
  const int tid = threadIdx.x, cl = tid / N2, l = tid - cl * N2;
  const int cell0 = blockIdx.x * CB;
  const int ncta = min(CB, a.ncells - cell0);
  const bool act = cl < ncta;
  T *su = sm + cl * 4 * TT;
  for (int i = tid; i < ncta * N3; i += NT) {
    const int c = i / N3, p = i - c * N3;
    const int cell = cell0 + c;
    const int g[3] = {(cell % a.m[0]) * a.deg + p % N, ((cell / a.m[0]) % a.m[1]) * a.deg + (p / N) % N,
                      (cell / (a.m[0] * a.m[1])) * a.deg + p / N2};
    const size_t gi = g[0] + (size_t)a.grid[0] * (g[1] + (size_t)a.grid[1] * g[2]);
    sm[c * 4 * TT + Tile<N>::idx(p)] = node_constrained(g, a.grid, a.bc) ? T(0) : a.u[gi];
  }
  __syncthreads();
#pragma unroll 1
  for (int d = 0; d < 3; ++d) {
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
    T *s = sm + c * 4 * TT + TT + Tile<N>::idx(p);
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
  T *eb = a.ebuf + (size_t)(cell0 + cl) * N3 + l;
#pragma unroll
  for (int q = 0; q < N; ++q) eb[q * N2] = y[q];
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

// Node pass: out[g] = sum over the cells sharing node g of ebuf, then the epilogue.
template <typename T>
__global__ void fe_gather_kernel(const FEArgs<T> a) {
  const long total = (long)a.grid[0] * a.grid[1] * a.grid[2];
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= total) return;
  const int n = a.deg + 1, n2 = n * n, n3 = n2 * n;
  const int g[3] = {(int)(gid % a.grid[0]), (int)((gid / a.grid[0]) % a.grid[1]),
                    (int)(gid / ((long)a.grid[0] * a.grid[1]))};
  const bool cons = node_constrained(g, a.grid, a.bc);
  T y;
  if (cons) {
    y = (a.mode == 3) ? T(0) : (a.mode == 4 ? T(1) : a.u[gid]);
  } else {
    // per direction: (cell, local index) pairs containing this node
    int cc[3][2], ll[3][2], cnt[3];
    for (int d = 0; d < 3; ++d) {
      const int c = g[d] / a.deg, r = g[d] - c * a.deg;
      cnt[d] = 0;
      if (r == 0 && c > 0) {
        cc[d][cnt[d]] = c - 1;
        ll[d][cnt[d]++] = a.deg;
      }
      if (c < a.m[d]) {
        cc[d][cnt[d]] = c;
        ll[d][cnt[d]++] = r;
      }
    }
    y = T(0);
    for (int z = 0; z < cnt[2]; ++z)
      for (int yy = 0; yy < cnt[1]; ++yy)
        for (int x = 0; x < cnt[0]; ++x) {
          const size_t cell = cc[0][x] + (size_t)a.m[0] * (cc[1][yy] + (size_t)a.m[1] * cc[2][z]);
          y += a.ebuf[cell * n3 + ll[0][x] + n * ll[1][yy] + n2 * ll[2][z]];
        }
  }
  if (a.mode == 0 || a.mode >= 3) {
    a.out[gid] = y;
  } else if (a.mode == 2) {
    a.out[gid] = a.b[gid] - y;
  } else {
    T v = a.c3 * a.dinv[gid] * (a.b[gid] - y);
    if (a.x) v = fma(a.c1, a.x[gid], v);
    if (a.xp) v = fma(a.c2, a.xp[gid], v);
    a.out[gid] = v;
  }
}

// c-transfer prolongation: x_dg[cell][i] += x_fe[node(cell, i)]  (injection).
template <typename T>
__global__ void c_prolongate_add_kernel(const FEArgs<T> a, const T *xc, T *xdg) {
  const int n = a.deg + 1, n2 = n * n, n3 = n2 * n;
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)a.ncells * n3) return;
  const int cell = (int)(idx / n3), p = (int)(idx - (long)cell * n3);
  const int g[3] = {(cell % a.m[0]) * a.deg + p % n, ((cell / a.m[0]) % a.m[1]) * a.deg + (p / n) % n,
                    (cell / (a.m[0] * a.m[1])) * a.deg + p / n2};
  if (node_constrained(g, a.grid, a.bc)) return;
  xdg[idx] += xc[g[0] + (size_t)a.grid[0] * (g[1] + (size_t)a.grid[1] * g[2])];
}

// p/h prolongation, one thread per fine node: the coarse FE function is
// evaluated at the node through the owning fine cell, x_f += P x_c.  The
// coarse function is continuous, so every cell sharing the node gives the
// same value and the multiplicity-weighted scatter of Section 3.2 reduces to
// one evaluation.  P1 holds the 1D interpolation matrices l^c_j(x^f_i)
// ([child][nf][nc]; child 0 only for the p-transfer).
template <typename T>
__global__ void fe_prolongate_add_kernel(const XferGeom G, const T *__restrict__ P1, const T *__restrict__ xc,
                                         T *__restrict__ xf) {
  const long total = (long)G.gf[0] * G.gf[1] * G.gf[2];
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= total) return;
  const int g[3] = {(int)(gid % G.gf[0]), (int)((gid / G.gf[0]) % G.gf[1]), (int)(gid / ((long)G.gf[0] * G.gf[1]))};
  if (node_constrained(g, G.gf, G.bc)) return;
  const int nf = G.pf + 1, nc = G.pc + 1;
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
  T sum = T(0);
  for (int jz = 0; jz < nc; ++jz)
    for (int jy = 0; jy < nc; ++jy) {
      const T wyz = row[1][jy] * row[2][jz];
      const size_t off = (size_t)G.gc[0] * ((base[1] + jy) + (size_t)G.gc[1] * (base[2] + jz));
      for (int jx = 0; jx < nc; ++jx) sum += row[0][jx] * wyz * xc[off + base[0] + jx];
    }
  xf[gid] += sum;
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
static cudaError_t run_fe_cells(const FEArgs<T> &a, cudaStream_t s) {
  constexpr int CB = default_cb(N);
  const size_t smem = (size_t)CB * 4 * Tile<N>::T3 * sizeof(T);
  const int grid = (a.ncells + CB - 1) / CB;
  if (grid == 0) return cudaSuccess;
  fe_cell_kernel<T, N, CURVED, CB><<<grid, CB * N * N, smem, s>>>(a);
  note_launch();
  return cudaGetLastError();
}

template <typename T, int N>
static cudaError_t prep_fe_n() {
  constexpr int CB = default_cb(N);
  const int smem = CB * 4 * Tile<N>::T3 * (int)sizeof(T);
  cudaError_t e = cudaFuncSetAttribute(fe_cell_kernel<T, N, false, CB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(fe_cell_kernel<T, N, true, CB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
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
cudaError_t launch_fe_cells(int n, bool curved, const FEArgs<T> &a, bool diag_only, cudaStream_t s) {
#define SIPG_FE_CASE(NN)                                                                     \
  case NN:                                                                                   \
    if (diag_only) {                                                                         \
      if constexpr (sizeof(T) == 8)                                                          \
        return curved ? run_fe_diag<NN, true>(a, s) : run_fe_diag<NN, false>(a, s);          \
      return cudaErrorInvalidValue;                                                          \
    }                                                                                        \
    return curved ? run_fe_cells<T, NN, true>(a, s) : run_fe_cells<T, NN, false>(a, s);
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

template <typename T>
cudaError_t launch_fe_gather(const FEArgs<T> &a, cudaStream_t s) {
  const long total = (long)a.grid[0] * a.grid[1] * a.grid[2];
  const int bs = 256;
  fe_gather_kernel<T><<<(int)((total + bs - 1) / bs), bs, 0, s>>>(a);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_c_prolongate_add(const FEArgs<T> &a, const T *xc, T *xdg, cudaStream_t s) {
  const int n = a.deg + 1;
  const long total = (long)a.ncells * n * n * n;
  const int bs = 256;
  c_prolongate_add_kernel<T><<<(int)((total + bs - 1) / bs), bs, 0, s>>>(a, xc, xdg);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fe_prolongate_add(const XferGeom &g, const T *P1, const T *xc, T *xf, cudaStream_t s) {
  const long total = (long)g.gf[0] * g.gf[1] * g.gf[2];
  const int bs = 256;
  fe_prolongate_add_kernel<T><<<(int)((total + bs - 1) / bs), bs, 0, s>>>(g, P1, xc, xf);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fe_restrict_cells(const XferGeom &g, const T *P1, const T *rf, T *ebuf, cudaStream_t s) {
  const int nf = g.pf + 1, nc = g.pc + 1;
  const long ncc = (long)g.mc[0] * g.mc[1] * g.mc[2];
  const size_t smem = (size_t)(nf * nf * nf + nf * nf * nc + nf * nc * nc + nc * nc * nc) * sizeof(T);
  if (ncc == 0) return cudaSuccess;
  fe_restrict_cells_kernel<T><<<(int)ncc, 128, smem, s>>>(g, P1, rf, ebuf);
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
    dg_transfer_kernel<T, true><<<(int)ncc, 128, smem, s>>>(g, P1, in, out);
  else
    dg_transfer_kernel<T, false><<<(int)ncc, 128, smem, s>>>(g, P1, in, out);
  note_launch();
  return cudaGetLastError();
}

#define SIPG_FE_INST(T)                                                                                   \
  template cudaError_t launch_fe_cells<T>(int, bool, const FEArgs<T> &, bool, cudaStream_t);            \
  template cudaError_t launch_fe_gather<T>(const FEArgs<T> &, cudaStream_t);                            \
  template cudaError_t launch_c_prolongate_add<T>(const FEArgs<T> &, const T *, T *, cudaStream_t);     \
  template cudaError_t launch_fe_prolongate_add<T>(const XferGeom &, const T *, const T *, T *,         \
                                                   cudaStream_t);                                       \
  template cudaError_t launch_fe_restrict_cells<T>(const XferGeom &, const T *, const T *, T *,         \
                                                   cudaStream_t);                                       \
  template cudaError_t launch_dg_transfer<T>(const XferGeom &, const T *, const T *, T *, bool, cudaStream_t);
SIPG_FE_INST(double)
SIPG_FE_INST(float)

}  // namespace sipg
