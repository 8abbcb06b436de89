// Matrix-free SIPG operator on the DG level (Section 4, Eq.
// MatrixFreeAbstractNotation; weak form Eq. WeakFormDG with the fluxes of
// Eqs. InteriorPenaltyFlux1/2 and the mirror boundary conditions of
// Eq. BoundaryConditions).
//
// Face integrals without atomics, in two passes over the cells:
//
//  eval pass      : u_e -> u at the Gauss points (3 interpolation sweeps) ->
//                   reference gradient at the Gauss points (3 collocation
//                   derivative sweeps), stored for the second pass; the value
//                   and the outward normal derivative on all six faces are
//                   extrapolated along the face normal and stored as the
//                   cell's face traces.
//  integrate pass : metric term on the stored gradient, then for every face
//                   the SIPG flux from the cell's own trace and the
//                   neighbour's trace, tested against the cell's own basis
//                   only (the neighbour integrates its own side in its own
//                   launch thread), then 3 transposed derivative sweeps and 3
//                   transposed interpolation sweeps, and the fused epilogue.
//
// Each cell writes only its own outputs, so no two threads ever update the
// same global value.  Per face point the own side computes, with [u] =
// u_own - u_nb and q = outward normal derivative of each side,
//   value coefficient   A = dA (tau_f [u] - (q_own - q_nb)/2)     (times v)
//   normal-deriv coeff. B = -dA [u] / 2                           (times d_n v)
// and on Dirichlet faces A = dA (2 tau_e u - q), B = -dA u; on Neumann faces
// A = B = 0.  This is the per-side form of
//   -{d_n v}[u] - [v]{d_n u} + tau [v][u]  and  -d_n v u - v d_n u + 2 tau v u.
#pragma once
#include "sumfac.cuh"

namespace sipg {

// Face point of the neighbour that sits at the own face point l = q1 + N q2
// (unstructured meshes): orientation code bit 0 swaps the two face
// directions, bits 1 and 2 reverse the first and second of them.
template <int N>
__device__ __forceinline__ int face_perm(const int code, const int l) {
  const int q1 = l % N, q2 = l / N;
  int a = (code & 1) ? q2 : q1, b = (code & 1) ? q1 : q2;
  if (code & 2) a = N - 1 - a;
  if (code & 4) b = N - 1 - b;
  return a + N * b;
}

// The interpolation of a cell's values to the Gauss points, reading u from
// global memory: the z-lines go straight from the loads through S (thread l
// of the cell reads its line u[l + q n^2], coalesced over the cell's
// threads) into the tile, then the x and y sweeps in place.  One tile store
// and one tile load per value fewer than staging u first.  Every thread of
// the block takes part in the barriers.
template <typename T, int N>
__device__ __forceinline__ void interpolate_from_global(const T *__restrict__ ucell, T *tile, const bool act,
                                                        const int l) {
  constexpr int N2 = N * N;
  if (act) {
    int base, stride;
    line_of<N>(2, l, base, stride);
    T x[N], y[N];
#pragma unroll
    for (int q = 0; q < N; ++q) x[q] = ucell[l + q * N2];
    apply_mat<T, N, MS>(x, y);
    store_line<T, N>(tile, base, stride, y);
  }
  __syncthreads();
#pragma unroll 1
  for (int d = 0; d < 2; ++d) {
    if (act) sweep_inplace<T, N, MS>(tile, d, l);
    __syncthreads();
  }
}

template <typename T>
struct VecPtrs {
  const T *u;
  T *out;
  const T *x, *xp, *b;
  T *grad, *trace;
};

// Evaluation pass for the cells cell0 .. cell0+ncta-1 of one problem, on a
// thread block of blockDim.x >= ncta * N^2 threads with 4 ncta N^3 values of
// shared memory at sm.  Shared by the per-problem and the batched kernels.
template <typename T, int N, bool CURVED, bool UNSTR = false>
__device__ __forceinline__ void dg_eval_body(const DGArgs<T> &a, const VecPtrs<T> &v, const int cell0, const int ncta, T *sm) {
  constexpr int N2 = N * N, N3 = N2 * N, TT = Tile<N>::T3;
  const int NT = blockDim.x;
  const int tid = threadIdx.x, cl = tid / N2, l = tid - cl * N2;
  const bool act = cl < ncta;
  T *su = sm + cl * Tile<N>::CS;

  interpolate_from_global<T, N>(v.u + (size_t)(cell0 + (act ? cl : 0)) * N3, su, act, l);
  // the gradient at the Gauss points (curved cells: the metric mixes its
  // components; an axis-aligned cell needs none of it here: its normal
  // derivatives come from the values through D^T l below, and its cell term
  // from the values through the collocation stiffness in the integration pass)
  if constexpr (CURVED) {
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
  }
  if (!a.recompute) {
    if constexpr (CURVED) {
      T *gg = v.grad + (size_t)cell0 * 3 * N3;
      for (int i = tid; i < ncta * 3 * N3; i += NT) {
        const int c = i / (3 * N3), r = i - c * 3 * N3, comp = r / N3;
        gg[i] = sm[c * Tile<N>::CS + (1 + comp) * TT + Tile<N>::idx(r - comp * N3)];
      }
    } else {   // the values at the Gauss points, [cell][n^3]
      T *gg = v.grad + (size_t)cell0 * N3;
      for (int i = tid; i < ncta * N3; i += NT) {
        const int c = i / N3;
        gg[i] = sm[c * Tile<N>::CS + Tile<N>::idx(i - c * N3)];
      }
    }
  }
  if (!act) return;
  const int cell = cell0 + cl;
  int ijk[3] = {0, 0, 0};
  if constexpr (!UNSTR) {
    ijk[0] = cell % a.m[0];
    ijk[1] = (cell / a.m[0]) % a.m[1];
    ijk[2] = cell / (a.m[0] * a.m[1]);
  }
  const Tables<T> &t = tab<T>();
#pragma unroll 1
  for (int d = 0; d < 3; ++d) {
    int base, stride;
    line_of<N>(d, l, base, stride);
    T x[N];
    load_line<T, N>(su, base, stride, x);
    T v0 = t.l0[N][0] * x[0], v1 = t.l1[N][0] * x[0];
#pragma unroll
    for (int q = 1; q < N; ++q) {
      v0 = fma(t.l0[N][q], x[q], v0);
      v1 = fma(t.l1[N][q], x[q], v1);
    }
    T q0, q1;
    if constexpr (!CURVED) {
      // l_s . (D x) = (D^T l_s) . x: the normal derivative from the values
      T g0 = t.dl0[N][0] * x[0], g1 = t.dl1[N][0] * x[0];
#pragma unroll
      for (int q = 1; q < N; ++q) {
        g0 = fma(t.dl0[N][q], x[q], g0);
        g1 = fma(t.dl1[N][q], x[q], g1);
      }
      q0 = -a.ih[d] * g0;
      q1 = a.ih[d] * g1;
    } else {
      T gr0[3], gr1[3];
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        T g[N];
        load_line<T, N>(su + (1 + b) * TT, base, stride, g);
        T g0 = t.l0[N][0] * g[0], g1 = t.l1[N][0] * g[0];
#pragma unroll
        for (int q = 1; q < N; ++q) {
          g0 = fma(t.l0[N][q], g[q], g0);
          g1 = fma(t.l1[N][q], g[q], g1);
        }
        gr0[b] = g0;
        gr1[b] = g1;
      }
      const T *c0, *c1;
      if constexpr (UNSTR) {   // own side's J^-1 n of the faces xi_d = 0 and xi_d = 1
        c0 = a.fc[0] + ((size_t)cell * 6 + 2 * d) * 3 * N2 + l;
        c1 = c0 + 3 * N2;
      } else {
        const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
        const size_t nfp = (size_t)a.m[t1] * a.m[t2];
        const size_t f0 = (size_t)ijk[d] * nfp + ijk[t1] + (size_t)a.m[t1] * ijk[t2];
        const size_t f1 = f0 + nfp;
        c0 = a.fc[d] + (f0 * 2 + 1) * 3 * N2 + l;   // this cell is the upper cell of plane i_d
        c1 = a.fc[d] + (f1 * 2 + 0) * 3 * N2 + l;   // and the lower cell of plane i_d+1
      }
      q0 = c0[0] * gr0[0] + c0[N2] * gr0[1] + c0[2 * N2] * gr0[2];
      q1 = c1[0] * gr1[0] + c1[N2] * gr1[1] + c1[2 * N2] * gr1[2];
    }
    T *tr = v.trace + ((size_t)cell * 6 + 2 * d) * 2 * N2 + l;
    tr[0] = v0;
    tr[N2] = q0;
    tr[2 * N2] = v1;
    tr[3 * N2] = q1;
  }
}

// Integration pass (same thread and shared-memory contract as the evaluation).
template <typename T, int N, bool CURVED, bool UNSTR = false>
__device__ __forceinline__ void dg_integrate_body(const DGArgs<T> &a, const VecPtrs<T> &v, const int cell0, const int ncta,
                                                  T *sm) {
  constexpr int N2 = N * N, N3 = N2 * N, TT = Tile<N>::T3;
  const int NT = blockDim.x;
  const int tid = threadIdx.x, cl = tid / N2, l = tid - cl * N2;
  const bool act = cl < ncta;
  T *st = sm + cl * Tile<N>::CS;   // value accumulator, then the integrated tile
  T *sg = st + TT;            // three gradient components (curved); the values (axis-aligned)

  if constexpr (!CURVED) {
    // An axis-aligned cell's term is sum_d alpha_d (D_d^T W D_d) applied to
    // the values at the Gauss points; W is a tensor product, so along a line
    // of direction d it is the collocation stiffness KG = D^T diag(w) D times
    // the line's weight alpha_d w_t1 w_t2: one product per direction (with the
    // face terms below) instead of a derivative and a transposed derivative.
    if (a.recompute) {
      interpolate_from_global<T, N>(v.u + (size_t)(cell0 + (act ? cl : 0)) * N3, sg, act, l);
    } else {
      const T *gg = v.grad + (size_t)cell0 * N3;
      for (int i = tid; i < ncta * N3; i += NT) {
        const int c = i / N3;
        sm[c * Tile<N>::CS + TT + Tile<N>::idx(i - c * N3)] = gg[i];
      }
      __syncthreads();
    }
  } else if (a.recompute) {
    // gradient at the Gauss points again from u: 3 interpolation and 3
    // collocation-derivative sweeps (the value slot st is free until the faces)
    interpolate_from_global<T, N>(v.u + (size_t)(cell0 + (act ? cl : 0)) * N3, st, act, l);
    if (act) {
#pragma unroll 1
      for (int d = 0; d < 3; ++d) {
        int base, stride;
        line_of<N>(d, l, base, stride);
        T x[N], y[N];
        load_line<T, N>(st, base, stride, x);
        apply_mat<T, N, MD>(x, y);
        store_line<T, N>(sg + d * TT, base, stride, y);
      }
    }
  } else {
    const T *gg = v.grad + (size_t)cell0 * 3 * N3;
    for (int i = tid; i < ncta * 3 * N3; i += NT) {
      const int c = i / (3 * N3), r = i - c * 3 * N3, comp = r / N3;
      sm[c * Tile<N>::CS + (1 + comp) * TT + Tile<N>::idx(r - comp * N3)] = gg[i];
    }
  }
  if constexpr (CURVED) {
    __syncthreads();
    for (int i = tid; i < ncta * N3; i += NT) {
      const int c = i / N3, p = i - c * N3, tp = Tile<N>::idx(p);
      T *s = sm + c * Tile<N>::CS + TT + tp;
      const T g0 = s[0], g1 = s[TT], g2 = s[2 * TT];
      const T *M = a.metric + (size_t)(cell0 + c) * 6 * N3 + p;
      const T xx = M[0], yy = M[N3], zz = M[2 * N3], xy = M[3 * N3], xz = M[4 * N3], yz = M[5 * N3];
      s[0] = xx * g0 + xy * g1 + xz * g2;
      s[TT] = xy * g0 + yy * g1 + yz * g2;
      s[2 * TT] = xz * g0 + yz * g1 + zz * g2;
    }
    __syncthreads();
  }

  const int cell = cell0 + cl;
  // cell coordinates and strides as scalars picked by direction (indexing a
  // small array with the runtime direction would put it in local memory)
  int i0 = 0, i1 = 0, i2 = 0;
  if (act && !UNSTR) {
    i0 = cell % a.m[0];
    i1 = (cell / a.m[0]) % a.m[1];
    i2 = cell / (a.m[0] * a.m[1]);
  }
  auto ijk = [&](int k) { return k == 0 ? i0 : (k == 1 ? i1 : i2); };
  auto mdim = [&](int k) { return k == 0 ? a.m[0] : (k == 1 ? a.m[1] : a.m[2]); };
  auto cstride = [&](int k) { return k == 0 ? 1 : (k == 1 ? a.m[0] : a.m[0] * a.m[1]); };
  const Tables<T> &t = tab<T>();
#pragma unroll 1
  for (int d = 0; d < 3; ++d) {
    if (act) {
      int base, stride;
      line_of<N>(d, l, base, stride);
      const T tau_e = a.tau[cell];
      T A[2], B[2];
      T cvec[2][3];
      const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
      const size_t nfp = (size_t)mdim(t1) * mdim(t2);
      const size_t ftan = ijk(t1) + (size_t)mdim(t1) * ijk(t2);
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const T *tr = v.trace + ((size_t)cell * 6 + 2 * d + s) * 2 * N2 + l;
        const T uo = tr[0], qo = tr[N2];
        if constexpr (UNSTR) {
          // neighbour, its local face and the orientation of the shared face
          const size_t cf = (size_t)cell * 6 + 2 * d + s;
          const int2 nf = a.ufn[cf];
          const T dA = a.fdA[0][cf * N2 + l];
          const T *c = a.fc[0] + cf * 3 * N2 + l;
          cvec[s][0] = c[0];
          cvec[s][1] = c[N2];
          cvec[s][2] = c[2 * N2];
          if (nf.x >= 0) {
            const T *tn = v.trace + ((size_t)nf.x * 6 + (nf.y & 7)) * 2 * N2 + face_perm<N>(nf.y >> 3, l);
            const T un = tn[0], qn = tn[N2];
            const T tau_f = max(tau_e, a.tau[nf.x]);
            const T jump = uo - un;
            const T hdA = T(0.5) * dA;
            A[s] = fma(dA * tau_f, jump, -hdA * (qo - qn));
            B[s] = -hdA * jump;
          } else if (nf.x == -1) {
            A[s] = fma(T(2) * dA * tau_e, uo, -dA * qo);
            B[s] = -dA * uo;
          } else {
            A[s] = T(0);
            B[s] = T(0);
          }
          continue;
        }
        T dA;
        const size_t face = (size_t)(ijk(d) + s) * nfp + ftan;
        if constexpr (CURVED) {
          dA = a.fdA[d][face * N2 + l];
          const T *c = a.fc[d] + (face * 2 + (s ? 0 : 1)) * 3 * N2 + l;
          cvec[s][0] = c[0];
          cvec[s][1] = c[N2];
          cvec[s][2] = c[2 * N2];
        } else {
          dA = a.fwcart[d * N2 + l];
        }
        const bool has_nb = s ? (ijk(d) < mdim(d) - 1) : (ijk(d) > 0);
        if (has_nb) {
          const int nb = cell + (s ? cstride(d) : -cstride(d));
          const T *tn = v.trace + ((size_t)nb * 6 + 2 * d + (1 - s)) * 2 * N2 + l;
          const T un = tn[0], qn = tn[N2];
          const T tau_f = max(tau_e, a.tau[nb]);
          const T jump = uo - un;
          const T hdA = T(0.5) * dA;
          A[s] = fma(dA * tau_f, jump, -hdA * (qo - qn));
          B[s] = -hdA * jump;
        } else if (a.bc[2 * d + s] == 0) {
          A[s] = fma(T(2) * dA * tau_e, uo, -dA * qo);
          B[s] = -dA * uo;
        } else {
          A[s] = T(0);
          B[s] = T(0);
        }
      }
      // extrapolation transposed: every point of the line gets l_s(q) times the
      // value coefficient of each side.  The normal-derivative test term adds
      // l_s(q) times its coefficient to the gradient component d along this
      // same line, which the transposed derivative sweep D^T along d reads
      // next; D^T applied to l_s is the fixed vector dl_s, so that term goes
      // into the value tile here as dl_s(q) times the coefficient (one
      // read-modify-write line less per direction, the same sum).
      T bn0, bn1;
      if constexpr (!CURVED) {
        bn0 = -a.ih[d] * B[0];
        bn1 = a.ih[d] * B[1];
      } else {
        bn0 = (d == 0 ? cvec[0][0] : (d == 1 ? cvec[0][1] : cvec[0][2])) * B[0];
        bn1 = (d == 0 ? cvec[1][0] : (d == 1 ? cvec[1][1] : cvec[1][2])) * B[1];
      }
      if constexpr (!CURVED && sizeof(T) == 4) {
        // the cell term along this line: KG times the line's weight, with the faces
        T x[N], y[N];
        load_line<T, N>(sg, base, stride, x);
        apply_mat<T, N, MKG>(x, y);
        const T cw = a.fwcart[d * N2 + l] * a.ih[d];
#pragma unroll
        for (int q = 0; q < N; ++q) {
          T *p = st + base + q * stride;
          const T f = fma(t.l0[N][q], A[0], fma(t.l1[N][q], A[1], fma(t.dl0[N][q], bn0, t.dl1[N][q] * bn1)));
          *p = fma(cw, y[q], d == 0 ? f : f + *p);
        }
      } else if (d == 0) {
#pragma unroll
        for (int q = 0; q < N; ++q)
          st[base + q * stride] = fma(t.l0[N][q], A[0], fma(t.l1[N][q], A[1], fma(t.dl0[N][q], bn0, t.dl1[N][q] * bn1)));
      } else {
#pragma unroll
        for (int q = 0; q < N; ++q) {
          T *p = st + base + q * stride;
          *p = fma(t.l0[N][q], A[0], fma(t.l1[N][q], A[1], fma(t.dl0[N][q], bn0, fma(t.dl1[N][q], bn1, *p))));
        }
      }
      if constexpr (CURVED) {
        // the tangential gradient components (J^-1 n has all three)
#pragma unroll
        for (int bb = 0; bb < 3; ++bb) {
          if (bb == d) continue;
          const T b0 = cvec[0][bb] * B[0], b1 = cvec[1][bb] * B[1];
          T *g = sg + bb * TT;
#pragma unroll
          for (int q = 0; q < N; ++q) {
            T *p = g + base + q * stride;
            *p = fma(t.l0[N][q], b0, fma(t.l1[N][q], b1, *p));
          }
        }
      }
    }
    __syncthreads();
  }
  if constexpr (CURVED) {
#pragma unroll 1
    for (int d = 0; d < 3; ++d) {
      if (act) {
        int base, stride;
        line_of<N>(d, l, base, stride);
        T x[N], y[N];
        load_line<T, N>(sg + d * TT, base, stride, x);
        apply_mat<T, N, MDt>(x, y);
#pragma unroll
        for (int q = 0; q < N; ++q) st[base + q * stride] += y[q];
      }
      __syncthreads();
    }
  } else if constexpr (sizeof(T) == 8) {
    // FP64: the cell term after the faces (within the face loop the sweep's
    // registers and the face coefficients' would not fit together)
#pragma unroll 1
    for (int d = 0; d < 3; ++d) {
      if (act) {
        int base, stride;
        line_of<N>(d, l, base, stride);
        T x[N], y[N];
        load_line<T, N>(sg, base, stride, x);
        apply_mat<T, N, MKG>(x, y);
        const T cw = a.fwcart[d * N2 + l] * a.ih[d];
#pragma unroll
        for (int q = 0; q < N; ++q) st[base + q * stride] = fma(cw, y[q], st[base + q * stride]);
      }
      __syncthreads();
    }
  }
#pragma unroll 1
  for (int d = 0; d < 2; ++d) {
    if (act) sweep_inplace<T, N, MSt>(st, d, l);
    __syncthreads();
  }
  if (!act) return;
  T x[N], y[N];
  {
    int base, stride;
    line_of<N>(2, l, base, stride);
    load_line<T, N>(st, base, stride, x);
  }
  apply_mat<T, N, MSt>(x, y);
  const size_t g0 = (size_t)cell * N3 + l;
  if (a.mode == 0) {
#pragma unroll
    for (int q = 0; q < N; ++q) v.out[g0 + q * N2] = y[q];
  } else if (a.mode == 2) {
#pragma unroll
    for (int q = 0; q < N; ++q) v.out[g0 + q * N2] = v.b[g0 + q * N2] - y[q];
  } else {
#pragma unroll
    for (int q = 0; q < N; ++q) {
      const size_t i = g0 + q * N2;
      T z = a.c3 * a.dinv[i] * (v.b[i] - y[q]);
      if (v.x) z = fma(a.c1, v.x[i], z);
      if (v.xp) z = fma(a.c2, v.xp[i], z);
      v.out[i] = z;
    }
  }
}

// Per-vector pointers of a multi-vector launch: vector r of u, out, x, xp, b
// and its scratch (geometry and inverse diagonal are shared).  A small
// struct of pointers only, so it stays in registers.
template <typename T>
__device__ __forceinline__ VecPtrs<T> vec_ptrs(const DGArgs<T> &a, const int r) {
  const int64_t o = r * a.vs;
  VecPtrs<T> v;
  v.u = a.u + o;
  v.out = a.out + o;
  v.x = a.x ? a.x + o : nullptr;
  v.xp = a.xp ? a.xp + o : nullptr;
  v.b = a.b ? a.b + o : nullptr;
  v.grad = a.grad ? a.grad + r * a.gs : nullptr;
  v.trace = a.trace + r * a.ts;
  return v;
}

// One thread block handles cb consecutive cells of one vector with cb N^2
// threads.  MULTI (several vectors of one operator): block b is cell group
// b / nv of vector b % nv, so the vectors of one group run side by side and
// share its geometry in L2.  The single-vector kernels are compiled apart:
// the per-vector offsets cost registers, which cost resident blocks (the FP32
// integration pass at 16 MDoF ran 14% slower with them).  cb is a launch
// parameter (picked per level and size by the tile-shape autotuner): one
// compiled kernel serves every block width up to kCellThreads threads.
// kMinCellBlocks caps FP32 variants at 40 registers (two blocks of
// kCellThreads per SM): left free, the compiler gave some of them 48-60
// (FP32 curved integration at k = 2: 50 registers, 16% slower at 16 MDoF).
// FP64 variants (56-64 registers, bound by the FP64 pipe) are left free.
template <typename T>
constexpr int kMinCellBlocks = sizeof(T) == 4 ? 2 : 1;

template <typename T, int N, bool CURVED, bool MULTI>
__global__ void __launch_bounds__(kCellThreads, kMinCellBlocks<T>) dg_eval_kernel(const DGArgs<T> a, const int cb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int grp = MULTI ? blockIdx.x / a.nv : blockIdx.x, vec = MULTI ? blockIdx.x - grp * a.nv : 0;
  const int cell0 = grp * cb;
  dg_eval_body<T, N, CURVED>(a, vec_ptrs(a, vec), cell0, min(cb, a.ncells - cell0), reinterpret_cast<T *>(smem_raw));
}

template <typename T, int N, bool CURVED, bool MULTI>
__global__ void __launch_bounds__(kCellThreads, kMinCellBlocks<T>) dg_integrate_kernel(const DGArgs<T> a, const int cb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int grp = MULTI ? blockIdx.x / a.nv : blockIdx.x, vec = MULTI ? blockIdx.x - grp * a.nv : 0;
  const int cell0 = grp * cb;
  dg_integrate_body<T, N, CURVED>(a, vec_ptrs(a, vec), cell0, min(cb, a.ncells - cell0),
                                  reinterpret_cast<T *>(smem_raw));
}

// Unstructured meshes: single-vector passes with general (curved) cell and
// face geometry and the neighbour of every local face from a.ufn.
template <typename T, int N>
__global__ void __launch_bounds__(kCellThreads, kMinCellBlocks<T>) dg_eval_unstr_kernel(const DGArgs<T> a, const int cb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int cell0 = blockIdx.x * cb;
  dg_eval_body<T, N, true, true>(a, vec_ptrs(a, 0), cell0, min(cb, a.ncells - cell0), reinterpret_cast<T *>(smem_raw));
}

template <typename T, int N>
__global__ void __launch_bounds__(kCellThreads, kMinCellBlocks<T>) dg_integrate_unstr_kernel(const DGArgs<T> a,
                                                                                            const int cb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int cell0 = blockIdx.x * cb;
  dg_integrate_body<T, N, true, true>(a, vec_ptrs(a, 0), cell0, min(cb, a.ncells - cell0),
                                      reinterpret_cast<T *>(smem_raw));
}

// Diagonal of the DG operator (setup, FP64), one thread per DoF: the cell
// term sum_q grad N_i^T M_q grad N_i and the face self-coupling
// dA (tau N_i^2 - N_i d_n N_i) on interior faces, dA (2 tau N_i^2 - 2 N_i d_n N_i)
// on Dirichlet faces.
struct DiagTabs {
  double S[81], Sd[81], lp0[9], lp1[9];
};

template <int N, bool CURVED>
__global__ void dg_diag_kernel(const DGArgs<double> a, const DiagTabs tb, double *diag) {
  constexpr int N2 = N * N, N3 = N2 * N;
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)a.ncells * N3) return;
  const int cell = (int)(idx / N3), i = (int)(idx - (long)cell * N3);
  const int ii[3] = {i % N, (i / N) % N, i / N2};
  const int ijk[3] = {cell % a.m[0], (cell / a.m[0]) % a.m[1], cell / (a.m[0] * a.m[1])};
  double sum = 0;
  for (int qz = 0; qz < N; ++qz)
    for (int qy = 0; qy < N; ++qy)
      for (int qx = 0; qx < N; ++qx) {
        const int p = qx + N * qy + N2 * qz;
        const double sx = tb.S[qx * N + ii[0]], sy = tb.S[qy * N + ii[1]], sz = tb.S[qz * N + ii[2]];
        const double g0 = tb.Sd[qx * N + ii[0]] * sy * sz;
        const double g1 = sx * tb.Sd[qy * N + ii[1]] * sz;
        const double g2 = sx * sy * tb.Sd[qz * N + ii[2]];
        if (!CURVED) {
          sum += a.wcart[p] * g0 * g0 + a.wcart[N3 + p] * g1 * g1 + a.wcart[2 * N3 + p] * g2 * g2;
        } else {
          const double *M = a.metric + (size_t)cell * 6 * N3 + p;
          sum += M[0] * g0 * g0 + M[N3] * g1 * g1 + M[2 * N3] * g2 * g2 +
                 2.0 * (M[3 * N3] * g0 * g1 + M[4 * N3] * g0 * g2 + M[5 * N3] * g1 * g2);
        }
      }
  const int cstride[3] = {1, a.m[0], a.m[0] * a.m[1]};
  for (int d = 0; d < 3; ++d) {
    const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
    for (int s = 0; s < 2; ++s) {
      if (ii[d] != (s ? N - 1 : 0)) continue;   // basis vanishes on this face
      const bool has_nb = s ? (ijk[d] < a.m[d] - 1) : (ijk[d] > 0);
      if (!has_nb && a.bc[2 * d + s] != 0) continue;   // Neumann: no term
      const double tau_e = a.tau[cell];
      const double tau_f = has_nb ? fmax(tau_e, a.tau[cell + (s ? cstride[d] : -cstride[d])]) : tau_e;
      const double lp = s ? tb.lp1[ii[d]] : tb.lp0[ii[d]];
      const size_t nfp = (size_t)a.m[t1] * a.m[t2];
      const size_t face = (size_t)(ijk[d] + s) * nfp + ijk[t1] + (size_t)a.m[t1] * ijk[t2];
      for (int q2 = 0; q2 < N; ++q2)
        for (int q1 = 0; q1 < N; ++q1) {
          const int lq = q1 + N * q2;
          const double s1 = tb.S[q1 * N + ii[t1]], s2 = tb.S[q2 * N + ii[t2]];
          const double nv = s1 * s2;
          double dA, dn;
          if (!CURVED) {
            dA = a.fwcart[d * N2 + lq];
            dn = (s ? a.ih[d] : -a.ih[d]) * lp * nv;
          } else {
            dA = a.fdA[d][face * N2 + lq];
            const double *c = a.fc[d] + (face * 2 + (s ? 0 : 1)) * 3 * N2 + lq;
            double gr[3];
            gr[d] = lp * nv;
            gr[t1] = tb.Sd[q1 * N + ii[t1]] * s2;
            gr[t2] = s1 * tb.Sd[q2 * N + ii[t2]];
            dn = c[0] * gr[0] + c[N2] * gr[1] + c[2 * N2] * gr[2];
          }
          if (has_nb)
            sum += dA * (tau_f * nv * nv - nv * dn);
          else
            sum += dA * (2.0 * tau_e * nv * nv - 2.0 * nv * dn);
        }
    }
  }
  diag[idx] = sum;
}

}  // namespace sipg
