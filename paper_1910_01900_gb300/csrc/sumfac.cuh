// Sum-factorisation building blocks (Section 4: interpolation and
// integration as 1D sweeps over the tensor-product structure, even-odd
// decomposition of the 1D matrices).
//
// A 1D sweep applies an n x n matrix along one direction of an n^3 tile in
// shared memory; one thread handles one line of n points.  The matrices of a
// symmetric basis on symmetric points satisfy M[i][j] = s M[n-1-i][n-1-j]
// (s = +1 interpolation, s = -1 derivative), so y = M x splits into an even
// part (x_j + x_{n-1-j}) and an odd part (x_j - x_{n-1-j}) with half the
// multiplications.  The split costs 2n additions, so it only saves FP64
// instructions for n >= 5; for n <= 4 the plain product is used.
#pragma once
#include "sipg_internal.h"

namespace sipg {

// Each translation unit owns its copy of the tables (static __constant__).
static __constant__ Tables<double> c_tab_d;
static __constant__ Tables<float> c_tab_f;

template <typename T>
__device__ __forceinline__ const Tables<T> &tab();
template <>
__device__ __forceinline__ const Tables<double> &tab<double>() { return c_tab_d; }
template <>
__device__ __forceinline__ const Tables<float> &tab<float>() { return c_tab_f; }

template <typename T>
static void upload_tables_tu(const Tables<T> &t) {
  if constexpr (sizeof(T) == 8)
    cudaMemcpyToSymbol(c_tab_d, &t, sizeof(t));
  else
    cudaMemcpyToSymbol(c_tab_f, &t, sizeof(t));
}

// y = M x for one line; P plain matrix (n <= 4), E/O even-odd blocks (n >= 5).
template <typename T, int N, int PAR>
__device__ __forceinline__ void mv(const T *__restrict__ P, const T *__restrict__ E,
                                   const T *__restrict__ O, const T (&x)[N], T (&y)[N]) {
  if constexpr (N <= 4) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      T s = P[i * N] * x[0];
#pragma unroll
      for (int j = 1; j < N; ++j) s = fma(P[i * N + j], x[j], s);
      y[i] = s;
    }
  } else {
    constexpr int H = N / 2, HC = (N + 1) / 2;
    T e[HC], o[H];
#pragma unroll
    for (int j = 0; j < H; ++j) {
      e[j] = x[j] + x[N - 1 - j];
      o[j] = x[j] - x[N - 1 - j];
    }
    if constexpr (N & 1) e[H] = x[H];
#pragma unroll
    for (int i = 0; i < H; ++i) {
      T se = E[i * 5] * e[0];
#pragma unroll
      for (int j = 1; j < HC; ++j) se = fma(E[i * 5 + j], e[j], se);
      T so = O[i * 4] * o[0];
#pragma unroll
      for (int j = 1; j < H; ++j) so = fma(O[i * 4 + j], o[j], so);
      if constexpr (PAR > 0) {
        y[i] = se + so;
        y[N - 1 - i] = se - so;
      } else {
        y[i] = se + so;
        y[N - 1 - i] = so - se;
      }
    }
    if constexpr (N & 1) {
      if constexpr (PAR > 0) {
        T s = E[H * 5] * e[0];
#pragma unroll
        for (int j = 1; j < HC; ++j) s = fma(E[H * 5 + j], e[j], s);
        y[H] = s;
      } else {
        T s = O[H * 4] * o[0];
#pragma unroll
        for (int j = 1; j < H; ++j) s = fma(O[H * 4 + j], o[j], s);
        y[H] = s;
      }
    }
  }
}

// Matrix selectors (compile-time n).
enum Mat { MS = 0, MSt = 1, MD = 2, MDt = 3, MM1 = 4, MK1 = 5, MKG = 6 };
template <typename T, int N, int M>
__device__ __forceinline__ void apply_mat(const T (&x)[N], T (&y)[N]) {
  const Tables<T> &t = tab<T>();
  if constexpr (M == MS) mv<T, N, +1>(t.S[N], t.SE[N], t.SO[N], x, y);
  if constexpr (M == MSt) mv<T, N, +1>(t.St[N], t.StE[N], t.StO[N], x, y);
  if constexpr (M == MD) mv<T, N, -1>(t.D[N], t.DE[N], t.DO[N], x, y);
  if constexpr (M == MDt) mv<T, N, -1>(t.Dt[N], t.DtE[N], t.DtO[N], x, y);
  if constexpr (M == MM1) mv<T, N, +1>(t.M1[N], t.M1E[N], t.M1O[N], x, y);
  if constexpr (M == MK1) mv<T, N, +1>(t.K1[N], t.K1E[N], t.K1O[N], x, y);
  if constexpr (M == MKG) mv<T, N, +1>(t.KG[N], t.KGE[N], t.KGO[N], x, y);
}

// Shared-memory layout of one cell: four tile arrays of N^3 values (x
// fastest, y step XP, z step ZP, array stride T3 = ZP N), cells CS values
// apart.  One thread walks one line per sweep; a warp's 32 lanes cover lines
// of up to two cells, and the lines of different directions start at
// different banks.  The pitches below were chosen, per N, by counting the
// shared-memory wavefronts (the most threads of a warp on one bank) of the
// three sweep directions and of the point loops at the default and half the
// default cells per block: 1.57 wavefronts per FP32 instruction at N = 6
// against 1.85 with the x pitch alone padded (N + 1 for even N), 1.72 against
// 3.7 at N = 2, 1.43 against 2.0 at N = 4.  The layout moves addresses only:
// every value is computed by the same thread in the same order.
__host__ __device__ constexpr int tile_xp(int n) { return n == 8 ? 9 : n; }
__host__ __device__ constexpr int tile_zp(int n) {
  return n == 2 ? 4 : n == 3 ? 9 : n == 4 ? 19 : n == 5 ? 25 : n == 6 ? 39 : n == 7 ? 52 : n == 8 ? 72 : 81;
}
// values of shared memory per cell (>= 4 tile arrays)
__host__ __device__ constexpr int cell_values(int n) {
  return n == 2 ? 36 : n == 3 ? 123 : n == 4 ? 304 : n == 5 ? 509 : n == 6 ? 964 : n == 7 ? 1457 : n == 8 ? 2304 : 2929;
}

template <int N>
struct Tile {
  static constexpr int XP = tile_xp(N);                  // step of y
  static constexpr int ZP = tile_zp(N);                  // step of z
  static constexpr int T3 = ZP * N;                      // values per tile array
  static constexpr int CS = cell_values(N);              // values per cell
  static_assert(XP >= N && ZP >= XP * N && CS >= 4 * T3, "tile arrays overlap");
  // tile position of the node or point with linear index p = x + N (y + N z)
  static __device__ __forceinline__ int idx(int p) {
    const int x = p % N, y = (p / N) % N, z = p / (N * N);
    return x + XP * y + ZP * z;
  }
};

// Offset and stride of line l (0 <= l < N^2) along direction d in a tile.
// The line index l = a + N*b runs over the two other directions in increasing
// order, so it equals the face-point index of the faces normal to d.
template <int N>
__device__ __forceinline__ void line_of(int d, int l, int &base, int &stride) {
  constexpr int XP = Tile<N>::XP, ZP = Tile<N>::ZP;
  const int a = l % N, b = l / N;
  if (d == 0) {
    base = XP * a + ZP * b;
    stride = 1;
  } else if (d == 1) {
    base = a + ZP * b;
    stride = XP;
  } else {
    base = a + XP * b;
    stride = ZP;
  }
}

template <typename T, int N>
__device__ __forceinline__ void load_line(const T *s, int base, int stride, T (&x)[N]) {
#pragma unroll
  for (int q = 0; q < N; ++q) x[q] = s[base + q * stride];
}
template <typename T, int N>
__device__ __forceinline__ void store_line(T *s, int base, int stride, const T (&x)[N]) {
#pragma unroll
  for (int q = 0; q < N; ++q) s[base + q * stride] = x[q];
}

// In-place sweep of matrix M along d on the tile s (one line per thread).
template <typename T, int N, int M>
__device__ __forceinline__ void sweep_inplace(T *s, int d, int l) {
  int base, stride;
  line_of<N>(d, l, base, stride);
  T x[N], y[N];
  load_line<T, N>(s, base, stride, x);
  apply_mat<T, N, M>(x, y);
  store_line<T, N>(s, base, stride, y);
}


// Most threads per block of the cell kernels (their __launch_bounds__: at
// most 85 registers a thread, which the sweeps need without spilling).
constexpr int kCellThreads = 768;

// Largest cells per thread block of the cell kernels (cell_values(n) values
// of shared memory per cell): kCellThreads threads and 227 KB of shared memory.
__host__ __device__ constexpr int max_cb(int n, int elem_bytes) {
  return (kCellThreads / (n * n)) < (232448 / (cell_values(n) * elem_bytes))
             ? (kCellThreads / (n * n))
             : (232448 / (cell_values(n) * elem_bytes));
}

// Cells per thread block for a tile size n (about 256 threads, n^2 threads per cell).
__host__ __device__ constexpr int default_cb(int n) {
  return n == 2 ? 64 : n == 3 ? 28 : n == 4 ? 16 : n == 5 ? 10 : n == 6 ? 7 : n == 7 ? 5 : n == 8 ? 4 : 3;
}

}  // namespace sipg
