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
enum Mat { MS = 0, MSt = 1, MD = 2, MDt = 3 };
template <typename T, int N, int M>
__device__ __forceinline__ void apply_mat(const T (&x)[N], T (&y)[N]) {
  const Tables<T> &t = tab<T>();
  if constexpr (M == MS) mv<T, N, +1>(t.S[N], t.SE[N], t.SO[N], x, y);
  if constexpr (M == MSt) mv<T, N, +1>(t.St[N], t.StE[N], t.StO[N], x, y);
  if constexpr (M == MD) mv<T, N, -1>(t.D[N], t.DE[N], t.DO[N], x, y);
  if constexpr (M == MDt) mv<T, N, -1>(t.Dt[N], t.DtE[N], t.DtO[N], x, y);
}

// Shared-memory tile of N^3 values, x fastest, with the x pitch padded to an
// odd number for even N: a warp walking lines along x then hits distinct
// banks (an even pitch like 8 puts 4-8 threads on one bank).
template <int N>
struct Tile {
  static constexpr int XP = (N % 2 == 0) ? N + 1 : N;   // pitch of a y step
  static constexpr int T3 = XP * N * N;                  // values per tile array
  // tile position of the node or point with linear index p = x + N (y + N z)
  static __device__ __forceinline__ int idx(int p) { return XP == N ? p : p + p / N; }
};

// Offset and stride of line l (0 <= l < N^2) along direction d in a tile.
// The line index l = a + N*b runs over the two other directions in increasing
// order, so it equals the face-point index of the faces normal to d.
template <int N>
__device__ __forceinline__ void line_of(int d, int l, int &base, int &stride) {
  constexpr int XP = Tile<N>::XP;
  const int a = l % N, b = l / N;
  if (d == 0) {
    base = XP * (a + N * b);
    stride = 1;
  } else if (d == 1) {
    base = a + XP * N * b;
    stride = XP;
  } else {
    base = a + XP * b;
    stride = XP * N;
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

// Values of one padded tile array for n points per direction (host and device).
__host__ __device__ constexpr int tile_values(int n) { return ((n % 2 == 0) ? n + 1 : n) * n * n; }

// Most threads per block of the cell kernels (their __launch_bounds__: at
// most 85 registers a thread, which the sweeps need without spilling).
constexpr int kCellThreads = 768;

// Largest cells per thread block of the cell kernels (four tile arrays of
// shared memory per cell): kCellThreads threads and 227 KB of shared memory.
__host__ __device__ constexpr int max_cb(int n, int elem_bytes) {
  return (kCellThreads / (n * n)) < (232448 / (4 * tile_values(n) * elem_bytes))
             ? (kCellThreads / (n * n))
             : (232448 / (4 * tile_values(n) * elem_bytes));
}

// Cells per thread block for a tile size n (about 256 threads, n^2 threads per cell).
__host__ __device__ constexpr int default_cb(int n) {
  return n == 2 ? 64 : n == 3 ? 28 : n == 4 ? 16 : n == 5 ? 10 : n == 6 ? 7 : n == 7 ? 5 : n == 8 ? 4 : 3;
}

}  // namespace sipg
