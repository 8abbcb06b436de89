// Launchers of the DG passes: dispatch over the runtime tile size n and the
// geometry kind to the compile-time kernels.  Included once per precision.
#pragma once
#include "dg_kernels.cuh"

namespace sipg {

template <typename T, int N, bool CURVED, int CB>
static cudaError_t run_dg(bool integrate, const DGArgs<T> &a, cudaStream_t s) {
  constexpr int N3 = N * N * N;
  const size_t smem = (size_t)CB * 4 * N3 * sizeof(T);
  const int grid = (a.ncells + CB - 1) / CB;
  if (grid == 0) return cudaSuccess;
  if (integrate) {
    auto k = dg_integrate_kernel<T, N, CURVED, CB>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, CB * N * N, smem, s>>>(a);
  } else {
    auto k = dg_eval_kernel<T, N, CURVED, CB>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, CB * N * N, smem, s>>>(a);
  }
  return cudaGetLastError();
}

template <typename T, int N, bool CURVED>
static cudaError_t run_dg_cb(bool integrate, const DGArgs<T> &a, cudaStream_t s, int cb) {
  // a few tile widths per n for the autotuner; 0 = default
  constexpr int D = default_cb(N);
  if (cb == 0 || cb == D) return run_dg<T, N, CURVED, D>(integrate, a, s);
  if (cb == 1) return run_dg<T, N, CURVED, 1>(integrate, a, s);
  if (cb == 2 * D) return run_dg<T, N, CURVED, 2 * D>(integrate, a, s);
  if (cb == (D + 1) / 2) return run_dg<T, N, CURVED, (D + 1) / 2>(integrate, a, s);
  return cudaErrorInvalidValue;
}

template <typename T>
static cudaError_t dispatch_dg(bool integrate, int n, bool curved, const DGArgs<T> &a, cudaStream_t s, int cb) {
#define SIPG_DG_CASE(NN)                                                        \
  case NN:                                                                      \
    return curved ? run_dg_cb<T, NN, true>(integrate, a, s, cb)                 \
                  : run_dg_cb<T, NN, false>(integrate, a, s, cb);
  switch (n) {
    SIPG_DG_CASE(2)
    SIPG_DG_CASE(3)
    SIPG_DG_CASE(4)
    SIPG_DG_CASE(5)
    SIPG_DG_CASE(6)
    SIPG_DG_CASE(7)
    SIPG_DG_CASE(8)
    SIPG_DG_CASE(9)
    default:
      return cudaErrorInvalidValue;
  }
#undef SIPG_DG_CASE
}

}  // namespace sipg
