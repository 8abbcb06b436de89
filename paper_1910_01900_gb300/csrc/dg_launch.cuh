// Launchers of the DG passes: dispatch over the runtime tile size n and the
// geometry kind to the compile-time kernels.  Included once per precision.
#pragma once
#include "dg_kernels.cuh"

namespace sipg {

template <typename T, int N, bool CURVED, int CB>
static cudaError_t run_dg(bool integrate, const DGArgs<T> &a, cudaStream_t s) {
  const size_t smem = (size_t)CB * 4 * Tile<N>::T3 * sizeof(T);
  const int grid = (a.ncells + CB - 1) / CB;
  if (grid == 0) return cudaSuccess;
  if (integrate)
    dg_integrate_kernel<T, N, CURVED, CB><<<grid, CB * N * N, smem, s>>>(a);
  else
    dg_eval_kernel<T, N, CURVED, CB><<<grid, CB * N * N, smem, s>>>(a);
  note_launch();
  return cudaGetLastError();
}

// Opt every compiled tile shape into its dynamic shared memory size (once per
// device, before any launch or stream capture).
template <typename T, int N, bool CURVED, int CB>
static cudaError_t prep_dg() {
  const int smem = CB * 4 * Tile<N>::T3 * (int)sizeof(T);
  cudaError_t e = cudaFuncSetAttribute(dg_integrate_kernel<T, N, CURVED, CB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(dg_eval_kernel<T, N, CURVED, CB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

template <typename T, int N>
static cudaError_t prep_dg_n() {
  constexpr int D = default_cb(N);
  cudaError_t e = cudaSuccess;
  for (cudaError_t r : {prep_dg<T, N, false, D>(), prep_dg<T, N, true, D>(), prep_dg<T, N, false, 1>(),
                        prep_dg<T, N, true, 1>(), prep_dg<T, N, false, 2 * D>(), prep_dg<T, N, true, 2 * D>(),
                        prep_dg<T, N, false, (D + 1) / 2>(), prep_dg<T, N, true, (D + 1) / 2>()})
    if (r != cudaSuccess) e = r;
  return e;
}

template <typename T>
static cudaError_t prep_dg_all() {
  cudaError_t e = cudaSuccess;
  for (cudaError_t r : {prep_dg_n<T, 2>(), prep_dg_n<T, 3>(), prep_dg_n<T, 4>(), prep_dg_n<T, 5>(),
                        prep_dg_n<T, 6>(), prep_dg_n<T, 7>(), prep_dg_n<T, 8>(), prep_dg_n<T, 9>()})
    if (r != cudaSuccess) e = r;
  return e;
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
