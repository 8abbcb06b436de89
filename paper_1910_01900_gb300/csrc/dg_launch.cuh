// Launchers of the DG passes: dispatch over the runtime tile size n and the
// geometry kind to the compile-time kernels.  Included once per precision.
#pragma once
#include "dg_kernels.cuh"

namespace sipg {

template <typename T, int N, bool CURVED>
static cudaError_t run_dg(bool integrate, const DGArgs<T> &a, cudaStream_t s, int cb) {
  if (cb <= 0) cb = default_cb(N);
  if (cb > max_cb(N, sizeof(T))) return cudaErrorInvalidValue;
  const size_t smem = (size_t)cb * Tile<N>::CS * sizeof(T);
  const int64_t grid = (int64_t)((a.ncells + cb - 1) / cb) * a.nv;
  if (grid == 0) return cudaSuccess;
  if (grid > 0x7fffffff) return cudaErrorInvalidValue;
  if (a.ufn) {   // unstructured mesh: general geometry, single vector
    if (!CURVED || a.nv != 1) return cudaErrorInvalidValue;
    if (integrate)
      dg_integrate_unstr_kernel<T, N><<<(unsigned)grid, cb * N * N, smem, s>>>(a, cb);
    else
      dg_eval_unstr_kernel<T, N><<<(unsigned)grid, cb * N * N, smem, s>>>(a, cb);
  } else if (a.nv > 1) {
    if (integrate)
      dg_integrate_kernel<T, N, CURVED, true><<<(unsigned)grid, cb * N * N, smem, s>>>(a, cb);
    else
      dg_eval_kernel<T, N, CURVED, true><<<(unsigned)grid, cb * N * N, smem, s>>>(a, cb);
  } else {
    if (integrate)
      dg_integrate_kernel<T, N, CURVED, false><<<(unsigned)grid, cb * N * N, smem, s>>>(a, cb);
    else
      dg_eval_kernel<T, N, CURVED, false><<<(unsigned)grid, cb * N * N, smem, s>>>(a, cb);
  }
  note_launch();
  return cudaGetLastError();
}

// Resident thread blocks per SM of one pass at cb cells per block.
template <typename T, int N, bool CURVED>
static cudaError_t occ_dg(bool integrate, int cb, int *blocks) {
  const size_t smem = (size_t)cb * Tile<N>::CS * sizeof(T);
  return integrate ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, dg_integrate_kernel<T, N, CURVED, false>,
                                                                   cb * N * N, smem)
                   : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, dg_eval_kernel<T, N, CURVED, false>,
                                                                   cb * N * N, smem);
}

// Opt every kernel into the shared memory of its widest block (once per
// device, before any launch or stream capture).
template <typename T, int N>
static cudaError_t prep_dg_n() {
  const int smem = max_cb(N, sizeof(T)) * Tile<N>::CS * (int)sizeof(T);
  cudaError_t e = cudaSuccess;
  for (cudaError_t r :
       {cudaFuncSetAttribute(dg_integrate_kernel<T, N, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
        cudaFuncSetAttribute(dg_integrate_kernel<T, N, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
        cudaFuncSetAttribute(dg_eval_kernel<T, N, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
        cudaFuncSetAttribute(dg_eval_kernel<T, N, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
        cudaFuncSetAttribute(dg_integrate_kernel<T, N, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
        cudaFuncSetAttribute(dg_integrate_kernel<T, N, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
        cudaFuncSetAttribute(dg_eval_kernel<T, N, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
        cudaFuncSetAttribute(dg_eval_kernel<T, N, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
        cudaFuncSetAttribute(dg_integrate_unstr_kernel<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
        cudaFuncSetAttribute(dg_eval_unstr_kernel<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)})
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

// pass 0 evaluation, 1 integration; op 0 launch, 1 occupancy query into *blocks
template <typename T>
static cudaError_t dispatch_dg(int pass, int op, int n, bool curved, const DGArgs<T> *a, cudaStream_t s, int cb,
                               int *blocks = nullptr) {
#define SIPG_DG_CASE(NN)                                                                            \
  case NN:                                                                                          \
    if (op == 1)                                                                                    \
      return curved ? occ_dg<T, NN, true>(pass == 1, cb, blocks) : occ_dg<T, NN, false>(pass == 1, cb, blocks); \
    return curved ? run_dg<T, NN, true>(pass == 1, *a, s, cb) : run_dg<T, NN, false>(pass == 1, *a, s, cb);
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
