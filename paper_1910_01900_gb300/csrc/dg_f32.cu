// FP32 instantiation of the DG passes (mixed-precision V-cycle, Section 4).
#include "dg_launch.cuh"

namespace sipg {

template <>
void upload_tables_dg<float>(const Tables<float> &t) { upload_tables_tu(t); }
template <>
cudaError_t launch_dg_eval<float>(int n, bool curved, const DGArgs<float> &a, cudaStream_t s, int cb) {
  return dispatch_dg<float>(0, 0, n, curved, &a, s, cb);
}
template <>
cudaError_t launch_dg_integrate<float>(int n, bool curved, const DGArgs<float> &a, cudaStream_t s, int cb) {
  return dispatch_dg<float>(1, 0, n, curved, &a, s, cb);
}
template <>
int dg_cells_per_block<float>(int n) { return default_cb(n); }
template <>
int dg_max_cells_per_block<float>(int n) { return max_cb(n, sizeof(float)); }
template <>
cudaError_t dg_blocks_per_sm<float>(int n, bool curved, int pass, int cb, int *blocks) {
  return dispatch_dg<float>(pass, 1, n, curved, nullptr, nullptr, cb, blocks);
}
template <>
cudaError_t prepare_dg_kernels<float>() { return prep_dg_all<float>(); }

}  // namespace sipg
