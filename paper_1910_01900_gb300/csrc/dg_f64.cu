// FP64 instantiation of the DG passes and the DG diagonal (setup).
#include "dg_launch.cuh"

namespace sipg {

template <>
void upload_tables_dg<double>(const Tables<double> &t) { upload_tables_tu(t); }
template <>
cudaError_t launch_dg_eval<double>(int n, bool curved, const DGArgs<double> &a, cudaStream_t s, int cb) {
  return dispatch_dg<double>(0, 0, n, curved, &a, s, cb);
}
template <>
cudaError_t launch_dg_integrate<double>(int n, bool curved, const DGArgs<double> &a, cudaStream_t s, int cb) {
  return dispatch_dg<double>(1, 0, n, curved, &a, s, cb);
}
template <>
int dg_cells_per_block<double>(int n) { return default_cb(n); }
template <>
int dg_max_cells_per_block<double>(int n) { return max_cb(n, sizeof(double)); }
template <>
cudaError_t dg_blocks_per_sm<double>(int n, bool curved, int pass, int cb, int *blocks) {
  return dispatch_dg<double>(pass, 1, n, curved, nullptr, nullptr, cb, blocks);
}
template <>
cudaError_t prepare_dg_kernels<double>() { return prep_dg_all<double>(); }

cudaError_t launch_dg_diag(int n, bool curved, const DGArgs<double> &a, double *diag, cudaStream_t s) {
  const Rules1D &r = rules(n);
  DiagTabs tb{};
  for (int i = 0; i < n * n; ++i) {
    tb.S[i] = r.S[i];
    tb.Sd[i] = r.Sd[i];
  }
  for (int i = 0; i < n; ++i) {
    tb.lp0[i] = r.lp0[i];
    tb.lp1[i] = r.lp1[i];
  }
  const long total = (long)a.ncells * n * n * n;
  const int bs = 128;
  const int grid = (int)((total + bs - 1) / bs);
  if (grid == 0) return cudaSuccess;
#define SIPG_DIAG_CASE(NN)                                                       \
  case NN:                                                                       \
    if (curved) dg_diag_kernel<NN, true><<<grid, bs, 0, s>>>(a, tb, diag);       \
    else dg_diag_kernel<NN, false><<<grid, bs, 0, s>>>(a, tb, diag);             \
    break;
  switch (n) {
    SIPG_DIAG_CASE(2)
    SIPG_DIAG_CASE(3)
    SIPG_DIAG_CASE(4)
    SIPG_DIAG_CASE(5)
    SIPG_DIAG_CASE(6)
    SIPG_DIAG_CASE(7)
    SIPG_DIAG_CASE(8)
    SIPG_DIAG_CASE(9)
    default:
      return cudaErrorInvalidValue;
  }
#undef SIPG_DIAG_CASE
  note_launch();
  return cudaGetLastError();
}

}  // namespace sipg
