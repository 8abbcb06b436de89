// Many independent SIPG problems (uneven mesh size and degree) or many
// right-hand sides of one problem, solved together.
//
// * The finest-level DG operator of all problems runs as ONE persistent
//   launch per pass: a fixed grid (SMs x resident blocks) walks a static list
//   of work items (problem, first cell, cell count), longest first, and
//   dispatches each item to the sum-factorisation body of that problem's
//   degree.  The same bodies as the per-problem kernels (dg_kernels.cuh).
// * The flexible-CG iterations of all problems run in lockstep: batched
//   operator applications, batched inner products and updates (one launch for
//   all problems, deterministic per-problem reductions), and each problem's
//   V-cycle replayed from its CUDA graph on its own stream, so the cycles of
//   different problems overlap on the GPU.
// Not in the paper (its solver handles one problem per run); the method per
// problem is unchanged.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "dg_kernels.cuh"

namespace sipg {

constexpr int kBatchThreads = 256;

// this translation unit's copy of the 1D tables (constant memory is per unit)
template <>
void upload_tables_batch<double>(const Tables<double> &t) { upload_tables_tu(t); }
template <>
void upload_tables_batch<float>(const Tables<float> &t) { upload_tables_tu(t); }

template <typename T, bool CURVED, bool INTEGRATE>
__global__ void __launch_bounds__(kBatchThreads)
    dg_batched_kernel(const BatchProb<T> *__restrict__ probs, const WorkItem *__restrict__ items, int nitems) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sm = reinterpret_cast<T *>(smem_raw);
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const WorkItem w = items[it];
    const BatchProb<T> &P = probs[w.p];
    if (P.active) {
#define SIPG_BATCH_CASE(NN)                                              \
  case NN:                                                               \
    if (INTEGRATE)                                                       \
      dg_integrate_body<T, NN, CURVED>(P.a, vec_ptrs(P.a, 0), w.cell0, w.ncta, sm); \
    else                                                                 \
      dg_eval_body<T, NN, CURVED>(P.a, vec_ptrs(P.a, 0), w.cell0, w.ncta, sm); \
    break;
      switch (P.n) {
        SIPG_BATCH_CASE(2)
        SIPG_BATCH_CASE(3)
        SIPG_BATCH_CASE(4)
        SIPG_BATCH_CASE(5)
        SIPG_BATCH_CASE(6)
        SIPG_BATCH_CASE(7)
        SIPG_BATCH_CASE(8)
        SIPG_BATCH_CASE(9)
        default:
          break;
      }
#undef SIPG_BATCH_CASE
    }
    __syncthreads();
  }
}

constexpr int kSegBlocks = kSegBlocksHost;   // blocks per system in the batched reductions

__device__ void seg_reduce2(double a, double b, double *partials, unsigned *counter, double *out) {
  // blocks (p, j), j < kSegBlocks: partial sums per block, the last block of
  // the problem sums them in order (deterministic) and resets the counter
  __shared__ double sa[256], sb[256];
  __shared__ bool last;
  const int p = blockIdx.x / kSegBlocks, j = blockIdx.x % kSegBlocks;
  sa[threadIdx.x] = a;
  sb[threadIdx.x] = b;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sa[threadIdx.x] += sa[threadIdx.x + w];
      sb[threadIdx.x] += sb[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[(p * kSegBlocks + j) * 2] = sa[0];
    partials[(p * kSegBlocks + j) * 2 + 1] = sb[0];
    __threadfence();
    last = atomicAdd(&counter[p], 1u) == kSegBlocks - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x == 0) {
    double ta = 0, tb = 0;
    for (int q = 0; q < kSegBlocks; ++q) {
      ta += ((volatile double *)partials)[(p * kSegBlocks + q) * 2];
      tb += ((volatile double *)partials)[(p * kSegBlocks + q) * 2 + 1];
    }
    out[0] = ta;
    out[1] = tb;
    counter[p] = 0;
  }
}

// which: 0 -> (b.b, r.r); 1 -> (r.z, 0); 2 -> (p.v, 0); 3 -> (r.z, z.v)
__global__ void seg_dot_kernel(const Seg *segs, int which, double *partials, unsigned *counter, double *sc,
                               int sc_stride, int slot) {
  const int p = blockIdx.x / kSegBlocks, j = blockIdx.x % kSegBlocks;
  const Seg S = segs[p];
  if (!S.active) return;   // whole problem inactive: every block of it returns
  double a = 0, b = 0;
  for (long i = (long)j * blockDim.x + threadIdx.x; i < S.n; i += (long)kSegBlocks * blockDim.x) {
    if (which == 0) {
      a = fma(S.b[i], S.b[i], a);
      b = fma(S.r[i], S.r[i], b);
    } else if (which == 1) {
      a = fma(S.r[i], S.z[i], a);
    } else if (which == 2) {
      a = fma(S.p[i], S.v[i], a);
    } else {
      a = fma(S.r[i], S.z[i], a);
      b = fma(S.z[i], S.v[i], b);
    }
  }
  seg_reduce2(a, b, partials, counter, sc + (size_t)p * sc_stride + slot);
}

// x += alpha p, r -= alpha v, alpha = sc[0]/sc[2]; sc[3] = r.r
__global__ void seg_update_xr_kernel(const Seg *segs, double *partials, unsigned *counter, double *sc,
                                     int sc_stride) {
  const int p = blockIdx.x / kSegBlocks, j = blockIdx.x % kSegBlocks;
  const Seg S = segs[p];
  if (!S.active) return;
  const double *s = sc + (size_t)p * sc_stride;
  const double alpha = s[0] / s[2];
  double a = 0;
  for (long i = (long)j * blockDim.x + threadIdx.x; i < S.n; i += (long)kSegBlocks * blockDim.x) {
    S.x[i] = fma(alpha, S.p[i], S.x[i]);
    const double ri = fma(-alpha, S.v[i], S.r[i]);
    S.r[i] = ri;
    a = fma(ri, ri, a);
  }
  seg_reduce2(a, 0.0, partials, counter, sc + (size_t)p * sc_stride + 3);
}

// p = z + beta p, beta = -sc[1]/sc[2]; or p = z (init)
__global__ void seg_update_p_kernel(const Seg *segs, const double *sc, int sc_stride, int init) {
  const int p = blockIdx.x / kSegBlocks, j = blockIdx.x % kSegBlocks;
  const Seg S = segs[p];
  if (!S.active) return;
  const double *s = sc + (size_t)p * sc_stride;
  const double beta = init ? 0.0 : -s[1] / s[2];
  for (long i = (long)j * blockDim.x + threadIdx.x; i < S.n; i += (long)kSegBlocks * blockDim.x)
    S.p[i] = init ? S.z[i] : fma(beta, S.p[i], S.z[i]);
}

// ------------------------------------------------------------------ host side

template <typename T>
cudaError_t batch_plan_build(BatchPlan<T> &P, const std::vector<DGArgs<T>> &args, const std::vector<int> &ns) {
  const int np = (int)args.size();
  P.probs.resize(np);
  P.items.clear();
  size_t smem = 0;
  for (int p = 0; p < np; ++p) {
    P.probs[p].a = args[p];
    P.probs[p].n = ns[p];
    P.probs[p].active = 1;
    const int n = ns[p], cb = kBatchThreads / (n * n);
    smem = std::max(smem, (size_t)cb * cell_values(n) * sizeof(T));
    for (int c = 0; c < args[p].ncells; c += cb) P.items.push_back({p, c, std::min(cb, args[p].ncells - c)});
  }
  // longest items first (cost ~ cells x n^4), then static striding over the grid
  std::stable_sort(P.items.begin(), P.items.end(), [&](const WorkItem &x, const WorkItem &y) {
    const double cx = (double)x.ncta * std::pow((double)ns[x.p], 4), cy = (double)y.ncta * std::pow((double)ns[y.p], 4);
    return cx > cy;
  });
  P.smem = smem;
  cudaError_t e;
  if ((e = cudaMalloc(&P.d_probs, np * sizeof(BatchProb<T>))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&P.d_items, std::max<size_t>(1, P.items.size()) * sizeof(WorkItem))) != cudaSuccess) return e;
  if ((e = cudaMemcpy(P.d_items, P.items.data(), P.items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice)) !=
      cudaSuccess)
    return e;
  auto k0 = dg_batched_kernel<T, false, false>, k1 = dg_batched_kernel<T, false, true>;
  auto k2 = dg_batched_kernel<T, true, false>, k3 = dg_batched_kernel<T, true, true>;
  for (auto k : {k0, k1, k2, k3})
    if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
      return e;
  int dev, nsm, occ = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k1, kBatchThreads, smem);
  P.grid = std::max(1, std::min<int>((int)P.items.size(), nsm * std::max(1, occ)));
  return cudaSuccess;
}

template <typename T>
void batch_plan_free(BatchPlan<T> &P) {
  cudaFree(P.d_probs);
  cudaFree(P.d_items);
  P.d_probs = nullptr;
  P.d_items = nullptr;
}

// Upload the current descriptors (pointers, modes, active flags) and run both
// passes as two persistent launches.
template <typename T>
cudaError_t batch_apply(BatchPlan<T> &P, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(P.d_probs, P.probs.data(), P.probs.size() * sizeof(BatchProb<T>),
                                  cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  if (P.items.empty()) return cudaSuccess;
  if (P.curved) {
    dg_batched_kernel<T, true, false><<<P.grid, kBatchThreads, P.smem, s>>>(P.d_probs, P.d_items, (int)P.items.size());
    dg_batched_kernel<T, true, true><<<P.grid, kBatchThreads, P.smem, s>>>(P.d_probs, P.d_items, (int)P.items.size());
  } else {
    dg_batched_kernel<T, false, false><<<P.grid, kBatchThreads, P.smem, s>>>(P.d_probs, P.d_items, (int)P.items.size());
    dg_batched_kernel<T, false, true><<<P.grid, kBatchThreads, P.smem, s>>>(P.d_probs, P.d_items, (int)P.items.size());
  }
  note_launch();
  note_launch();
  return cudaGetLastError();
}

template cudaError_t batch_plan_build<double>(BatchPlan<double> &, const std::vector<DGArgs<double>> &,
                                              const std::vector<int> &);
template cudaError_t batch_plan_build<float>(BatchPlan<float> &, const std::vector<DGArgs<float>> &,
                                             const std::vector<int> &);
template void batch_plan_free<double>(BatchPlan<double> &);
template void batch_plan_free<float>(BatchPlan<float> &);
template cudaError_t batch_apply<double>(BatchPlan<double> &, cudaStream_t);
template cudaError_t batch_apply<float>(BatchPlan<float> &, cudaStream_t);

cudaError_t seg_dot(const Seg *segs, int np, int which, double *partials, unsigned *counter, double *sc,
                    int sc_stride, int slot, cudaStream_t s) {
  seg_dot_kernel<<<np * kSegBlocks, 256, 0, s>>>(segs, which, partials, counter, sc, sc_stride, slot);
  note_launch();
  return cudaGetLastError();
}
cudaError_t seg_update_xr(const Seg *segs, int np, double *partials, unsigned *counter, double *sc, int sc_stride,
                          cudaStream_t s) {
  seg_update_xr_kernel<<<np * kSegBlocks, 256, 0, s>>>(segs, partials, counter, sc, sc_stride);
  note_launch();
  return cudaGetLastError();
}
cudaError_t seg_update_p(const Seg *segs, int np, const double *sc, int sc_stride, int init, cudaStream_t s) {
  seg_update_p_kernel<<<np * kSegBlocks, 256, 0, s>>>(segs, sc, sc_stride, init);
  note_launch();
  return cudaGetLastError();
}

}  // namespace sipg
