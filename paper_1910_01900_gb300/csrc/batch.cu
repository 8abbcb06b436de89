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

// segs (optional): the flexible-CG systems; a problem whose system has left
// the iteration (segs[p].active == 0, set on the device) is skipped too
// (register budget as the single-problem passes: FP32, bound by shared
// memory traffic and latency, keeps 6 blocks of 256 threads resident)
template <typename T, bool CURVED, bool INTEGRATE>
__global__ void __launch_bounds__(kBatchThreads, sizeof(T) == 4 ? 6 : 3)
    dg_batched_kernel(const BatchProb<T> *__restrict__ probs, const WorkItem *__restrict__ items, int nitems,
                      const Seg *__restrict__ segs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sm = reinterpret_cast<T *>(smem_raw);
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const WorkItem w = items[it];
    const BatchProb<T> &P = probs[w.p];
    if (P.active && (!segs || segs[w.p].active)) {
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

// Blocks of the batched vector kernels: system p gets g.nb[p] blocks (one
// per kSegChunk entries, at least one), block b works on system g.map[b].x as
// its g.map[b].y-th block, so that a large system gets as many blocks as its
// size asks for and the launch is balanced over the GPU.

__device__ void seg_reduce2(const SegGrid &g, int p, int j, double a, double b, double *partials, unsigned *counter,
                            double *out) {
  // per block partial sums; the last block of the system sums them in block
  // order (deterministic) and resets the system's counter
  __shared__ double sa[256], sb[256];
  __shared__ bool last;
  const int nb = g.nb[p], off = g.off[p];
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
    partials[(off + j) * 2] = sa[0];
    partials[(off + j) * 2 + 1] = sb[0];
    __threadfence();
    last = atomicAdd(&counter[p], 1u) == (unsigned)nb - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x == 0) {
    double ta = 0, tb = 0;
    for (int q = 0; q < nb; ++q) {
      ta += ((volatile double *)partials)[(off + q) * 2];
      tb += ((volatile double *)partials)[(off + q) * 2 + 1];
    }
    out[0] = ta;
    out[1] = tb;
    counter[p] = 0;
  }
}

// which: 0 -> (b.b, r.r); 1 -> (r.z, 0); 2 -> (p.v, 0); 3 -> (r.z, z.v)
__global__ void seg_dot_kernel(const Seg *segs, const SegGrid g, int which, double *partials, unsigned *counter,
                               double *sc, int sc_stride, int slot) {
  const int p = g.map[blockIdx.x].x, j = g.map[blockIdx.x].y, nb = g.nb[p];
  const Seg S = segs[p];
  if (!S.active) return;   // whole system inactive: every block of it returns
  double a = 0, b = 0;
  for (long i = (long)j * blockDim.x + threadIdx.x; i < S.n; i += (long)nb * blockDim.x) {
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
  seg_reduce2(g, p, j, a, b, partials, counter, sc + (size_t)p * sc_stride + slot);
}

// x += alpha p, r -= alpha v, alpha = sc[0]/sc[2]; sc[3] = r.r
__global__ void seg_update_xr_kernel(const Seg *segs, const SegGrid g, double *partials, unsigned *counter, double *sc,
                                     int sc_stride) {
  const int p = g.map[blockIdx.x].x, j = g.map[blockIdx.x].y, nb = g.nb[p];
  const Seg S = segs[p];
  if (!S.active) return;
  const double *s = sc + (size_t)p * sc_stride;
  const double alpha = s[0] / s[2];
  double a = 0;
  for (long i = (long)j * blockDim.x + threadIdx.x; i < S.n; i += (long)nb * blockDim.x) {
    S.x[i] = fma(alpha, S.p[i], S.x[i]);
    const double ri = fma(-alpha, S.v[i], S.r[i]);
    S.r[i] = ri;
    a = fma(ri, ri, a);
  }
  seg_reduce2(g, p, j, a, 0.0, partials, counter, sc + (size_t)p * sc_stride + 3);
}

// p = z + beta p, beta = -sc[1]/sc[2]; or p = z (init)
__global__ void seg_update_p_kernel(const Seg *segs, const SegGrid g, const double *sc, int sc_stride, int init) {
  const int p = g.map[blockIdx.x].x, j = g.map[blockIdx.x].y, nb = g.nb[p];
  const Seg S = segs[p];
  if (!S.active) return;
  const double *s = sc + (size_t)p * sc_stride;
  const double beta = init ? 0.0 : -s[1] / s[2];
  for (long i = (long)j * blockDim.x + threadIdx.x; i < S.n; i += (long)nb * blockDim.x)
    S.p[i] = init ? S.z[i] : fma(beta, S.p[i], S.z[i]);
}

// ------------------------------------------ lockstep flexible CG gated on the device
// After x += alpha p, r -= alpha v of every active system: count the
// iteration, record ||r||, and take each system out of the iteration on
// convergence (||r|| <= rtol ||r_0||, the host loop's test), breakdown
// (status 1) or maxit (status 2); the next step's condition is 1 while any
// system is still active.  prm = {rtol, maxit} in device memory (the
// captured launch outlives one solve's arguments).  One block; systems
// strided over its threads.
__global__ void batch_fcg_check_kernel(const double *sc, int stride, Seg *segs, int np, int *it, int *status,
                                       double *hist, double *rn, const double *r0, const double *prm, int *any,
                                       cudaGraphConditionalHandle next) {
  const double rtol = prm[0];
  const int maxit = (int)prm[1];
  __shared__ int s_any;
  if (threadIdx.x == 0) s_any = 0;
  __syncthreads();
  int live = 0;
  for (int p = threadIdx.x; p < np; p += blockDim.x) {
    if (!segs[p].active) continue;
    const double *q = sc + (size_t)p * stride;
    const int k = it[p] + 1;
    it[p] = k;
    if (!(q[2] > 0) || !isfinite(q[3])) {
      segs[p].active = 0;
      status[p] = 1;
      continue;
    }
    const double r = sqrt(q[3]);
    rn[p] = r;
    if (k <= 256) hist[(size_t)p * 257 + k] = r;
    if (r <= rtol * r0[p]) {
      segs[p].active = 0;
    } else if (k >= maxit) {
      segs[p].active = 0;
      status[p] = 2;
    } else {
      live = 1;
    }
  }
  if (live) atomicOr(&s_any, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    *any = s_any;
    cudaGraphSetConditional(next, s_any ? 1u : 0u);
  }
}

__global__ void batch_fcg_cond_kernel(const int *any, cudaGraphConditionalHandle h) {
  cudaGraphSetConditional(h, *any ? 1u : 0u);
}

cudaError_t launch_batch_fcg_check(const double *sc, int stride, Seg *segs, int np, int *it, int *status, double *hist,
                                   double *rn, const double *r0, const double *prm, int *any,
                                   cudaGraphConditionalHandle next, cudaStream_t s) {
  batch_fcg_check_kernel<<<1, 256, 0, s>>>(sc, stride, segs, np, it, status, hist, rn, r0, prm, any, next);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_batch_fcg_cond(const int *any, cudaGraphConditionalHandle h, cudaStream_t s) {
  batch_fcg_cond_kernel<<<1, 1, 0, s>>>(any, h);
  note_launch();
  return cudaGetLastError();
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
cudaError_t batch_dg_pass(const BatchPlan<T> &P, const BatchProb<T> *probs, bool integrate, const Seg *segs,
                          cudaStream_t s);

template <typename T>
cudaError_t batch_apply(BatchPlan<T> &P, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(P.d_probs, P.probs.data(), P.probs.size() * sizeof(BatchProb<T>),
                                  cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  if (P.items.empty()) return cudaSuccess;
  if ((e = batch_dg_pass<T>(P, P.d_probs, false, nullptr, s)) != cudaSuccess) return e;
  return batch_dg_pass<T>(P, P.d_probs, true, nullptr, s);
}

// One pass over the plan's work items with the descriptors probs (device).
template <typename T>
cudaError_t batch_dg_pass(const BatchPlan<T> &P, const BatchProb<T> *probs, bool integrate, const Seg *segs,
                          cudaStream_t s) {
  const int ni = (int)P.items.size();
  if (ni == 0) return cudaSuccess;
  if (P.curved) {
    if (integrate) dg_batched_kernel<T, true, true><<<P.grid, kBatchThreads, P.smem, s>>>(probs, P.d_items, ni, segs);
    else dg_batched_kernel<T, true, false><<<P.grid, kBatchThreads, P.smem, s>>>(probs, P.d_items, ni, segs);
  } else {
    if (integrate) dg_batched_kernel<T, false, true><<<P.grid, kBatchThreads, P.smem, s>>>(probs, P.d_items, ni, segs);
    else dg_batched_kernel<T, false, false><<<P.grid, kBatchThreads, P.smem, s>>>(probs, P.d_items, ni, segs);
  }
  note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------- batched vector steps of the V-cycle
// op 0: y (FP32) = x (FP64); 1: y (FP64) = x (FP32); 2: y = c d x in FP32;
// 3: y = c d x in FP64; 4: y = x (FP64).  kBatchNodeThreads entries per item.
__global__ void __launch_bounds__(kBatchNodeThreads)
    vec_batched_kernel(const VecTask *__restrict__ tasks, const NodeItem *__restrict__ items,
                       const Seg *__restrict__ segs) {
  const NodeItem w = items[blockIdx.x];
  if (segs && !segs[w.p].active) return;
  const VecTask &V = tasks[w.p];
  const long i = (long)w.blk * kBatchNodeThreads + threadIdx.x;
  if (i >= V.n) return;
  switch (V.op) {
    case 0:
      ((float *)V.y)[i] = (float)((const double *)V.x)[i];
      break;
    case 1:
      ((double *)V.y)[i] = (double)((const float *)V.x)[i];
      break;
    case 2: {
      const float c = (float)V.c;
      ((float *)V.y)[i] = c * ((const float *)V.d)[i] * ((const float *)V.x)[i];
      break;
    }
    case 3:
      ((double *)V.y)[i] = V.c * ((const double *)V.d)[i] * ((const double *)V.x)[i];
      break;
    default:
      ((double *)V.y)[i] = ((const double *)V.x)[i];
  }
}

cudaError_t launch_vec_batched(const VecTask *tasks, const NodeItem *items, int nitems, const Seg *segs,
                               cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  vec_batched_kernel<<<nitems, kBatchNodeThreads, 0, s>>>(tasks, items, segs);
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
template cudaError_t batch_dg_pass<double>(const BatchPlan<double> &, const BatchProb<double> *, bool, const Seg *,
                                           cudaStream_t);
template cudaError_t batch_dg_pass<float>(const BatchPlan<float> &, const BatchProb<float> *, bool, const Seg *,
                                          cudaStream_t);

cudaError_t seg_dot(const Seg *segs, const SegGrid &g, int which, double *partials, unsigned *counter, double *sc,
                    int sc_stride, int slot, cudaStream_t s) {
  if (g.blocks <= 0) return cudaSuccess;
  seg_dot_kernel<<<g.blocks, 256, 0, s>>>(segs, g, which, partials, counter, sc, sc_stride, slot);
  note_launch();
  return cudaGetLastError();
}
cudaError_t seg_update_xr(const Seg *segs, const SegGrid &g, double *partials, unsigned *counter, double *sc,
                          int sc_stride, cudaStream_t s) {
  if (g.blocks <= 0) return cudaSuccess;
  seg_update_xr_kernel<<<g.blocks, 256, 0, s>>>(segs, g, partials, counter, sc, sc_stride);
  note_launch();
  return cudaGetLastError();
}
cudaError_t seg_update_p(const Seg *segs, const SegGrid &g, const double *sc, int sc_stride, int init, cudaStream_t s) {
  if (g.blocks <= 0) return cudaSuccess;
  seg_update_p_kernel<<<g.blocks, 256, 0, s>>>(segs, g, sc, sc_stride, init);
  note_launch();
  return cudaGetLastError();
}

// The block map of systems of sizes n; device arrays appended to allocs.
cudaError_t seg_grid_build(const std::vector<long> &n, SegGrid &g, std::vector<void *> &allocs) {
  std::vector<int2> map;
  std::vector<int> off, nb;
  for (size_t p = 0; p < n.size(); ++p) {
    const long k = std::max<long>(1, (n[p] + kSegChunk - 1) / kSegChunk);
    off.push_back((int)map.size());
    nb.push_back((int)k);
    for (long j = 0; j < k; ++j) map.push_back(make_int2((int)p, (int)j));
  }
  g.blocks = (int)map.size();
  int2 *dm = nullptr;
  int *doff = nullptr, *dnb = nullptr;
  cudaError_t e = cudaMalloc(&dm, std::max<size_t>(1, map.size()) * sizeof(int2));
  if (e == cudaSuccess) allocs.push_back(dm);
  if (e == cudaSuccess && (e = cudaMalloc(&doff, std::max<size_t>(1, off.size()) * sizeof(int))) == cudaSuccess)
    allocs.push_back(doff);
  if (e == cudaSuccess && (e = cudaMalloc(&dnb, std::max<size_t>(1, nb.size()) * sizeof(int))) == cudaSuccess)
    allocs.push_back(dnb);
  if (e == cudaSuccess) e = cudaMemcpy(dm, map.data(), map.size() * sizeof(int2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(doff, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dnb, nb.data(), nb.size() * sizeof(int), cudaMemcpyHostToDevice);
  g.map = dm;
  g.off = doff;
  g.nb = dnb;
  return e;
}

}  // namespace sipg
