// Vector kernels of the solver (Section 3: Algorithm 1 vector updates and
// inner products, the coarse solve) and the arithmetic-peak probe.
//
// Inner products are deterministic: a fixed grid of blocks writes one partial
// per block, and the last block to finish (detected with a counter that it
// resets) sums the partials in block order.  Scalars stay in device memory;
// update kernels read them there, so the host only synchronizes to test
// convergence.
#include <cmath>

#include "sipg_internal.h"

namespace sipg {

constexpr int kRedBlocks = 304;   // 2 x 152 SMs
constexpr int kRedThreads = 256;

template <typename T>
__global__ void fill_kernel(T *x, T v, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) x[i] = v;
}
template <typename Tout, typename Tin>
__global__ void cast_kernel(Tout *y, const Tin *x, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    y[i] = (Tout)x[i];
}
// b = (T) r and the first Chebyshev step from x = 0, x = c D^-1 b (xdb_kernel's arithmetic), in one pass
template <typename T, typename Tin>
__global__ void cast_xdb_kernel(T *b, T *x, T c, const T *dinv, const Tin *r, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const T v = (T)r[i];
    b[i] = v;
    x[i] = c * dinv[i] * v;
  }
}
template <typename T>
__global__ void axpy_kernel(T *y, T a, const T *x, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    y[i] = fma(a, x[i], y[i]);
}
__global__ void invert_kernel(double *d, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    d[i] = 1.0 / d[i];
}

static int grid_for(long n, int bs = 256) {
  long g = (n + bs - 1) / bs;
  if (g > 152L * 16) g = 152L * 16;
  return (int)(g < 1 ? 1 : g);
}

template <typename T>
cudaError_t launch_fill(T *x, T v, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  fill_kernel<T><<<grid_for(n), 256, 0, s>>>(x, v, n);
  note_launch();
  return cudaGetLastError();
}
template <typename Tout, typename Tin>
cudaError_t launch_cast(Tout *y, const Tin *x, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  cast_kernel<Tout, Tin><<<grid_for(n), 256, 0, s>>>(y, x, n);
  note_launch();
  return cudaGetLastError();
}
template <typename T, typename Tin>
cudaError_t launch_cast_xdb(T *b, T *x, T c, const T *dinv, const Tin *r, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  cast_xdb_kernel<T, Tin><<<grid_for(n), 256, 0, s>>>(b, x, c, dinv, r, n);
  note_launch();
  return cudaGetLastError();
}
template cudaError_t launch_cast_xdb<float, double>(float *, float *, float, const float *, const double *, int64_t,
                                                    cudaStream_t);
template cudaError_t launch_cast_xdb<double, double>(double *, double *, double, const double *, const double *,
                                                     int64_t, cudaStream_t);
template <typename T>
cudaError_t launch_axpy(T *y, T a, const T *x, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  axpy_kernel<T><<<grid_for(n), 256, 0, s>>>(y, a, x, n);
  note_launch();
  return cudaGetLastError();
}
cudaError_t launch_invert(double *d, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  invert_kernel<<<grid_for(n), 256, 0, s>>>(d, n);
  note_launch();
  return cudaGetLastError();
}
template cudaError_t launch_fill<double>(double *, double, int64_t, cudaStream_t);
template cudaError_t launch_fill<float>(float *, float, int64_t, cudaStream_t);
template cudaError_t launch_cast<float, double>(float *, const double *, int64_t, cudaStream_t);
template cudaError_t launch_cast<double, float>(double *, const float *, int64_t, cudaStream_t);
template cudaError_t launch_cast<double, double>(double *, const double *, int64_t, cudaStream_t);
template cudaError_t launch_cast<float, float>(float *, const float *, int64_t, cudaStream_t);
template cudaError_t launch_axpy<double>(double *, double, const double *, int64_t, cudaStream_t);
template cudaError_t launch_axpy<float>(float *, float, const float *, int64_t, cudaStream_t);

// Block reduction of two values; the last block sums the partials in order.
__device__ void reduce2_finish(double a, double b, double *partials, unsigned *counter, double *out) {
  __shared__ double sa[kRedThreads], sb[kRedThreads];
  __shared__ bool last;
  sa[threadIdx.x] = a;
  sb[threadIdx.x] = b;
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sa[threadIdx.x] += sa[threadIdx.x + w];
      sb[threadIdx.x] += sb[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = sa[0];
    partials[2 * blockIdx.x + 1] = sb[0];
    __threadfence();
    const unsigned done = atomicAdd(counter, 1u);
    last = (done == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double pa = 0, pb = 0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += kRedThreads) {
    pa += ((volatile double *)partials)[2 * i];
    pb += ((volatile double *)partials)[2 * i + 1];
  }
  sa[threadIdx.x] = pa;
  sb[threadIdx.x] = pb;
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sa[threadIdx.x] += sa[threadIdx.x + w];
      sb[threadIdx.x] += sb[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = sa[0];
    out[1] = sb[0];
    *counter = 0;
  }
}

__global__ void dot2_kernel(const double *x, const double *y, const double *z, const double *w, long n,
                            double *partials, unsigned *counter, double *out) {
  double a = 0, b = 0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    a = fma(x[i], y[i], a);
    if (z) b = fma(z[i], w[i], b);
  }
  reduce2_finish(a, b, partials, counter, out);
}

cudaError_t launch_dot2(const double *x, const double *y, const double *z, const double *w, int64_t n,
                        double *partials, unsigned *counter, double *out, cudaStream_t s) {
  dot2_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(x, y, z, w, n, partials, counter, out);
  note_launch();
  return cudaGetLastError();
}

// FCG scalar slots: sc[0] = gamma = r.z, sc[1] = z.Ap, sc[2] = p.Ap, sc[3] = r.r
// x += alpha p, r -= alpha v with alpha = gamma / p.Ap; out[0] = r.r
__global__ void fcg_update_xr_kernel(double *x, double *r, const double *p, const double *v, long n,
                                     const double *sc, double *partials, unsigned *counter, double *out) {
  const double alpha = sc[0] / sc[2];
  double a = 0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = fma(-alpha, v[i], r[i]);
    r[i] = ri;
    a = fma(ri, ri, a);
  }
  reduce2_finish(a, 0.0, partials, counter, out);
}
cudaError_t launch_fcg_update_xr(double *x, double *r, const double *p, const double *v, int64_t n,
                                 const double *sc, double *partials, unsigned *counter, double *out,
                                 cudaStream_t s) {
  fcg_update_xr_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(x, r, p, v, n, sc, partials, counter, out);
  note_launch();
  return cudaGetLastError();
}
// p = z + beta p with beta = -z.Ap / p.Ap (flexible CG, one retained direction)
__global__ void fcg_update_p_kernel(double *p, const double *z, const double *sc, long n) {
  const double beta = -sc[1] / sc[2];
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    p[i] = fma(beta, p[i], z[i]);
}
cudaError_t launch_fcg_update_p(double *p, const double *z, const double *sc, int64_t n, cudaStream_t s) {
  fcg_update_p_kernel<<<grid_for(n), 256, 0, s>>>(p, z, sc, n);
  note_launch();
  return cudaGetLastError();
}

// ------------------------------------------ flexible CG steps gated on the device
// State of a solve kept in device memory so that chunks of iterations run as
// one captured graph whose steps are conditional nodes: st[0] iterations,
// st[1] done, st[2] status (0 ok, 1 breakdown, 2 maxit reached); prm: the
// relative tolerance, maxit, the fixed iteration count (0: to the tolerance);
// the initial residual norm in sc[20]; hist[j] = ||r_j|| for j <= 256.  The
// test ||r|| <= rtol ||r_0|| is the host loop's, in the same arithmetic.
struct FcgParams {
  double rtol;
  int maxit, fixed;
};

// After x += alpha p, r -= alpha v (sc[3] = r.r): count the iteration, record
// ||r||, decide convergence or breakdown, and set the condition of the
// preconditioning step that follows (1: the solve goes on).
__global__ void fcg_check_kernel(const double *sc, double *hist, int *st, const FcgParams *prm,
                                 cudaGraphConditionalHandle next) {
  const int it = st[0] + 1;
  st[0] = it;
  int done = 0;
  const double pv = sc[2], rr = sc[3];
  if (!(pv > 0) || !isfinite(sc[0]) || !isfinite(rr)) {
    st[2] = 1;
    done = 1;
  } else {
    const double rn = sqrt(rr);
    if (it <= 256) hist[it] = rn;
    if (prm->fixed > 0) {
      done = it >= prm->fixed;
    } else if (rn <= prm->rtol * sc[20]) {
      done = 1;
    } else if (it >= prm->maxit) {
      st[2] = 2;
      done = 1;
    }
  }
  st[1] = done;
  cudaGraphSetConditional(next, done ? 0u : 1u);
}

// The condition of an iteration's first step: 1 while the solve is not done.
__global__ void fcg_cond_kernel(const int *st, cudaGraphConditionalHandle h) {
  cudaGraphSetConditional(h, st[1] ? 0u : 1u);
}

cudaError_t launch_fcg_check(const double *sc, double *hist, int *st, const void *prm, cudaGraphConditionalHandle next,
                             cudaStream_t s) {
  fcg_check_kernel<<<1, 1, 0, s>>>(sc, hist, st, (const FcgParams *)prm, next);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_fcg_cond(const int *st, cudaGraphConditionalHandle h, cudaStream_t s) {
  fcg_cond_kernel<<<1, 1, 0, s>>>(st, h);
  note_launch();
  return cudaGetLastError();
}

// ------------------------------------------ coarse-level Jacobi-PCG
// Kernels of a fixed number of preconditioned CG iterations on vectors of the
// cycle's precision with FP64 scalars that stay in device memory (so the
// iteration can be captured in the V-cycle's graph): deterministic dot
// products, and updates that read their step lengths from the scalar slots.
template <typename T>
__global__ void cg_dot_kernel(const T *x, const T *y, long n, double *partials, unsigned *counter, double *out) {
  double a = 0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    a = fma((double)x[i], (double)y[i], a);
  reduce2_finish(a, 0.0, partials, counter, out);
}
template <typename T>
cudaError_t launch_cg_dot(const T *x, const T *y, int64_t n, double *partials, unsigned *counter, double *out,
                          cudaStream_t s) {
  cg_dot_kernel<T><<<kRedBlocks, kRedThreads, 0, s>>>(x, y, n, partials, counter, out);
  note_launch();
  return cudaGetLastError();
}
// x += alpha p, r -= alpha q with alpha = gamma / pq (0 when pq is not positive)
template <typename T>
__global__ void cg_update_xr_kernel(T *x, T *r, const T *p, const T *q, long n, const double *gamma,
                                    const double *pq) {
  const double alpha = pq[0] > 0 ? gamma[0] / pq[0] : 0.0;
  const T a = (T)alpha;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    x[i] = fma(a, p[i], x[i]);
    r[i] = fma(-a, q[i], r[i]);
  }
}
template <typename T>
cudaError_t launch_cg_update_xr(T *x, T *r, const T *p, const T *q, int64_t n, const double *gamma, const double *pq,
                                cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  cg_update_xr_kernel<T><<<grid_for(n), 256, 0, s>>>(x, r, p, q, n, gamma, pq);
  note_launch();
  return cudaGetLastError();
}
// p = z + beta p with beta = gamma_new / gamma_old (0 when gamma_old is not positive)
template <typename T>
__global__ void cg_update_p_kernel(T *p, const T *z, long n, const double *gnew, const double *gold) {
  const double beta = gold[0] > 0 ? gnew[0] / gold[0] : 0.0;
  const T b = (T)beta;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    p[i] = fma(b, p[i], z[i]);
}
template <typename T>
cudaError_t launch_cg_update_p(T *p, const T *z, int64_t n, const double *gnew, const double *gold, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  cg_update_p_kernel<T><<<grid_for(n), 256, 0, s>>>(p, z, n, gnew, gold);
  note_launch();
  return cudaGetLastError();
}
#define SIPG_CG_INST(T)                                                                                      \
  template cudaError_t launch_cg_dot<T>(const T *, const T *, int64_t, double *, unsigned *, double *,       \
                                        cudaStream_t);                                                       \
  template cudaError_t launch_cg_update_xr<T>(T *, T *, const T *, const T *, int64_t, const double *,       \
                                              const double *, cudaStream_t);                                 \
  template cudaError_t launch_cg_update_p<T>(T *, const T *, int64_t, const double *, const double *,        \
                                             cudaStream_t);
SIPG_CG_INST(double)
#undef SIPG_CG_INST

// Coarse solve x = A0^-1 b with the explicit inverse (one warp per row, FP64).
template <typename Tb, typename Tx>
__global__ void dense_gemv_kernel(const double *__restrict__ Ainv, const Tb *__restrict__ b, Tx *__restrict__ x,
                                  int n) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n) return;
  b += (size_t)blockIdx.y * n;   // vector blockIdx.y
  x += (size_t)blockIdx.y * n;
  const double *row = Ainv + (size_t)warp * n;
  double s = 0;
  for (int j = lane; j < n; j += 32) s = fma(row[j], (double)b[j], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) x[warp] = (Tx)s;
}
template <typename Tb, typename Tx>
cudaError_t launch_dense_gemv(const double *Ainv, const Tb *b, Tx *x, int n, cudaStream_t s, int nv) {
  const int bs = 256, wpb = bs / 32;
  if (n <= 0) return cudaSuccess;
  dense_gemv_kernel<Tb, Tx><<<dim3((n + wpb - 1) / wpb, nv), bs, 0, s>>>(Ainv, b, x, n);
  note_launch();
  return cudaGetLastError();
}
template cudaError_t launch_dense_gemv<double, double>(const double *, const double *, double *, int, cudaStream_t,
                                                       int);
template cudaError_t launch_dense_gemv<float, float>(const double *, const float *, float *, int, cudaStream_t, int);

// ------------------------------------------------------------ peak probe
// Eight independent FMA chains per thread, all SMs busy; the result is kept
// live through a conditional store so the compiler cannot drop the chains.
template <typename T>
__global__ void fma_probe_kernel(T *sink, int iters, T a, T b) {
  T acc[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) acc[k] = (T)(threadIdx.x + k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = fma(acc[k], a, b);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += acc[k];
  if (s == (T)-12345.678) sink[0] = s;
}

// FP64 tensor-core probe: four independent m8n8k4 FP64 mma.sync chains per
// warp (512 flops each per instruction), all SMs busy.
__global__ void dmma_probe_kernel(double *sink, int iters) {
  const double a = 1.0 + 1e-9 * threadIdx.x, b = 0.999999;
  double c[4][2];
#pragma unroll
  for (int k = 0; k < 4; ++k) c[k][0] = c[k][1] = (double)k;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};\n"
                   : "+d"(c[k][0]), "+d"(c[k][1])
                   : "d"(a), "d"(b));
  }
  double t = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) t += c[k][0] + c[k][1];
  if (t == -12345.678) sink[0] = t;
}

cudaError_t fma_peak(int precision, cudaStream_t s, double *flops) {
  int dev, nsm;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = nsm * 8, threads = 256;
  const int iters = precision == 1 ? 65536 : 2048;
  void *sink;
  cudaError_t e = cudaMalloc(&sink, 16);
  if (e != cudaSuccess) return e;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0, s);
    if (precision == 0)
      fma_probe_kernel<double><<<blocks, threads, 0, s>>>((double *)sink, iters, 0.999999, 1e-7);
    else if (precision == 1)
      fma_probe_kernel<float><<<blocks, threads, 0, s>>>((float *)sink, iters, 0.999999f, 1e-7f);
    else
      dmma_probe_kernel<<<blocks, threads, 0, s>>>((double *)sink, iters);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  const double per_thread_iter = precision == 2 ? 4.0 * 512.0 / 32.0 : 2.0 * 8.0;   // flops
  *flops = per_thread_iter * (double)iters * blocks * threads / (best * 1e-3);
  return e;
}

}  // namespace sipg

namespace sipg {
// x = c * dinv * b (first Chebyshev step from a zero start)
template <typename T>
__global__ void xdb_kernel(T *x, T c, const T *dinv, const T *b, long n) {
  x += blockIdx.y * n;   // vector blockIdx.y; dinv is shared
  b += blockIdx.y * n;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    x[i] = c * dinv[i] * b[i];
}
template <typename T>
cudaError_t launch_xdb(T *x, T c, const T *dinv, const T *b, int64_t n, cudaStream_t s, int nv) {
  if (n <= 0) return cudaSuccess;
  xdb_kernel<T><<<dim3(grid_for(n), nv), 256, 0, s>>>(x, c, dinv, b, n);
  note_launch();
  return cudaGetLastError();
}
// p = z + beta p
template <typename T>
__global__ void xpby_kernel(T *p, const T *z, T beta, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    p[i] = fma(beta, p[i], z[i]);
}
template <typename T>
cudaError_t launch_xpby(T *p, const T *z, T beta, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  xpby_kernel<T><<<grid_for(n), 256, 0, s>>>(p, z, beta, n);
  note_launch();
  return cudaGetLastError();
}
template cudaError_t launch_xdb<double>(double *, double, const double *, const double *, int64_t, cudaStream_t, int);
template cudaError_t launch_xdb<float>(float *, float, const float *, const float *, int64_t, cudaStream_t, int);
template cudaError_t launch_xpby<double>(double *, const double *, double, int64_t, cudaStream_t);
template cudaError_t launch_xpby<float>(float *, const float *, float, int64_t, cudaStream_t);
}  // namespace sipg
