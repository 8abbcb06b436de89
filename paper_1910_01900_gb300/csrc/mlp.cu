// Learned per-cell smoother: feature gathering, BF16 tensor-core GEMMs with
// FP32 accumulation (forward and backward), Adam, and the smoothing step.
// Not in the paper: a network that maps a cell's local residual to a
// correction of the cell's values, trained on residual -> error pairs that the
// plain multigrid produces, used in place of the Chebyshev smoother on the
// finest level inside flexible CG.
//
// GEMM: C[M x N] = sum_k A(m, k) B(k, n) with A, B in BF16 addressed through
// row and column strides (so transposed operands need no copy), FP32
// accumulation on mma.sync m16n8k16 tensor-core instructions, 64 x 64 block
// tiles (4 warps of 32 x 32), optional bias, ReLU and BF16 or FP32 output.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "sipg_internal.h"

namespace sipg {

namespace {

constexpr int TM = 64, TN = 64, TK = 16;

__device__ __forceinline__ unsigned pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (unsigned)__bfloat16_as_ushort(lo) | ((unsigned)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

struct GemmArgs {
  const __nv_bfloat16 *A;
  long sam, sak;   // A(m,k) = A[m*sam + k*sak]
  const __nv_bfloat16 *B;
  long sbk, sbn;   // B(k,n) = B[k*sbk + n*sbn]
  int M, N, K;
  const float *bias;   // [N] or null
  int relu;
  float *Cf;           // fp32 output (or null)
  __nv_bfloat16 *Cb;   // bf16 output (or null)
  long ldc;
  int accumulate;      // Cf += result
};

__global__ void __launch_bounds__(128) gemm_bf16_kernel(const GemmArgs g) {
  __shared__ __nv_bfloat16 As[TM][TK + 8];
  __shared__ __nv_bfloat16 Bs[TK][TN + 8];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int gid = lane >> 2, tig = lane & 3;
  float acc[2][4][4];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 4; ++j)
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
  const __nv_bfloat16 zero = __float2bfloat16(0.f);
  for (int k0 = 0; k0 < g.K; k0 += TK) {
    for (int i = tid; i < TM * TK; i += 128) {
      const int r = i / TK, c = i % TK;
      const int gm = m0 + r, gk = k0 + c;
      As[r][c] = (gm < g.M && gk < g.K) ? g.A[gm * g.sam + gk * g.sak] : zero;
    }
    for (int i = tid; i < TK * TN; i += 128) {
      const int r = i / TN, c = i % TN;
      const int gk = k0 + r, gn = n0 + c;
      Bs[r][c] = (gk < g.K && gn < g.N) ? g.B[gk * g.sbk + gn * g.sbn] : zero;
    }
    __syncthreads();
    unsigned af[2][4], bfr[4][2];
    for (int i = 0; i < 2; ++i) {
      const int r = wm + i * 16 + gid;
      af[i][0] = pack2(As[r][tig * 2], As[r][tig * 2 + 1]);
      af[i][1] = pack2(As[r + 8][tig * 2], As[r + 8][tig * 2 + 1]);
      af[i][2] = pack2(As[r][tig * 2 + 8], As[r][tig * 2 + 9]);
      af[i][3] = pack2(As[r + 8][tig * 2 + 8], As[r + 8][tig * 2 + 9]);
    }
    for (int j = 0; j < 4; ++j) {
      const int c = wn + j * 8 + gid;
      bfr[j][0] = pack2(Bs[tig * 2][c], Bs[tig * 2 + 1][c]);
      bfr[j][1] = pack2(Bs[tig * 2 + 8][c], Bs[tig * 2 + 9][c]);
    }
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bfr[j]);
    __syncthreads();
  }
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 4; ++j)
      for (int r = 0; r < 4; ++r) {
        const int gm = m0 + wm + i * 16 + gid + (r >= 2 ? 8 : 0);
        const int gn = n0 + wn + j * 8 + tig * 2 + (r & 1);
        if (gm >= g.M || gn >= g.N) continue;
        float v = acc[i][j][r];
        if (g.bias) v += g.bias[gn];
        if (g.relu) v = fmaxf(v, 0.f);
        if (g.Cf) {
          if (g.accumulate) g.Cf[gm * g.ldc + gn] += v;
          else g.Cf[gm * g.ldc + gn] = v;
        }
        if (g.Cb) g.Cb[gm * g.ldc + gn] = __float2bfloat16(v);
      }
}

// Features of cells (first cell c0, count nc) from a DG residual: the cell's
// n^3 values, then per face (-x,+x,-y,+y,-z,+z) the neighbour's n^2 values on
// the shared face (zeros on the boundary); scaled by their RMS.  One warp per cell.
template <typename T>
__global__ void gather_features_kernel(const T *r, int n, int m0, int m1, int m2, const int *cells, int ncells_sel,
                                       int c0, int nc, __nv_bfloat16 *X, int ldx, float *scale) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= nc) return;
  const int cell = cells ? cells[c0 + w] : c0 + w;
  (void)ncells_sel;
  const int n2 = n * n, n3 = n2 * n, nf = n3 + 6 * n2;
  const int ijk[3] = {cell % m0, (cell / m0) % m1, cell / (m0 * m1)};
  const int mm[3] = {m0, m1, m2};
  const int stride[3] = {1, m0, m0 * m1};
  auto value = [&](int j) -> double {
    if (j < n3) return (double)r[(size_t)cell * n3 + j];
    const int f = (j - n3) / n2, q = (j - n3) % n2;
    const int d = f >> 1, s = f & 1;
    const bool has = s ? (ijk[d] < mm[d] - 1) : (ijk[d] > 0);
    if (!has) return 0.0;
    const int nb = cell + (s ? stride[d] : -stride[d]);
    const int a = q % n, b = q / n, idx = s ? 0 : n - 1;
    int node;
    if (d == 0) node = idx + n * (a + n * b);
    else if (d == 1) node = a + n * (idx + n * b);
    else node = a + n * (b + n * idx);
    return (double)r[(size_t)nb * n3 + node];
  };
  double ss = 0;
  for (int j = lane; j < nf; j += 32) {
    const double v = value(j);
    ss += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  // a cell whose local residual is (numerically) zero gets zero inputs and scale 0
  const double s = sqrt(ss / nf);
  const bool ok = s > 1e-30 && s < 1e30;
  for (int j = lane; j < ldx; j += 32)
    X[(size_t)w * ldx + j] = __float2bfloat16(ok && j < nf ? (float)(value(j) / s) : 0.f);
  if (lane == 0) scale[w] = ok ? (float)s : 0.f;
}

// x[cell] += c * s_cell * y[cell][0..n^3)   (the learned smoothing step)
template <typename T>
__global__ void apply_correction_kernel(T *x, int n3, int c0, int nc, const float *Y, int ldy, const float *scale,
                                        float c) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long)nc * n3) return;
  const int w = (int)(i / n3), j = (int)(i - (long)w * n3);
  const float y = Y[(size_t)w * ldy + j];
  if (isfinite(y)) x[(size_t)(c0 + w) * n3 + j] += (T)(c * scale[w] * y);   // a non-finite output is skipped
}

// dY = (Y - T) / B as bf16 and the loss partial sums
__global__ void mse_grad_kernel(const float *Y, const float *Tg, long ldt, int B, int N, int ld, __nv_bfloat16 *dY,
                                float *dYf, double *loss) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long)B * ld) return;
  const int r = (int)(i / ld), c = (int)(i - (long)r * ld);
  float d = 0.f;
  if (c < N) d = Y[i] - Tg[(size_t)r * ldt + c];
  if (c < N) atomicAdd(loss, 0.5 * (double)d * d / B);
  dY[i] = __float2bfloat16(d / B);
  dYf[i] = d / B;
}

// dH = dH * (H > 0) in place (bf16)
__global__ void relu_mask_kernel(__nv_bfloat16 *dH, const __nv_bfloat16 *H, long n) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && !(__bfloat162float(H[i]) > 0.f)) dH[i] = __float2bfloat16(0.f);
}

// column sums of a [B x N] matrix (bias gradient); one thread per column
__global__ void colsum_kernel(const __nv_bfloat16 *D, int B, int N, int ld, float *g) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  float s = 0.f;
  for (int r = 0; r < B; ++r) s += __bfloat162float(D[(size_t)r * ld + c]);
  g[c] = s;
}
__global__ void colsum_f_kernel(const float *D, int B, int N, int ld, float *g) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  float s = 0.f;
  for (int r = 0; r < B; ++r) s += D[(size_t)r * ld + c];
  g[c] = s;
}

// Adam on fp32 master parameters; refresh the bf16 copy
__global__ void adam_kernel(float *p, float *mom, float *vel, const float *g, long n, float lr, float b1, float b2,
                            float eps, float c1, float c2, __nv_bfloat16 *pb) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float m = b1 * mom[i] + (1 - b1) * gi;
  const float v = b2 * vel[i] + (1 - b2) * gi * gi;
  mom[i] = m;
  vel[i] = v;
  const float q = p[i] - lr * (m / c1) / (sqrtf(v / c2) + eps);
  p[i] = q;
  if (pb) pb[i] = __float2bfloat16(q);
}

__global__ void f2bf_kernel(const float *x, __nv_bfloat16 *y, long n) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = __float2bfloat16(x[i]);
}

// T[w][j] = e[cell_w][j] / s_w for j < n3, 0 in the padding
__global__ void targets_kernel(const double *e, int n3, const int *cells, int c0, int nc, const float *scale, float *T,
                               int ldt) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long)nc * ldt) return;
  const int w = (int)(i / ldt), j = (int)(i - (long)w * ldt);
  const int cell = cells[c0 + w];
  T[i] = (j < n3 && scale[w] > 0.f) ? (float)(e[(size_t)cell * n3 + j] / (double)scale[w]) : 0.f;
}
__global__ void sumsq_kernel(const float *x, long n, double *out) {
  double s = 0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    s += (double)x[i] * x[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}
// max |x| over the finite entries (as ordered bits) and the number of non-finite entries
__global__ void stats_kernel(const float *x, long n, unsigned *maxbits, unsigned long long *bad) {
  unsigned m = 0;
  unsigned long long nb = 0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const float v = x[i];
    if (!isfinite(v)) ++nb;
    else m = max(m, __float_as_uint(fabsf(v)));
  }
  atomicMax(maxbits, m);
  if (nb) atomicAdd(bad, nb);
}
__global__ void scale_kernel(float *x, long n, float a) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] *= a;
}
// row-padded fp32 -> bf16: Y[r][c] = X[r][c] for c < F, 0 for F <= c < Fp
__global__ void pad_f2bf_kernel(const float *X, int B, int F, int Fp, __nv_bfloat16 *Y) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long)B * Fp) return;
  const int r = (int)(i / Fp), c = (int)(i - (long)r * Fp);
  Y[i] = __float2bfloat16(c < F ? X[(size_t)r * F + c] : 0.f);
}
__global__ void bf2f_kernel(const __nv_bfloat16 *X, long n, float *Y) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) Y[i] = __bfloat162float(X[i]);
}

inline int blocks(long n, int bs = 256) { return (int)((n + bs - 1) / bs); }

}  // namespace

// ------------------------------------------------------------------ launchers

cudaError_t mlp_gemm(const void *A, long sam, long sak, const void *B, long sbk, long sbn, int M, int N, int K,
                     const float *bias, int relu, float *Cf, void *Cb, long ldc, int accumulate, cudaStream_t s) {
  GemmArgs g{(const __nv_bfloat16 *)A, sam, sak, (const __nv_bfloat16 *)B, sbk, sbn, M, N, K, bias, relu, Cf,
             (__nv_bfloat16 *)Cb, ldc, accumulate};
  dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM);
  gemm_bf16_kernel<<<grid, 128, 0, s>>>(g);
  note_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t mlp_gather(const T *r, int n, const int m[3], const int *cells, int c0, int nc, void *X, int ldx,
                       float *scale, cudaStream_t s) {
  if (nc <= 0) return cudaSuccess;
  gather_features_kernel<T><<<blocks((long)nc * 32, 256), 256, 0, s>>>(r, n, m[0], m[1], m[2], cells, 0, c0, nc,
                                                                        (__nv_bfloat16 *)X, ldx, scale);
  note_launch();
  return cudaGetLastError();
}
template cudaError_t mlp_gather<float>(const float *, int, const int *, const int *, int, int, void *, int, float *,
                                       cudaStream_t);
template cudaError_t mlp_gather<double>(const double *, int, const int *, const int *, int, int, void *, int,
                                        float *, cudaStream_t);

template <typename T>
cudaError_t mlp_correct(T *x, int n3, int c0, int nc, const float *Y, int ldy, const float *scale, float c,
                        cudaStream_t s) {
  if (nc <= 0) return cudaSuccess;
  apply_correction_kernel<T><<<blocks((long)nc * n3), 256, 0, s>>>(x, n3, c0, nc, Y, ldy, scale, c);
  note_launch();
  return cudaGetLastError();
}
template cudaError_t mlp_correct<float>(float *, int, int, int, const float *, int, const float *, float,
                                        cudaStream_t);
template cudaError_t mlp_correct<double>(double *, int, int, int, const float *, int, const float *, float,
                                         cudaStream_t);

cudaError_t mlp_mse_grad(const float *Y, const float *Tg, long ldt, int B, int N, int ld, void *dY, float *dYf,
                         double *loss, cudaStream_t s) {
  mse_grad_kernel<<<blocks((long)B * ld), 256, 0, s>>>(Y, Tg, ldt, B, N, ld, (__nv_bfloat16 *)dY, dYf, loss);
  note_launch();
  return cudaGetLastError();
}
cudaError_t mlp_relu_mask(void *dH, const void *H, long n, cudaStream_t s) {
  relu_mask_kernel<<<blocks(n), 256, 0, s>>>((__nv_bfloat16 *)dH, (const __nv_bfloat16 *)H, n);
  note_launch();
  return cudaGetLastError();
}
cudaError_t mlp_colsum(const void *D, int bf16, int B, int N, int ld, float *g, cudaStream_t s) {
  if (bf16)
    colsum_kernel<<<blocks(N, 128), 128, 0, s>>>((const __nv_bfloat16 *)D, B, N, ld, g);
  else
    colsum_f_kernel<<<blocks(N, 128), 128, 0, s>>>((const float *)D, B, N, ld, g);
  note_launch();
  return cudaGetLastError();
}
cudaError_t mlp_adam(float *p, float *m, float *v, const float *g, long n, float lr, int step, void *pb,
                     cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  adam_kernel<<<blocks(n), 256, 0, s>>>(p, m, v, g, n, lr, b1, b2, 1e-8f, c1, c2, (__nv_bfloat16 *)pb);
  note_launch();
  return cudaGetLastError();
}
cudaError_t mlp_f2bf(const float *x, void *y, long n, cudaStream_t s) {
  f2bf_kernel<<<blocks(n), 256, 0, s>>>(x, (__nv_bfloat16 *)y, n);
  note_launch();
  return cudaGetLastError();
}

cudaError_t mlp_targets(const double *e, int n3, const int *cells, int c0, int nc, const float *scale, float *T,
                        int ldt, cudaStream_t s) {
  if (nc <= 0) return cudaSuccess;
  targets_kernel<<<blocks((long)nc * ldt), 256, 0, s>>>(e, n3, cells, c0, nc, scale, T, ldt);
  note_launch();
  return cudaGetLastError();
}
cudaError_t mlp_sumsq(const float *x, long n, double *out, cudaStream_t s) {
  sumsq_kernel<<<std::min(blocks(n), 152 * 8), 256, 0, s>>>(x, n, out);
  note_launch();
  return cudaGetLastError();
}
cudaError_t mlp_stats(const float *x, long n, unsigned *maxbits, unsigned long long *bad, cudaStream_t s) {
  stats_kernel<<<std::min(blocks(n), 152 * 8), 256, 0, s>>>(x, n, maxbits, bad);
  note_launch();
  return cudaGetLastError();
}
cudaError_t mlp_scale(float *x, long n, float a, cudaStream_t s) {
  scale_kernel<<<blocks(n), 256, 0, s>>>(x, n, a);
  note_launch();
  return cudaGetLastError();
}
cudaError_t mlp_pad_f2bf(const float *X, int B, int F, int Fp, void *Y, cudaStream_t s) {
  pad_f2bf_kernel<<<blocks((long)B * Fp), 256, 0, s>>>(X, B, F, Fp, (__nv_bfloat16 *)Y);
  note_launch();
  return cudaGetLastError();
}
cudaError_t mlp_bf2f(const void *X, long n, float *Y, cudaStream_t s) {
  bf2f_kernel<<<blocks(n), 256, 0, s>>>((const __nv_bfloat16 *)X, n, Y);
  note_launch();
  return cudaGetLastError();
}

}  // namespace sipg
