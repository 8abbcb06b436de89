// Learned per-cell smoother: feature gathering, BF16 tensor-core GEMMs with
// FP32 accumulation (forward and backward), Adam, and the smoothing step.
// Not in the paper: a network that maps a cell's local residual to a
// correction of the cell's values, trained on residual -> error pairs that the
// plain multigrid produces, used in place of the Chebyshev smoother on the
// finest level inside flexible CG.
//
// GEMMs: the forward pass (the smoother's inference inside the V-cycle and
// training's forward) runs on the tcgen05 tensor cores with the accumulator in
// tensor memory (gemm_tc_kernel below; activations and transposed weights both
// K-contiguous).  The backward pass's GEMMs, whose operands are transposed
// through strides, use C[M x N] = sum_k A(m, k) B(k, n) with A, B in BF16
// addressed through row and column strides, FP32 accumulation on mma.sync
// m16n8k16 instructions, 64 x 64 block tiles (4 warps of 32 x 32), optional
// bias, ReLU and BF16 or FP32 output.
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

// ---------------------------------------------------- tcgen05 GEMM
// C[M x N] = A[M x K] Bt[N x K]^T on the 5th-generation tensor cores, for the
// network's forward pass (activations times weights, both K-contiguous; the
// weights are kept transposed for it).  One CTA computes a 128 x N tile (N =
// the whole output width, a multiple of 16 up to 256) with tcgen05.mma
// (kind::f16, BF16 operands, FP32 accumulator in tensor memory).  Both
// operands are staged through shared memory in the K-major canonical layout
// without swizzle: 8-row x 16-byte core matrices, adjacent along K at 128
// bytes (leading byte offset), adjacent along M/N at (KC/8) x 128 bytes
// (stride byte offset).  K runs in chunks of KC = 64 through two shared-memory
// stages: the 128 threads copy the 16-byte pieces of chunk i + 1 with cp.async
// (zero-filled outside the matrices) while the tensor core works on chunk i;
// once a chunk has landed it is made visible to the tensor core
// (fence.proxy.async) and one thread issues four K = 16 MMAs and commits them
// to the stage's mbarrier, which every thread waits on (bounded) before the
// stage is refilled.  The epilogue reads the
// accumulator with tcgen05.ld (warp w owns lanes 32w..32w+31 = tile rows),
// adds the bias, applies ReLU and stores FP32 or BF16.
constexpr int TC_M = 128, TC_KC = 64;
// one stage: A (128 x 64 bf16 = 16 KB) then B (up to 256 x 64 bf16 = 32 KB);
// the two stages interleave: stage b of A at b x TC_STAGE, of B at 16 KB + b x TC_STAGE
constexpr int TC_STAGE = 48 * 1024;
// dynamic shared memory per CTA: two stages, 96 KB, which also keeps at most
// two CTAs on an SM, so their tensor-memory columns (<= 256 each) always fit
// in the SM's 512 and tcgen05.alloc never waits
constexpr int TC_SMEM = 2 * TC_STAGE;
constexpr int TC_WAIT_LIMIT = 1 << 22;   // mbarrier polls before a CTA gives up
__device__ int g_tc_timeout;             // set by a CTA whose MMA wait ran out

struct TcArgs {
  const __nv_bfloat16 *A;    // [M][lda], K contiguous
  const __nv_bfloat16 *Bt;   // [N][ldb], K contiguous
  long lda, ldb;
  int M, N, K;
  const float *bias;   // [N] or null
  int relu;
  float *Cf;           // fp32 output (or null)
  __nv_bfloat16 *Cb;   // bf16 output (or null)
  long ldc;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start address, leading / stride byte
// offsets (all >> 4), fixed version bits 46-48 = 0b001, no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}

// byte offset of the 16-byte piece (row r, K group g of 8) in a core-matrix tile
__device__ __forceinline__ uint32_t tc_core_off(int r, int g) {
  return (uint32_t)(((r >> 3) * (TC_KC >> 3) + g) * 128 + (r & 7) * 16);
}

__device__ __forceinline__ void tc_copy16(uint32_t dst, const void *src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0)
               : "memory");
}

__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity) {
  for (int it = 0; it < TC_WAIT_LIMIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__global__ void __launch_bounds__(128) gemm_tc_kernel(const TcArgs g, const uint32_t ncols) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  __shared__ __align__(8) unsigned long long mbar[2];
  __shared__ uint32_t tmem_slot;
  // stage b: A tile (TC_M x TC_KC bf16) at sA + b TC_STAGE, B tile (N x TC_KC) at sB + b TC_STAGE
  const uint32_t sA = smem_u32(tc_smem);
  const uint32_t sB = smem_u32(tc_smem + TC_M * TC_KC * 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * TC_M;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  // instruction descriptor: D FP32 (bit 4), A and B BF16 (bits 7, 10), both
  // K-major, N >> 3 at bit 17, M >> 4 at bit 24
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(g.N >> 3) << 17) |
                         ((uint32_t)(TC_M >> 4) << 24);
  constexpr int G = TC_KC / 8;   // 16-byte groups per row and chunk
  // two stages: the copies of chunk i + 1 are in flight while the tensor core
  // works on chunk i.  Stage b holds chunks b, b + 2, ...; barrier b completes
  // once per MMA batch issued on stage b (parity = use count & 1).
  const int nch = (g.K + TC_KC - 1) / TC_KC;
  auto stage = [&](int chunk) {
    const int k0 = chunk * TC_KC;
    const uint32_t a0 = sA + (uint32_t)(chunk & 1) * TC_STAGE, b0 = sB + (uint32_t)(chunk & 1) * TC_STAGE;
    for (int i = tid; i < TC_M * G; i += 128) {   // K group fastest: each row read in 128-byte runs
      const int r = i / G, q = i - r * G;
      const bool valid = m0 + r < g.M && k0 + 8 * q < g.K;
      tc_copy16(a0 + tc_core_off(r, q), valid ? g.A + (long)(m0 + r) * g.lda + k0 + 8 * q : g.A, valid);
    }
    for (int i = tid; i < g.N * G; i += 128) {
      const int r = i / G, q = i - r * G;
      const bool valid = k0 + 8 * q < g.K;
      tc_copy16(b0 + tc_core_off(r, q), valid ? g.Bt + (long)r * g.ldb + k0 + 8 * q : g.Bt, valid);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  auto mma_wait = [&](int chunk) {   // every thread: the MMAs of `chunk` are done
    return tc_wait(smem_u32(&mbar[chunk & 1]), (uint32_t)((chunk >> 1) & 1)) ? 1 : 0;
  };
  int ok = 1, issued = -1;   // last chunk whose MMAs were issued
  stage(0);
  for (int i = 0; i < nch && ok; ++i) {
    if (i + 1 < nch) {
      // stage (i + 1) & 1 was last read by the MMAs of chunk i - 1
      if (i >= 1) ok = __syncthreads_and(mma_wait(i - 1));
      if (!ok) break;
      stage(i + 1);
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");   // chunk i has landed
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = sA + (uint32_t)(i & 1) * TC_STAGE, b0 = sB + (uint32_t)(i & 1) * TC_STAGE;
#pragma unroll
      for (int kk = 0; kk < TC_KC; kk += 16) {
        const uint64_t ad = tc_desc(a0 + (kk >> 3) * 128, 128, G * 128);
        const uint64_t bd = tc_desc(b0 + (kk >> 3) * 128, 128, G * 128);
        const uint32_t acc = (i > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&mbar[i & 1]))
                   : "memory");
    }
    issued = i;
  }
  // MMAs complete in issue order: the last chunk's barrier covers them all
  if (ok) {
    ok = __syncthreads_and(mma_wait(nch - 1));
  } else {
    // a wait ran out: drain the copies, give the MMAs in flight one more
    // bounded wait, then write nothing and free the tensor memory below
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    if (issued >= 0) (void)mma_wait(issued);
    __syncthreads();
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    const int gm = m0 + warp * 32 + lane;
    for (int c0 = 0; c0 < g.N; c0 += 16) {
      uint32_t v[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
          "[%16];\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (gm < g.M) {
        // the thread's 16 consecutive outputs of its row go out as whole
        // 16-byte vectors (full 32-byte sectors), not as scattered scalars
        float x[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          x[j] = __uint_as_float(v[j]);
          if (g.bias) x[j] += g.bias[c0 + j];
          if (g.relu) x[j] = fmaxf(x[j], 0.f);
        }
        if (g.Cf) {
          float4 *dst = reinterpret_cast<float4 *>(g.Cf + (long)gm * g.ldc + c0);
#pragma unroll
          for (int q = 0; q < 4; ++q) dst[q] = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
        }
        if (g.Cb) {
          uint32_t w[8];
#pragma unroll
          for (int q = 0; q < 8; ++q)
            w[q] = pack2(__float2bfloat16(x[2 * q]), __float2bfloat16(x[2 * q + 1]));
          uint4 *dst = reinterpret_cast<uint4 *>(g.Cb + (long)gm * g.ldc + c0);
          dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
          dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
        }
      }
    }
  } else if (tid == 0) {
    atomicExch(&g_tc_timeout, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// The whole network in one kernel (hidden width 256, output width <= 256):
// one CTA per 128-row tile runs the three layers back to back.  The tile's
// hidden activations never leave the SM: each layer's FP32 accumulator sits
// in tensor memory, the epilogue (bias, ReLU, BF16) writes it into a 64 KB
// shared-memory tile in the K-major core-matrix layout that the next layer's
// MMAs read as their A operand.  The weights (and the first layer's
// features) are packed in global memory in that same layout, one contiguous
// block per K chunk of 32 (mlp_pack_core), so that a pipeline stage is one
// or two bulk copies (cp.async.bulk, the TMA engine) completed on the
// stage's "full" mbarrier; one thread issues the copies and the MMAs and
// commits each MMA batch to the stage's "empty" mbarrier, which the refill
// of that stage waits on.  Every wait is bounded: a CTA that runs out
// drains what it issued (bounded), writes nothing, frees its tensor memory
// and sets the flag the host turns into SIPG_ETIMEOUT.  Optionally the
// hidden activations also go to global memory (training keeps them for the
// backward pass).
constexpr int FZ_H = 256;
constexpr int FZ_T = 256;                                  // threads: eight warps
constexpr int FZ_KC = 32;                                  // K per chunk
constexpr int FZ_S = 6;                                    // stages
constexpr int FZ_P = 4;                                    // chunks in flight ahead of the MMAs
constexpr int FZ_STAGE_A = TC_M * FZ_KC * 2;               // 8 KB of features
constexpr int FZ_STAGE = FZ_STAGE_A + FZ_H * FZ_KC * 2;    // + 16 KB of weights
constexpr int FZ_HTILE = TC_M * FZ_H * 2;                  // 64 KB hidden tile: 4 K-chunks of 64
constexpr int FZ_SMEM = FZ_S * FZ_STAGE + FZ_HTILE;        // 208 KB: one CTA per SM

// byte offset of the 16-byte piece (row r, K group g) in a core-matrix block
// of kc columns (8-row x 16-byte core matrices, K groups adjacent at 128 B)
__host__ __device__ __forceinline__ uint32_t fz_core_off(int r, int g, int kc) {
  return (uint32_t)(((r >> 3) * (kc >> 3) + g) * 128 + (r & 7) * 16);
}

// dst = src [rows][K] (row stride ld) in blocks of rt rows x FZ_KC columns,
// block (tile t, chunk j) at (t * nch + j) * rt * FZ_KC elements, inside a
// block the core-matrix layout of fz_core_off; rows >= rows and columns >= K
// are zero.  One thread per 16-byte piece.
__global__ void pack_core_kernel(const __nv_bfloat16 *src, long ld, int rows, int K, int rt, int nch, int ntiles,
                                 __nv_bfloat16 *dst) {
  const long pieces = (long)ntiles * rt * nch * (FZ_KC / 8);
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < pieces; i += (long)gridDim.x * blockDim.x) {
    const int g = (int)(i % (FZ_KC / 8));
    long rem = i / (FZ_KC / 8);
    const int j = (int)(rem % nch);
    rem /= nch;
    const int rr = (int)(rem % rt), t = (int)(rem / rt);
    const int row = t * rt + rr, k0 = j * FZ_KC + 8 * g;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (row < rows && k0 < K) v = *reinterpret_cast<const uint4 *>(src + (long)row * ld + k0);
    unsigned char *blk = reinterpret_cast<unsigned char *>(dst + ((long)t * nch + j) * rt * FZ_KC);
    *reinterpret_cast<uint4 *>(blk + fz_core_off(rr, g, FZ_KC)) = v;
  }
}

struct FusedArgs {
  const __nv_bfloat16 *Xc;  // features packed in 128-row tiles, nch1 chunks per tile
  int M, nch1, No;
  const __nv_bfloat16 *W1c, *W2c, *W3c;   // packed weights: 256 x (32 nch1), 256 x 256, No x 256
  const float *b1, *b2, *b3;
  float *Y;                 // [M][ldy] fp32 outputs (bias, no ReLU)
  long ldy;
  __nv_bfloat16 *H1, *H2;   // [M][256] hidden activations or null
};

__device__ __forceinline__ void fz_expect(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void fz_bulk(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}

__global__ void __launch_bounds__(FZ_T) mlp_fused_tc_kernel(const FusedArgs g) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  __shared__ __align__(8) unsigned long long full[FZ_S], empty[FZ_S];
  __shared__ uint32_t tmem_slot;
  __shared__ int fail;
  __shared__ float sbias[3][FZ_H];
  const uint32_t s0 = smem_u32(tc_smem);
  const uint32_t sH = smem_u32(tc_smem + FZ_S * FZ_STAGE);
  unsigned char *hptr = tc_smem + FZ_S * FZ_STAGE;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * TC_M;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(256)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int b = 0; b < FZ_S; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[b])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[b])) : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fail = 0;
  }
  for (int j = tid; j < 3 * FZ_H; j += FZ_T) {   // the biases, read by every epilogue
    const int l = j / FZ_H, col = j - l * FZ_H;
    const float *bsrc = l == 0 ? g.b1 : (l == 1 ? g.b2 : g.b3);
    sbias[l][col] = (l < 2 || col < g.No) ? bsrc[col] : 0.f;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  // chunk c (numbered across the layers) uses stage c % FZ_S; its copies
  // complete phase c / FZ_S of full[stage], its MMAs that of empty[stage]
  auto wait_full = [&](int c) { return tc_wait(smem_u32(&full[c % FZ_S]), (uint32_t)((c / FZ_S) & 1)); };
  auto wait_empty = [&](int c) { return tc_wait(smem_u32(&empty[c % FZ_S]), (uint32_t)((c / FZ_S) & 1)); };
  int cbase = 0, produced = -1, issued = -1;
  for (int layer = 0; layer < 3; ++layer) {
    const int N = layer == 2 ? g.No : FZ_H;
    const int nch = layer == 0 ? g.nch1 : FZ_H / FZ_KC;
    const __nv_bfloat16 *Wc = layer == 0 ? g.W1c : (layer == 1 ? g.W2c : g.W3c);
    const float *bias = sbias[layer];
    if (tid == 0 && !fail) {
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
                             ((uint32_t)(TC_M >> 4) << 24);
      auto produce = [&](int i) {   // chunk i of this layer (stage (cbase + i) % FZ_S)
        const int c = cbase + i, b = c % FZ_S;
        const uint32_t a0 = s0 + (uint32_t)b * FZ_STAGE, b0 = a0 + FZ_STAGE_A;
        const uint32_t bytes_b = (uint32_t)N * FZ_KC * 2;
        fz_expect(smem_u32(&full[b]), bytes_b + (layer == 0 ? FZ_STAGE_A : 0u));
        if (layer == 0) fz_bulk(a0, g.Xc + ((long)blockIdx.x * g.nch1 + i) * TC_M * FZ_KC, FZ_STAGE_A, smem_u32(&full[b]));
        fz_bulk(b0, Wc + (long)i * N * FZ_KC, bytes_b, smem_u32(&full[b]));
        produced = c;
      };
      // the stages of this layer's first chunks were last read by batches
      // before cbase, all complete (the previous layer waited for cbase - 1)
      for (int i = 0; i < FZ_P && i < nch; ++i) produce(i);
      for (int i = 0; i < nch; ++i) {
        const int c = cbase + i, b = c % FZ_S;
        if (!wait_full(c)) {
          fail = 1;
          break;
        }
        const uint32_t a0 = s0 + (uint32_t)b * FZ_STAGE, b0 = a0 + FZ_STAGE_A;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int kk = 0; kk < FZ_KC; kk += 16) {
          uint64_t ad;
          if (layer == 0) {
            ad = tc_desc(a0 + (kk >> 3) * 128, 128, (FZ_KC / 8) * 128);
          } else {   // the hidden tile, K-chunks of 64 columns
            const int k = i * FZ_KC + kk;
            ad = tc_desc(sH + (uint32_t)(k / TC_KC) * (TC_M * TC_KC * 2) + ((k % TC_KC) >> 3) * 128, 128,
                         (TC_KC / 8) * 128);
          }
          const uint64_t bd = tc_desc(b0 + (kk >> 3) * 128, 128, (FZ_KC / 8) * 128);
          const uint32_t acc = (i > 0 || kk > 0) ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
              : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&empty[b]))
                     : "memory");
        issued = c;
        if (i + FZ_P < nch) {
          const int prev = c + FZ_P - FZ_S;   // the batch that last read the stage of chunk i + FZ_P
          if (prev >= 0 && !wait_empty(prev)) {
            fail = 1;
            break;
          }
          produce(i + FZ_P);
        }
      }
    }
    __syncthreads();
    // the layer's MMAs complete in issue order: its last batch covers them all
    int ok = !fail;
    if (ok) ok = __syncthreads_and(tc_wait(smem_u32(&empty[(cbase + nch - 1) % FZ_S]),
                                           (uint32_t)(((cbase + nch - 1) / FZ_S) & 1)) ? 1 : 0);
    if (!ok) {
      if (tid == 0) {
        fail = 1;
        // bounded drains: the copies and MMAs this CTA issued must land before it exits
        for (int c = (produced - FZ_S + 1 > 0 ? produced - FZ_S + 1 : 0); c <= produced; ++c) (void)wait_full(c);
        if (issued >= 0) (void)wait_empty(issued);
      }
      __syncthreads();
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // warps w and w + 4 read the same 32 accumulator lanes (rows), the even
    // and the odd 32-column groups, one tensor-memory load of 32 columns each
    const int quarter = warp & 3, half = warp >> 2;
    const int r = quarter * 32 + lane, gm = m0 + r;
    for (int c32 = half * 32; c32 < N; c32 += 64) {
      uint32_t v[32];
      const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c32;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
          "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
            "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
            "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int h16 = 0; h16 < 2; ++h16) {
        const int c0 = c32 + 16 * h16;
        if (c0 >= N) break;
        float x[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          x[j] = __uint_as_float(v[16 * h16 + j]) + bias[c0 + j];
          if (layer < 2) x[j] = fmaxf(x[j], 0.f);
        }
        if (layer < 2) {
          uint32_t w[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) w[q] = pack2(__float2bfloat16(x[2 * q]), __float2bfloat16(x[2 * q + 1]));
          // the next layer's A operand: K chunk c0 / 64, 16-byte groups (c0 % 64) / 8 and + 1
          const int ch = c0 / TC_KC, gq = (c0 % TC_KC) / 8;
          unsigned char *hb = hptr + (size_t)ch * (TC_M * TC_KC * 2);
          *reinterpret_cast<uint4 *>(hb + tc_core_off(r, gq)) = make_uint4(w[0], w[1], w[2], w[3]);
          *reinterpret_cast<uint4 *>(hb + tc_core_off(r, gq + 1)) = make_uint4(w[4], w[5], w[6], w[7]);
          __nv_bfloat16 *Hg = layer == 0 ? g.H1 : g.H2;
          if (Hg && gm < g.M) {
            uint4 *dst = reinterpret_cast<uint4 *>(Hg + (long)gm * FZ_H + c0);
            dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
            dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
          }
        } else if (gm < g.M) {
          float4 *dst = reinterpret_cast<float4 *>(g.Y + (long)gm * g.ldy + c0);
#pragma unroll
          for (int q = 0; q < 4; ++q) dst[q] = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
        }
      }
    }
    // the hidden tile (generic-proxy stores) is read next by the tensor core,
    // and the accumulator columns just read are overwritten by its MMAs
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    cbase += nch;
  }
  if (fail && tid == 0) atomicExch(&g_tc_timeout, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256) : "memory");
}

// Weights transposed for the forward GEMM: Wt[n][k] = W[k][n] for the three
// layers (W1 [Fp][H], W2 [H][H], W3 [H][No] in the parameter vector).
__global__ void transpose_weights_kernel(const __nv_bfloat16 *Pb, long oW1, long oW2, long oW3, int Fp, int H,
                                         int No, __nv_bfloat16 *Pt) {
  const long n1 = (long)H * Fp, n2 = (long)H * H, n3 = (long)No * H;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n1 + n2 + n3; i += (long)gridDim.x * blockDim.x) {
    if (i < n1) {
      const long n = i / Fp, k = i - n * Fp;
      Pt[i] = Pb[oW1 + k * H + n];
    } else if (i < n1 + n2) {
      const long j = i - n1, n = j / H, k = j - n * H;
      Pt[i] = Pb[oW2 + k * H + n];
    } else {
      const long j = i - n1 - n2, n = j / H, k = j - n * H;
      Pt[i] = Pb[oW3 + k * No + n];
    }
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
  // one reciprocal per cell, then FP32 products (the inputs are BF16 anyway;
  // an FP64 division per value would cost more than the whole network here)
  const float inv = ok ? (float)(1.0 / s) : 0.f;
  for (int j = lane; j < ldx; j += 32)
    X[(size_t)w * ldx + j] = __float2bfloat16(j < nf ? (float)value(j) * inv : 0.f);
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

// output errors of the energy-norm objective: row e (a cell), column q < n3:
// factor * c * s_e * g[e n3 + q] (the chain rule through the step
// d_e = c s_e y_e), zero in the padding columns
__global__ void energy_grad_kernel(const double *g, int n3, int E, const float *scale, float cs, double factor,
                                   int ld, __nv_bfloat16 *dY, float *dYf) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long)E * ld) return;
  const int r = (int)(i / ld), q = (int)(i - (long)r * ld);
  const float d = q < n3 ? (float)(factor * (double)cs * (double)scale[r] * g[(size_t)r * n3 + q]) : 0.f;
  dY[i] = __float2bfloat16(d);
  dYf[i] = d;
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
  if (M <= 0 || N <= 0) return cudaSuccess;
  dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM);
  gemm_bf16_kernel<<<grid, 128, 0, s>>>(g);
  note_launch();
  return cudaGetLastError();
}

// Y[c][r] = X[r][c] for r < rows, c < cols (bf16), and Y[c][r] = 0 for rows
// <= r < ldy: the K-contiguous (transposed, zero-padded) operands of the
// weight-gradient products, whose contraction runs over the batch rows.
__global__ void transpose_bf16_kernel(const __nv_bfloat16 *X, int rows, int cols, long ldx, __nv_bfloat16 *Y,
                                      int ldy) {
  __shared__ __nv_bfloat16 t[32][34];
  const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int j = ty; j < 32; j += 8) {
    const int r = r0 + j, c = c0 + tx;
    t[j][tx] = (r < rows && c < cols) ? X[(long)r * ldx + c] : __float2bfloat16(0.f);
  }
  __syncthreads();
  for (int j = ty; j < 32; j += 8) {
    const int c = c0 + j, r = r0 + tx;
    if (c < cols && r < ldy) Y[(long)c * ldy + r] = t[tx][j];
  }
}

cudaError_t mlp_transpose_bf16(const void *X, int rows, int cols, long ldx, void *Y, int ldy, cudaStream_t s) {
  if (rows < 0 || cols < 1 || ldy < rows) return cudaErrorInvalidValue;
  if (ldy == 0) return cudaSuccess;
  const dim3 grid((ldy + 31) / 32, (cols + 31) / 32), block(32, 8);
  transpose_bf16_kernel<<<grid, block, 0, s>>>((const __nv_bfloat16 *)X, rows, cols, ldx, (__nv_bfloat16 *)Y, ldy);
  note_launch();
  return cudaGetLastError();
}

// Pack a [rows][K] bf16 matrix (row stride ld) into blocks of rt rows x 32
// columns in the tensor cores' core-matrix layout (see pack_core_kernel).
cudaError_t mlp_pack_core(const void *src, long ld, int rows, int K, int rt, void *dst, cudaStream_t s) {
  if (rows < 0 || K < 1 || rt < 8 || rt % 8 || ld % 8 || ((uintptr_t)src & 15) || ((uintptr_t)dst & 15))
    return cudaErrorInvalidValue;
  const int nch = (K + FZ_KC - 1) / FZ_KC, ntiles = (rows + rt - 1) / rt;
  const long pieces = (long)ntiles * rt * nch * (FZ_KC / 8);
  if (pieces == 0) return cudaSuccess;
  const int grid = (int)std::min<long>((pieces + 255) / 256, 152L * 16);
  pack_core_kernel<<<grid, 256, 0, s>>>((const __nv_bfloat16 *)src, ld, rows, K, rt, nch, ntiles,
                                        (__nv_bfloat16 *)dst);
  note_launch();
  return cudaGetLastError();
}

// The three layers in one launch (see mlp_fused_tc_kernel): Xc the features
// packed in 128-row tiles of ceil(Fp / 32) chunks, Wc the packed weights
// [256][32 ceil(Fp / 32)], [256][256], [No][256] at oC1, oC2, oC3.
cudaError_t mlp_forward_fused(const void *Xc, int M, int Fp, int No, const void *Wc, long oC1, long oC2, long oC3,
                              const float *b1, const float *b2, const float *b3, float *Y, long ldy, void *H1,
                              void *H2, cudaStream_t s) {
  if (M <= 0) return cudaSuccess;
  if (Fp < 16 || No < 16 || No > 256 || No % 16 || ldy % 4 || ((uintptr_t)Xc & 15) || ((uintptr_t)Y & 15) ||
      ((uintptr_t)H1 & 15) || ((uintptr_t)H2 & 15) || (oC1 % 8) || (oC2 % 8) || (oC3 % 8) || ((uintptr_t)Wc & 15))
    return cudaErrorInvalidValue;
  static bool attr_set[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && !attr_set[dev]) {
    e = cudaFuncSetAttribute(mlp_fused_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, FZ_SMEM);
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  const __nv_bfloat16 *P = (const __nv_bfloat16 *)Wc;
  FusedArgs g{(const __nv_bfloat16 *)Xc, M, (Fp + FZ_KC - 1) / FZ_KC, No, P + oC1, P + oC2, P + oC3, b1, b2, b3,
              Y, ldy, (__nv_bfloat16 *)H1, (__nv_bfloat16 *)H2};
  mlp_fused_tc_kernel<<<(M + TC_M - 1) / TC_M, FZ_T, FZ_SMEM, s>>>(g);
  note_launch();
  return cudaGetLastError();
}

cudaError_t mlp_gemm_tc(const void *A, long lda, const void *Bt, long ldb, int M, int N, int K, const float *bias,
                        int relu, float *Cf, void *Cb, long ldc, cudaStream_t s) {
  if (M <= 0) return cudaSuccess;
  // 16-byte pieces in and out: K-contiguous rows and output rows start on 16 bytes
  if (N < 16 || N > 256 || N % 16 || K < 16 || K % 16 || lda % 8 || ldb % 8 || ldc % 8 || ((uintptr_t)A & 15) ||
      ((uintptr_t)Bt & 15) || ((uintptr_t)Cf & 15) || ((uintptr_t)Cb & 15))
    return cudaErrorInvalidValue;
  static bool attr_set[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && !attr_set[dev]) {
    e = cudaFuncSetAttribute(gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  uint32_t ncols = 32;
  while (ncols < (uint32_t)N) ncols <<= 1;
  TcArgs g{(const __nv_bfloat16 *)A, (const __nv_bfloat16 *)Bt, lda, ldb, M, N, K, bias, relu, Cf,
           (__nv_bfloat16 *)Cb, ldc};
  gemm_tc_kernel<<<(M + TC_M - 1) / TC_M, 128, TC_SMEM, s>>>(g, ncols);
  note_launch();
  return cudaGetLastError();
}

cudaError_t mlp_transpose_weights(const void *Pb, long oW1, long oW2, long oW3, int Fp, int H, int No, void *Pt,
                                  cudaStream_t s) {
  const long n = (long)H * Fp + (long)H * H + (long)No * H;
  transpose_weights_kernel<<<(int)std::min<long>(blocks(n), 152L * 8), 256, 0, s>>>(
      (const __nv_bfloat16 *)Pb, oW1, oW2, oW3, Fp, H, No, (__nv_bfloat16 *)Pt);
  note_launch();
  return cudaGetLastError();
}

cudaError_t mlp_tc_status(int *timed_out) {
  int v = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_tc_timeout, sizeof(int));
  if (e == cudaSuccess && v) {
    const int z = 0;
    e = cudaMemcpyToSymbol(g_tc_timeout, &z, sizeof(int));
  }
  *timed_out = v;
  return e;
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
cudaError_t mlp_energy_grad(const double *g, int n3, int E, const float *scale, float cs, double factor, int ld,
                            void *dY, float *dYf, cudaStream_t s) {
  if (E <= 0) return cudaSuccess;
  energy_grad_kernel<<<blocks((long)E * ld), 256, 0, s>>>(g, n3, E, scale, cs, factor, ld, (__nv_bfloat16 *)dY, dYf);
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
