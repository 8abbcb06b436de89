// Internal interfaces of libsipg: kernel argument blocks, level data and the
// launchers each translation unit provides.  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sipg.h"

namespace sipg {

constexpr int kMaxN = 9;   // points per direction, k = 1..8

// Host copy of the 1D tables for one n (points per direction), in double.
// Basis: Lagrange on the n Gauss-Lobatto nodes; quadrature: n-point Gauss.
struct Rules1D {
  int n = 0;
  std::vector<double> gl;      // GL nodes on [0,1]
  std::vector<double> xq, wq;  // Gauss points and weights on [0,1]
  std::vector<double> S;       // S[q*n+i]  = l_i(x_q)                 (Gauss x GL)
  std::vector<double> Sd;      // Sd[q*n+i] = l_i'(x_q)
  std::vector<double> D;       // D[q*n+r]  = lG_r'(x_q), Lagrange on Gauss points
  std::vector<double> l0, l1;  // lG_q(0), lG_q(1)
  std::vector<double> lp0, lp1;// l_i'(0), l_i'(1)  (GL basis)
};
const Rules1D &rules(int n);
void gauss_rule(int n, std::vector<double> &x, std::vector<double> &w);   // any n >= 1, on [0,1]
std::vector<double> lagrange_values(const std::vector<double> &nodes, double x);
std::vector<double> lagrange_derivs(const std::vector<double> &nodes, double x);

// Device-side 1D tables for all n in one block, uploaded to constant memory of
// every translation unit that launches sum-factorisation kernels.
template <typename T>
struct Tables {
  // plain n x n matrices (used for n <= 4), stride n
  T S[kMaxN + 1][16], St[kMaxN + 1][16], D[kMaxN + 1][16], Dt[kMaxN + 1][16];
  // even-odd blocks (n >= 5): E[hc][hc] stride 5, O[hc][h] stride 4
  T SE[kMaxN + 1][25], SO[kMaxN + 1][20], StE[kMaxN + 1][25], StO[kMaxN + 1][20];
  T DE[kMaxN + 1][25], DO[kMaxN + 1][20], DtE[kMaxN + 1][25], DtO[kMaxN + 1][20];
  T l0[kMaxN + 1][kMaxN], l1[kMaxN + 1][kMaxN];
  // D^T l0 and D^T l1: the transposed derivative sweep applied to the face
  // extrapolation vectors (a face's normal-derivative test term enters the
  // integrated tile through these directly)
  T dl0[kMaxN + 1][kMaxN], dl1[kMaxN + 1][kMaxN];
  // 1D mass and stiffness matrices of the GL basis under the Gauss rule,
  // M1[i][j] = sum_q w_q l_i(x_q) l_j(x_q), K1[i][j] = sum_q w_q l_i'(x_q) l_j'(x_q)
  // (both M[i][j] = M[n-1-i][n-1-j]): the factors of the Cartesian FE cell matrix
  T M1[kMaxN + 1][16], K1[kMaxN + 1][16];
  T M1E[kMaxN + 1][25], M1O[kMaxN + 1][20], K1E[kMaxN + 1][25], K1O[kMaxN + 1][20];
  // the collocation stiffness at the Gauss points, KG[i][j] = sum_q D[q][i] w_q D[q][j]
  // (KG[i][j] = KG[n-1-i][n-1-j]): the cell term of an axis-aligned DG cell along one direction
  T KG[kMaxN + 1][16], KGE[kMaxN + 1][25], KGO[kMaxN + 1][20];
};
template <typename T>
void build_tables(Tables<T> &t);

// Arguments of the DG evaluation / integration passes.
template <typename T>
struct DGArgs {
  const T *u;          // input vector (cell-major, n^3 per cell)
  T *out;              // output (mode dependent)
  T *grad;             // scratch: reference gradient at Gauss points, [cell][3][n^3]
  T *trace;            // scratch: face traces, [cell][6 faces][2 (value, d_n)][n^2]
  const T *metric;     // curved: [cell][6][n^3] = w|detJ| J^-1 J^-T (xx,yy,zz,xy,xz,yz)
  const T *wcart;      // Cartesian: [3][n^3] = w_q * prod(h)/h_d^2
  const T *fdA[3];     // curved: [face][n^2] area element times weights
  const T *fc[3];      // curved: [face][2 roles][3][n^2] = J^-1 n_outward (own side)
  const T *fwcart;     // Cartesian: [3][n^2] = w_q1 w_q2 h_t1 h_t2
  const T *tau;        // [cell] penalty tau_e
  T ih[3];             // Cartesian 1/h_d
  int m[3];
  int ncells;
  int bc[6];
  // 1: the evaluation pass does not store the gradient and the integration
  // pass recomputes it from u (less traffic, more arithmetic: used in FP32)
  int recompute;
  // epilogue: mode 0 out = Au; 1 out = c1 x + c2 xp + c3 dinv (b - Au); 2 out = b - Au
  int mode;
  const T *x, *xp, *b, *dinv;
  T c1, c2, c3;
  // nv vectors of one operator at once (right-hand sides): vector r of u,
  // out, x, xp, b starts at r * vs, its scratch at r * gs (grad) and r * ts
  // (trace); dinv and the geometry are shared
  int nv = 1;
  int64_t vs = 0, gs = 0, ts = 0;
  // unstructured meshes (null on the structured box): per cell and local face
  // f = 2 d + s (the face xi_d = s), x = neighbour cell or -1 (Dirichlet) /
  // -2 (Neumann), y = neighbour's local face | orientation code << 3; the
  // face geometry is then per cell and local face: fdA[0] [cell][6][n^2],
  // fc[0] [cell][6][3][n^2] (own side J^-1 n, n the outward unit normal)
  const int2 *ufn = nullptr;
};

// Arguments of the FE cell pass and the node gather pass.
template <typename T>
struct FEArgs {
  const T *u;
  T *ebuf;             // [cell][n^3]
  T *out;
  const T *metric;     // curved [cell][6][n^3]
  const T *wcart;      // Cartesian [3][n^3]
  int m[3];
  int deg;             // polynomial degree p (n = p+1)
  int grid[3];         // node grid = m*p+1
  int ncells;
  int bc[6];
  int mode;            // gather: 0 apply, 1 chebyshev, 2 residual, 3 restrict (sum, constrained -> 0),
                       //         4 diagonal (sum, constrained -> 1), 5 restrict and the coarse
                       //         level's first Chebyshev step: out2 = c3 dinv out
  const T *x, *xp, *b, *dinv;
  T c1, c2, c3;
  T alpha[3];          // Cartesian: prod(h) / h_d^2, the scale of direction d's term
  T *out2 = nullptr;   // mode 5
  // nv vectors at once: vector r of u, out, x, xp, b starts at r * vs, its
  // element buffer at r * es
  int nv = 1;
  int64_t vs = 0, es = 0;
};

// One multigrid level.
struct Level {
  int kind = 0;         // 0 DG, 1 FE
  int deg = 1, n = 2;
  int m[3] = {1, 1, 1};
  int grid[3] = {1, 1, 1};
  int64_t ncells = 0, ndofs = 0;
  bool curved = false;
  double h[3] = {1, 1, 1};
  // geometry in both precisions ([0] double, [1] float)
  void *metric[2] = {nullptr, nullptr};
  void *wcart[2] = {nullptr, nullptr};
  void *fdA[2][3] = {{nullptr}}, *fc[2][3] = {{nullptr}};
  void *fwcart[2] = {nullptr, nullptr};
  void *tau[2] = {nullptr, nullptr};
  int2 *ufn = nullptr;   // unstructured face neighbours (DGArgs::ufn)
  void *dinv[2] = {nullptr, nullptr};
  double lambda = 0;
  // cells per thread block of the cell kernels, [precision][DG evaluation,
  // DG integration, FE cells]: cb0 is the setup default (the compiled
  // default, lowered on meshes with fewer blocks than SMs), cb the width in
  // use (cb0, the autotuner's choice or a set value; 0 = compiled default)
  int cb[2][3] = {{0, 0, 0}, {0, 0, 0}};
  int cb0[2][3] = {{0, 0, 0}, {0, 0, 0}};
  // FE levels of low degree: assembled stencil [(2p+1)^3][nodes] in both
  // precisions (nullptr: matrix-free)
  void *stencil[2] = {nullptr, nullptr};
  // transfer from level l-1 (coarser) to this level
  int t_kind = -1;      // 0 c-transfer, 1 FE p, 2 FE h, 3 DG p, 4 DG h
  void *P1[2] = {nullptr, nullptr};   // [2 children][nf][nc] interpolation tables
  // V-cycle work vectors in the V-cycle precision (and FP64 for setup)
  void *vb[2] = {nullptr, nullptr}, *vx[2] = {nullptr, nullptr}, *vr[2] = {nullptr, nullptr},
       *vt[2] = {nullptr, nullptr};
};

// Launchers (one per precision; defined in the kernel translation units).
template <typename T>
void upload_tables_dg(const Tables<T> &t);
template <typename T>
void upload_tables_fe(const Tables<T> &t);
template <typename T>
void upload_tables_batch(const Tables<T> &t);

template <typename T>
cudaError_t launch_dg_eval(int n, bool curved, const DGArgs<T> &a, cudaStream_t s, int cb = 0);
template <typename T>
cudaError_t launch_dg_integrate(int n, bool curved, const DGArgs<T> &a, cudaStream_t s, int cb = 0);
template <typename T>
int dg_cells_per_block(int n);
template <typename T>
int dg_max_cells_per_block(int n);
// resident blocks per SM of a DG pass (0 evaluation, 1 integration) at cb cells per block
template <typename T>
cudaError_t dg_blocks_per_sm(int n, bool curved, int pass, int cb, int *blocks);

cudaError_t launch_dg_diag(int n, bool curved, const DGArgs<double> &a, double *diag, cudaStream_t s);

// FE cell pass at cb cells per block (0 = default); diag_only: the cell-local
// diagonal (setup, FP64)
template <typename T>
cudaError_t launch_fe_cells(int n, bool curved, const FEArgs<T> &a, bool diag_only, cudaStream_t s, int cb = 0);
template <typename T>
int fe_max_cells_per_block(int n);
template <typename T>
cudaError_t fe_blocks_per_sm(int n, bool curved, int cb, int *blocks);
template <typename T>
cudaError_t launch_fe_gather(const FEArgs<T> &a, cudaStream_t s);
// Assembled stencil of an FE level of degree 1 or 2 (setup, FP64):
// coef[o][node], o over the (2p+1)^3 offsets, x fastest
cudaError_t launch_fe_stencil_setup(bool curved, const FEArgs<double> &a, double *coef, cudaStream_t s);
// the level operator from its stencil with the gather's epilogue (modes 0-2)
template <typename T>
cudaError_t launch_fe_stencil_apply(const FEArgs<T> &a, const T *coef, cudaStream_t s);

// Transfers.  For the c-transfer the coarse space is the FE space on the same
// mesh with the same degree: prolongation injects, restriction sums duplicates.
// (nv vectors: xc at r * fe.vs, xdg at r * dg_stride)
template <typename T>
cudaError_t launch_c_prolongate_add(const FEArgs<T> &fe, const T *xc, T *xdg, cudaStream_t s, int64_t dg_stride = 0);
struct XferGeom {
  int kind;             // 1 FE p, 2 FE h, 3 DG p, 4 DG h
  int mf[3], mc[3];     // cells of fine and coarse mesh
  int pf, pc;           // degrees
  int gf[3], gc[3];     // node grids
  int bc[6];
  // nv vectors at once: vector r of the fine / coarse vector starts at r * sf
  // / r * sc, of the coarse element buffer at r * se
  int nv = 1;
  int64_t sf = 0, sc = 0, se = 0;
};
template <typename T>
cudaError_t launch_fe_prolongate_add(const XferGeom &g, const T *P1, const T *xc, T *xf, cudaStream_t s);
template <typename T>
cudaError_t launch_fe_restrict_cells(const XferGeom &g, const T *P1, const T *rf, T *ebuf_c, cudaStream_t s);
// node-by-node restriction r_c = P^T r_f in one launch, for the transfers
// degree 2 -> 1 on one mesh and degree 1 across a 2:1 refinement
inline bool fe_restrict_nodes_ok(const XferGeom &g) {
  return (g.kind == 1 && g.pf == 2 && g.pc == 1) || (g.kind == 2 && g.pf == 1 && g.pc == 1);
}
template <typename T>
cudaError_t launch_fe_restrict_nodes(const XferGeom &g, const T *P1, const T *rf, T *rc, cudaStream_t s);

// The lower end of the V-cycle (Algorithm 2 below a size bound) in one
// launch of one thread-block cluster: the degree-1 FE levels applied by their
// 27-point stencils, the 2:1 transfers between them and the dense coarse
// inverse, each step a pass over the level's nodes followed by a cluster
// barrier.  Every value is computed with the arithmetic, in the order, of the
// per-step kernels (launch_xdb, launch_fe_stencil_apply, launch_fe_restrict_nodes,
// launch_dense_gemv, launch_fe_prolongate_add), so both give the same bits.
enum TailOp : int { kTailXdb = 0, kTailStencil = 1, kTailRestrict = 2, kTailCoarse = 3, kTailProlong = 4 };
template <typename T>
struct alignas(16) TailStep {
  int op;                 // TailOp
  int mode;               // kTailStencil: 1 Chebyshev step, 2 residual (as FEArgs::mode)
  int n;                  // nodes of the step's output (kTailCoarse: unknowns of the coarse level)
  int grid[3];            // node grid of the level (kTailStencil)
  int bc[6];
  const T *u;             // stencil: operand; transfers: input vector
  const T *x, *xp, *b, *dinv, *coef;
  T *out;                 // xdb, stencil, restriction, coarse: written; prolongation: out += P u
  T c1, c2, c3;
  XferGeom g;             // kTailRestrict, kTailProlong
  const T *P1;
  const double *Ainv;     // kTailCoarse: [n][n]
};
constexpr int kTailThreads = 512;     // threads per block of the cluster
constexpr int kTailMaxNodes = 8192;   // largest level taken into the fused tail
constexpr int kTailMaxCoarse = 1000;  // largest dense coarse level taken
constexpr int kTailMaxSteps = 160;    // the program sits in shared memory
// the cluster size the device runs the tail kernel with (16, else 8; 0: none)
template <typename T>
int fe_tail_cluster(int nsteps);
template <typename T>
cudaError_t launch_fe_tail(const TailStep<T> *prog, int nsteps, int cluster, cudaStream_t s);
// DG -> DG transfers (kind 3 p, 4 h): prolong: out += P in; else out = P^T in
template <typename T>
cudaError_t launch_dg_transfer(const XferGeom &g, const T *P1, const T *in, T *out, bool prolong, cudaStream_t s);

// Vector kernels.
template <typename T>
cudaError_t launch_fill(T *x, T v, int64_t n, cudaStream_t s);
template <typename Tout, typename Tin>
cudaError_t launch_cast(Tout *y, const Tin *x, int64_t n, cudaStream_t s);
// b = (T) r and x = c D^-1 b (the first Chebyshev step from x = 0) in one pass
template <typename T, typename Tin>
cudaError_t launch_cast_xdb(T *b, T *x, T c, const T *dinv, const Tin *r, int64_t n, cudaStream_t s);
template <typename T>
cudaError_t launch_axpy(T *y, T a, const T *x, int64_t n, cudaStream_t s);   // y += a x
cudaError_t launch_invert(double *d, int64_t n, cudaStream_t s);
template <typename T>
cudaError_t launch_xdb(T *x, T c, const T *dinv, const T *b, int64_t n, cudaStream_t s,
                      int nv = 1);   // x = c dinv b, nv vectors of length n (dinv shared)
template <typename T>
cudaError_t launch_xpby(T *p, const T *z, T beta, int64_t n, cudaStream_t s);              // p = z + beta p
// deterministic dot products into device scalars: out[0] = x.y (and out[1] = z.w if z)
cudaError_t launch_dot2(const double *x, const double *y, const double *z, const double *w, int64_t n,
                        double *partials, unsigned *counter, double *out, cudaStream_t s);
// FCG helpers (scalars in device memory, see solver.cu for the layout)
cudaError_t launch_fcg_update_xr(double *x, double *r, const double *p, const double *v, int64_t n,
                                 const double *sc, double *partials, unsigned *counter, double *out,
                                 cudaStream_t s);
cudaError_t launch_fcg_update_p(double *p, const double *z, const double *sc, int64_t n, cudaStream_t s);
// device-gated flexible-CG steps (vec_kernels.cu): prm points to {double rtol; int maxit, fixed;}
cudaError_t launch_fcg_check(const double *sc, double *hist, int *st, const void *prm, cudaGraphConditionalHandle next,
                             cudaStream_t s);
cudaError_t launch_fcg_cond(const int *st, cudaGraphConditionalHandle h, cudaStream_t s);
// coarse-level Jacobi-PCG with device-resident FP64 scalars (cycle precision T)
template <typename T>
cudaError_t launch_cg_dot(const T *x, const T *y, int64_t n, double *partials, unsigned *counter, double *out,
                          cudaStream_t s);
template <typename T>
cudaError_t launch_cg_update_xr(T *x, T *r, const T *p, const T *q, int64_t n, const double *gamma, const double *pq,
                                cudaStream_t s);
template <typename T>
cudaError_t launch_cg_update_p(T *p, const T *z, int64_t n, const double *gnew, const double *gold, cudaStream_t s);
template <typename Tb, typename Tx>
cudaError_t launch_dense_gemv(const double *Ainv, const Tb *b, Tx *x, int n, cudaStream_t s, int nv = 1);

cudaError_t fma_peak(int precision, cudaStream_t s, double *flops);

// ---- batched problems (batch.cu)
template <typename T>
struct BatchProb {
  DGArgs<T> a;
  int n;
  int active;
};

struct WorkItem {
  int p, cell0, ncta;
};

// Per-problem segments for the batched vector kernels.
struct Seg {
  double *x, *r, *p, *v, *z;
  const double *b;
  long n;
  int active;
};

// Batched FE passes (fe_kernels.cu): one task per problem, one thread block
// per item.  Cell items cover kBatchCellThreads / n^2 cells, node items
// kBatchNodeThreads nodes (or DG points for the c-prolongation).
constexpr int kBatchCellThreads = 256;
constexpr int kBatchNodeThreads = 256;
template <typename T>
struct FETask {
  FEArgs<T> a;
  const T *xc = nullptr;   // c-prolongation: FE input and DG output
  T *xdg = nullptr;
};
struct NodeItem {
  int p, blk;
};
template <typename T>
cudaError_t launch_fe_cells_batched(bool curved, const FETask<T> *tasks, const WorkItem *items, int nitems,
                                    size_t smem, const Seg *segs, cudaStream_t s);
// kind 0: gather with each task's mode and epilogue; 1: c-prolongation
template <typename T>
cudaError_t launch_fe_nodes_batched(const FETask<T> *tasks, const NodeItem *items, int nitems, const Seg *segs,
                                    int kind, cudaStream_t s);
template <typename T>
cudaError_t prep_fe_cells_batched(size_t smem);
int tile_values(int n);   // shared-memory values per cell of the cell passes (sumfac.cuh)
// batched vector steps (batch.cu); op as in vec_batched_kernel
struct VecTask {
  int op = 0;
  long n = 0;
  void *y = nullptr;
  const void *x = nullptr, *d = nullptr;
  double c = 0;
};
cudaError_t launch_vec_batched(const VecTask *tasks, const NodeItem *items, int nitems, const Seg *segs,
                               cudaStream_t s);
// lockstep flexible CG gated on the device (batch.cu): per-system iteration
// count, status (1 breakdown, 2 maxit), ||r|| history [np][257] and last
// ||r||; prm = {rtol, maxit} (device); *any = some system still iterates
cudaError_t launch_batch_fcg_check(const double *sc, int stride, Seg *segs, int np, int *it, int *status, double *hist,
                                   double *rn, const double *r0, const double *prm, int *any,
                                   cudaGraphConditionalHandle next, cudaStream_t s);
cudaError_t launch_batch_fcg_cond(const int *any, cudaGraphConditionalHandle h, cudaStream_t s);

template <typename T>
struct BatchPlan {
  std::vector<BatchProb<T>> probs;
  std::vector<WorkItem> items;
  BatchProb<T> *d_probs = nullptr;
  WorkItem *d_items = nullptr;
  size_t smem = 0;
  int grid = 0;
  bool curved = false;
};

template <typename T>
cudaError_t batch_plan_build(BatchPlan<T> &P, const std::vector<DGArgs<T>> &args, const std::vector<int> &ns);
template <typename T>
void batch_plan_free(BatchPlan<T> &P);
template <typename T>
cudaError_t batch_apply(BatchPlan<T> &P, cudaStream_t s);
// one pass of the batched DG operator with the descriptors probs (device)
template <typename T>
cudaError_t batch_dg_pass(const BatchPlan<T> &P, const BatchProb<T> *probs, bool integrate, const Seg *segs,
                          cudaStream_t s);
constexpr int kSegSlots = 8;   // scalar slots per problem (FCG layout of solver.cu, 4: b.b, 5: r0.r0)
// Block map of the batched vector kernels (batch.cu): g.nb[p] blocks for
// system p, one per kSegChunk entries (at least one), its partial sums at
// partials[2 (g.off[p] + j)]; partials hold 2 g.blocks values
constexpr long kSegChunk = 8192;
struct SegGrid {
  const int2 *map = nullptr;
  const int *off = nullptr, *nb = nullptr;
  int blocks = 0;
};
cudaError_t seg_grid_build(const std::vector<long> &n, SegGrid &g, std::vector<void *> &allocs);
cudaError_t seg_dot(const Seg *segs, const SegGrid &g, int which, double *partials, unsigned *counter, double *sc,
                    int sc_stride, int slot, cudaStream_t s);
cudaError_t seg_update_xr(const Seg *segs, const SegGrid &g, double *partials, unsigned *counter, double *sc,
                          int sc_stride, cudaStream_t s);
cudaError_t seg_update_p(const Seg *segs, const SegGrid &g, const double *sc, int sc_stride, int init, cudaStream_t s);

// ---- learned smoother network (mlp.cu); bf16 buffers passed as void*
cudaError_t mlp_gemm(const void *A, long sam, long sak, const void *B, long sbk, long sbn, int M, int N, int K,
                     const float *bias, int relu, float *Cf, void *Cb, long ldc, int accumulate, cudaStream_t s);
// C = A Bt^T on tcgen05 tensor cores (A [M][lda], Bt [N][ldb], both K
// contiguous, BF16; N a multiple of 16 up to 256, K a multiple of 16)
cudaError_t mlp_gemm_tc(const void *A, long lda, const void *Bt, long ldb, int M, int N, int K, const float *bias,
                        int relu, float *Cf, void *Cb, long ldc, cudaStream_t s);
// Pt = the three weight matrices transposed (K contiguous) for mlp_gemm_tc
cudaError_t mlp_transpose_weights(const void *Pb, long oW1, long oW2, long oW3, int Fp, int H, int No, void *Pt,
                                  cudaStream_t s);
// reads and clears the flag a tensor-core GEMM sets when its MMA completion
// wait ran out (the CTA then wrote no output)
cudaError_t mlp_tc_status(int *timed_out);
cudaError_t mlp_transpose_bf16(const void *X, int rows, int cols, long ldx, void *Y, int ldy, cudaStream_t s);
cudaError_t mlp_pack_core(const void *src, long ld, int rows, int K, int rt, void *dst, cudaStream_t s);
cudaError_t mlp_forward_fused(const void *Xc, int M, int Fp, int No, const void *Wc, long oC1, long oC2, long oC3,
                              const float *b1, const float *b2, const float *b3, float *Y, long ldy, void *H1,
                              void *H2, cudaStream_t s);
template <typename T>
cudaError_t mlp_gather(const T *r, int n, const int m[3], const int *cells, int c0, int nc, void *X, int ldx,
                       float *scale, cudaStream_t s);
template <typename T>
cudaError_t mlp_correct(T *x, int n3, int c0, int nc, const float *Y, int ldy, const float *scale, float c,
                        cudaStream_t s);
cudaError_t mlp_mse_grad(const float *Y, const float *Tg, long ldt, int B, int N, int ld, void *dY, float *dYf,
                         double *loss, cudaStream_t s);
cudaError_t mlp_relu_mask(void *dH, const void *H, long n, cudaStream_t s);
// output errors of the energy-norm objective from g = dL/dd (DG vector) through d_e = cs s_e y_e
cudaError_t mlp_energy_grad(const double *g, int n3, int E, const float *scale, float cs, double factor, int ld,
                            void *dY, float *dYf, cudaStream_t s);
cudaError_t mlp_colsum(const void *D, int bf16, int B, int N, int ld, float *g, cudaStream_t s);
cudaError_t mlp_adam(float *p, float *m, float *v, const float *g, long n, float lr, int step, void *pb,
                     cudaStream_t s);
cudaError_t mlp_f2bf(const float *x, void *y, long n, cudaStream_t s);
cudaError_t mlp_targets(const double *e, int n3, const int *cells, int c0, int nc, const float *scale, float *T,
                        int ldt, cudaStream_t s);
cudaError_t mlp_sumsq(const float *x, long n, double *out, cudaStream_t s);
cudaError_t mlp_scale(float *x, long n, float a, cudaStream_t s);
cudaError_t mlp_stats(const float *x, long n, unsigned *maxbits, unsigned long long *bad, cudaStream_t s);
cudaError_t mlp_pad_f2bf(const float *X, int B, int F, int Fp, void *Y, cudaStream_t s);
cudaError_t mlp_bf2f(const void *X, long n, float *Y, cudaStream_t s);

// Kernel-launch accounting (every launch of the library increments it).
void note_launch();
unsigned long long launch_count();

// Smoothed-aggregation AMG-CG coarse solver (amg.cu).
struct Csr;
struct AmgCoarse;
AmgCoarse *amg_create(const Csr &A0, double rtol, int maxit, double cheb_lo, double cheb_hi, std::string *err);
void amg_destroy(AmgCoarse *M);
int amg_level_sizes(const AmgCoarse *M, int *sizes, int max);
cudaError_t amg_vcycle(AmgCoarse *M, const double *b, double *x, cudaStream_t s);
cudaError_t amg_solve(AmgCoarse *M, const double *b, double *x, cudaStream_t s);
cudaError_t amg_last_iterations(AmgCoarse *M, int *iterations, cudaStream_t s);
template <typename T>
cudaError_t prepare_dg_kernels();
cudaError_t prepare_fe_kernels();

// Text returned by sipg_last_error(NULL).
void set_global_error(const std::string &msg);

}  // namespace sipg
