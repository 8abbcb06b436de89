// Context, setup, V-cycle, Chebyshev smoother, flexible CG and the C ABI
// (Section 3 of the paper: Algorithms 1-3, the cph level hierarchy, the
// coarse solve; Section 4: mixed precision).
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <map>
#include <memory>
#include <mutex>
#include <stdexcept>
#include <string>
#include <tuple>

#include "geometry.h"
#include "sipg_internal.h"

using namespace sipg;

struct sipg_ctx {
  bool unstructured = false;   // built by sipg_create_unstructured (operator only)
  sipg_mesh mesh{};
  sipg_params prm{};
  MeshDesc md{};
  cudaStream_t stream = nullptr;
  bool solver = false;
  std::vector<Level> lv;   // 0 = coarsest, L = finest DG
  int L = 0;
  void *dg_grad[2] = {nullptr, nullptr}, *dg_trace[2] = {nullptr, nullptr};
  void *ebuf[2] = {nullptr, nullptr};
  double *Ainv = nullptr;
  int n0 = 0;
  // coarsest level too large for the dense inverse: fixed Jacobi-PCG
  // iterations on it (p, q work vectors in both precisions)
  bool coarse_cg = false;
  double *cg_p = nullptr, *cg_q = nullptr;   // FP64 search and product vectors of the coarse CG
  AmgCoarse *amg = nullptr;                  // coarse_solver 0: the AMG-CG instead of Jacobi-PCG
  double *fr = nullptr, *fz = nullptr, *fp = nullptr, *fv = nullptr, *fx = nullptr, *fb = nullptr;
  double *scal = nullptr, *partials = nullptr;
  unsigned *counter = nullptr;
  std::vector<void *> allocs;
  std::string err;
  // V-cycle of the solver captured as a CUDA graph (per precision), reading
  // fr and writing fz; captured on the second use, replayed afterwards
  cudaGraphExec_t vgraph[2] = {nullptr, nullptr};
  int vcalls[2] = {0, 0};
  // learned smoother of the finest level (see "learned smoother" below)
  struct Net {
    bool ready = false;    // weights allocated
    bool trained = false;
    int F = 0, Fp = 0, H = 256, No = 0, n3 = 0;
    long oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0, np = 0;
    float cscale = 1.f;    // output scale c: correction = c * s * y
    float *P = nullptr, *M = nullptr, *V = nullptr, *G = nullptr;   // fp32 params, Adam moments, grads
    void *Pb = nullptr;    // bf16 copy of P
    void *Pt = nullptr;    // bf16 weights transposed (K contiguous) for the tensor-core forward pass
    long oT1 = 0, oT2 = 0, oT3 = 0;
    // packed operands of the fused forward (hidden width 256, outputs <= 256):
    // weights in K chunks of 32 at oC1..oC3, features of up to `rows` rows
    void *Wc = nullptr, *Xc = nullptr;
    long oC1 = 0, oC2 = 0, oC3 = 0;
    int Fc = 0;   // first layer's K rounded up to whole chunks
    // inference / training buffers for up to `rows` rows
    long rows = 0;
    void *X = nullptr, *H1 = nullptr, *H2 = nullptr, *dY = nullptr, *dH = nullptr;
    void *TA = nullptr, *TB = nullptr;   // transposed operands of the weight gradients [feature][row]
    float *Y = nullptr, *dYf = nullptr, *scale = nullptr;
    double *loss = nullptr;
    double rho_cheb = 1.0;  // average rate of the Chebyshev cycle (judge of the learned one)
    // time of one flexible-CG iteration with each cycle (V-cycle + outer
    // operator), measured after training; the learned cycle must reduce the
    // residual at least as fast per unit time as the Chebyshev cycle
    double t_iter_cheb = 0, t_iter_learned = 0;
    double omega = 1;       // damping applied to the trained output scale
    double step_reduction = 1;   // residual reduction of one damped step on that data
    int steps_pre = 0, steps_post = 1;   // Chebyshev pre-smoothing, one network post-step
    // full-mesh snapshots of the training data (residual, error of the state
    // the post-smoother starts from), kept for the energy-norm fine-tuning
    int nsnap = 0;
    double *snap_r = nullptr, *snap_e = nullptr;
  } net;
  // Several right-hand sides at once (sipg_solve_multi, sipg_operator_apply_multi):
  // nv vectors of every level's V-cycle data and of the cell-kernel scratch,
  // vector r of a level at r * (that level's length).  nv = 1 uses the
  // single-vector buffers above.
  int nv = 1;
  struct Multi {
    int cap = 0;                               // vectors allocated
    std::vector<void *> v;                     // [level][vb, vx, vr, vt], V-cycle precision
    void *grad[2] = {nullptr, nullptr}, *trace[2] = {nullptr, nullptr}, *ebuf[2] = {nullptr, nullptr};
    double *r = nullptr, *z = nullptr, *p = nullptr, *v_ = nullptr;   // flexible-CG vectors
    std::vector<Seg> segs;
    Seg *d_segs = nullptr;
    SegGrid sg;                                // block map of the batched vector kernels
    std::vector<void *> sg_allocs;
    double *sc = nullptr, *partials = nullptr;
    unsigned *counters = nullptr;
    cudaGraphExec_t graph = nullptr;           // V-cycle of graph_nv vectors
    int graph_nv = 0, calls = 0;
  } mv;
  int smoother = 0;          // 0 Chebyshev, 1 learned (finest level), 2 learned without fallback
  int use_learned = 0;       // current cycle uses the learned smoother
  cudaGraphExec_t vgraph_l[2] = {nullptr, nullptr};   // graphs of the learned cycle
  int vcalls_l[2] = {0, 0};
  // Flexible-CG iterations gated on the device (non-default stream,
  // Chebyshev cycle, one vector): a chunk of kFcgChunk iterations captured
  // once per cycle precision, each iteration two conditional (IF) nodes whose
  // conditions the iteration's own kernels set; the host reads the state once
  // per chunk.  State and parameters in device memory (see fcg_check_kernel).
  cudaGraphExec_t fcg_graph[2] = {nullptr, nullptr};
  int *fcg_state = nullptr;
  double *fcg_hist = nullptr;
  void *fcg_prm = nullptr;
  cudaStream_t cap_stream = nullptr;   // captures the bodies of the conditional nodes
  std::vector<long long> fcg_kA, fcg_kB;   // kernels in each iteration's two bodies
  // kernels captured into each graph, added to the launch count per replay
  std::map<cudaGraphExec_t, long long> graph_kernels;
  // The fused lower cycle (launch_fe_tail) in the cycle precision: for every
  // level t = 1..tail_top the device program of vcycle_rec(t) and the buffer
  // that holds x^(t) after it (index t; entry 0 unused)
  int tail_top = 0, tail_cluster = 0;
  std::vector<void *> tail_prog, tail_x;
  std::vector<int> tail_steps;
};

static std::string g_create_err;

void sipg::set_global_error(const std::string &msg) { g_create_err = msg; }

static std::atomic<unsigned long long> g_launches{0};
// while a stream capture runs on this thread, launches go to its tally
static thread_local long long *t_capture_tally = nullptr;
void sipg::note_launch() {
  if (t_capture_tally) ++*t_capture_tally;
  else g_launches.fetch_add(1, std::memory_order_relaxed);
}
static void note_kernels(long long k) { g_launches.fetch_add((unsigned long long)k, std::memory_order_relaxed); }
// counts the launches noted in its scope into *tally instead of the total
struct CaptureTally {
  long long *prev;
  explicit CaptureTally(long long *tally) : prev(t_capture_tally) { t_capture_tally = tally; }
  ~CaptureTally() { t_capture_tally = prev; }
};
unsigned long long sipg::launch_count() { return g_launches.load(std::memory_order_relaxed); }

namespace {

struct Fail {
  sipg_status st;
};

#define CK(...)                                                                        \
  do {                                                                                 \
    cudaError_t e_ = (__VA_ARGS__);                                                         \
    if (e_ != cudaSuccess) {                                                           \
      throw_cuda(e_, #__VA_ARGS__, __LINE__);                                               \
    }                                                                                  \
  } while (0)

thread_local std::string *t_err = nullptr;

[[noreturn]] void throw_cuda(cudaError_t e, const char *what, int line) {
  if (t_err) {
    char buf[512];
    snprintf(buf, sizeof(buf), "CUDA error %s (%s) at solver.cu:%d in %s", cudaGetErrorName(e),
             cudaGetErrorString(e), line, what);
    *t_err = buf;
  }
  throw Fail{e == cudaErrorMemoryAllocation ? SIPG_ENOMEM : SIPG_ECUDA};
}
[[noreturn]] void throw_inval(const std::string &msg) {
  if (t_err) *t_err = msg;
  throw Fail{SIPG_EINVAL};
}

template <typename T>
T *dalloc(sipg_ctx *c, int64_t n) {
  void *p = nullptr;
  CK(cudaMalloc(&p, (size_t)std::max<int64_t>(n, 1) * sizeof(T)));
  c->allocs.push_back(p);
  return (T *)p;
}

// upload host doubles as both precisions
void upload2(sipg_ctx *c, const std::vector<double> &h, void *out[2]) {
  if (h.empty()) {
    out[0] = out[1] = nullptr;
    return;
  }
  double *d = dalloc<double>(c, (int64_t)h.size());
  float *f = dalloc<float>(c, (int64_t)h.size());
  CK(cudaMemcpy(d, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice));
  CK(launch_cast<float, double>(f, d, (int64_t)h.size(), nullptr));
  out[0] = d;
  out[1] = f;
}

template <typename T>
constexpr int pidx() {
  return sizeof(T) == 8 ? 0 : 1;
}

template <typename T>
DGArgs<T> dg_args(sipg_ctx *c, const Level &L) {
  constexpr int pi = pidx<T>();
  DGArgs<T> a{};
  a.grad = (T *)(c->nv > 1 ? c->mv.grad[pi] : c->dg_grad[pi]);
  a.trace = (T *)(c->nv > 1 ? c->mv.trace[pi] : c->dg_trace[pi]);
  a.nv = c->nv;
  a.vs = L.ndofs;
  a.gs = L.ncells * 3 * (int64_t)L.n * L.n * L.n;
  a.ts = L.ncells * 12 * (int64_t)L.n * L.n;
  a.metric = (const T *)L.metric[pi];
  a.wcart = (const T *)L.wcart[pi];
  for (int d = 0; d < 3; ++d) {
    a.fdA[d] = (const T *)L.fdA[pi][d];
    a.fc[d] = (const T *)L.fc[pi][d];
    a.ih[d] = (T)(1.0 / L.h[d]);
    a.m[d] = L.m[d];
  }
  a.fwcart = (const T *)L.fwcart[pi];
  a.tau = (const T *)L.tau[pi];
  a.ufn = L.ufn;
  a.ncells = (int)L.ncells;
  for (int s = 0; s < 6; ++s) a.bc[s] = c->mesh.bc[s];
  // FP64 is bound by its arithmetic: store the gradient once; FP32 is bound
  // by traffic: recompute it instead of a 24 B/DoF round trip
  a.recompute = sizeof(T) == 4 ? 1 : 0;
  return a;
}

template <typename T>
FEArgs<T> fe_args(sipg_ctx *c, const Level &L) {
  constexpr int pi = pidx<T>();
  FEArgs<T> a{};
  a.ebuf = (T *)(c->nv > 1 ? c->mv.ebuf[pi] : c->ebuf[pi]);
  a.nv = c->nv;
  a.vs = L.ndofs;
  a.es = L.ncells * (int64_t)L.n * L.n * L.n;
  a.metric = (const T *)L.metric[pi];
  a.wcart = (const T *)L.wcart[pi];
  a.deg = L.deg;
  a.ncells = (int)L.ncells;
  for (int d = 0; d < 3; ++d) {
    a.m[d] = L.m[d];
    a.grid[d] = L.grid[d];
    a.alpha[d] = (T)(L.h[0] * L.h[1] * L.h[2] / (L.h[d] * L.h[d]));
  }
  for (int s = 0; s < 6; ++s) a.bc[s] = c->mesh.bc[s];
  return a;
}

// out = epilogue(A_l u): mode 0 Au, 1 c1 x + c2 xp + c3 dinv (b - Au), 2 b - Au
template <typename T>
void apply_level(sipg_ctx *c, int l, const T *u, T *out, int mode, const T *x = nullptr, const T *xp = nullptr,
                 const T *b = nullptr, const T *dinv = nullptr, T c1 = 0, T c2 = 0, T c3 = 0) {
  const Level &L = c->lv[l];
  if (L.kind == 0) {
    DGArgs<T> a = dg_args<T>(c, L);
    a.u = u;
    a.out = out;
    a.mode = mode;
    a.x = x;
    a.xp = xp;
    a.b = b;
    a.dinv = dinv;
    a.c1 = c1;
    a.c2 = c2;
    a.c3 = c3;
    CK(launch_dg_eval<T>(L.n, L.curved, a, c->stream, L.cb[pidx<T>()][0]));
    CK(launch_dg_integrate<T>(L.n, L.curved, a, c->stream, L.cb[pidx<T>()][1]));
  } else {
    FEArgs<T> a = fe_args<T>(c, L);
    a.u = u;
    a.out = out;
    a.mode = mode;
    a.x = x;
    a.xp = xp;
    a.b = b;
    a.dinv = dinv;
    a.c1 = c1;
    a.c2 = c2;
    a.c3 = c3;
    if (L.stencil[pidx<T>()]) {
      CK(launch_fe_stencil_apply<T>(a, (const T *)L.stencil[pidx<T>()], c->stream));
    } else {
      CK(launch_fe_cells<T>(L.n, L.curved, a, false, c->stream, L.cb[pidx<T>()][2]));
      CK(launch_fe_gather<T>(a, c->stream));
    }
  }
}

XferGeom xfer(sipg_ctx *c, int l) {
  const Level &F = c->lv[l], &C = c->lv[l - 1];
  XferGeom g{};
  g.kind = F.t_kind;
  for (int d = 0; d < 3; ++d) {
    g.mf[d] = F.m[d];
    g.mc[d] = C.m[d];
    g.gf[d] = F.grid[d];
    g.gc[d] = C.grid[d];
  }
  g.pf = F.deg;
  g.pc = C.deg;
  for (int s = 0; s < 6; ++s) g.bc[s] = c->mesh.bc[s];
  g.nv = c->nv;
  g.sf = F.ndofs;
  g.sc = C.ndofs;
  g.se = C.ncells * (int64_t)C.n * C.n * C.n;
  return g;
}

// rc = R r from level l to l-1.  With x0: where the restriction ends in a
// node pass, that pass also writes level l-1's first Chebyshev step from
// x = 0, x0 = c3 D^-1 rc (the xdb step, same arithmetic); returns whether it did.
template <typename T>
bool restrict_level(sipg_ctx *c, int l, const T *r, T *rc, T *x0 = nullptr, T c3 = 0) {
  constexpr int pi = pidx<T>();
  const Level &F = c->lv[l];
  if (F.t_kind >= 3) {   // DG -> DG: cell-local transpose
    CK(launch_dg_transfer<T>(xfer(c, l), (const T *)F.P1[pi], r, rc, false, c->stream));
    return false;
  }
  if (F.t_kind != 0 && fe_restrict_nodes_ok(xfer(c, l))) {   // small transfer: one node pass
    CK(launch_fe_restrict_nodes<T>(xfer(c, l), (const T *)F.P1[pi], r, rc, c->stream));
    return false;
  }
  FEArgs<T> a = fe_args<T>(c, c->lv[l - 1]);
  a.mode = 3;
  a.out = rc;
  if (x0) {
    a.mode = 5;
    a.out2 = x0;
    a.c3 = c3;
    a.dinv = (const T *)c->lv[l - 1].dinv[pi];
  }
  if (F.t_kind == 0) {
    a.ebuf = const_cast<T *>(r);   // the DG vector is the element buffer of the FE level
  } else {
    CK(launch_fe_restrict_cells<T>(xfer(c, l), (const T *)F.P1[pi], r,
                                   (T *)(c->nv > 1 ? c->mv.ebuf[pi] : c->ebuf[pi]), c->stream));
  }
  CK(launch_fe_gather<T>(a, c->stream));
  return x0 != nullptr;
}

// x += P xc from level l-1 to l
template <typename T>
void prolongate_level(sipg_ctx *c, int l, const T *xc, T *x) {
  constexpr int pi = pidx<T>();
  const Level &F = c->lv[l];
  if (F.t_kind >= 3) {
    CK(launch_dg_transfer<T>(xfer(c, l), (const T *)F.P1[pi], xc, x, true, c->stream));
  } else if (F.t_kind == 0) {
    FEArgs<T> a = fe_args<T>(c, c->lv[l - 1]);
    CK(launch_c_prolongate_add<T>(a, xc, x, c->stream, F.ndofs));
  } else {
    CK(launch_fe_prolongate_add<T>(xfer(c, l), (const T *)F.P1[pi], xc, x, c->stream));
  }
}

// The steps of Algorithm 3 on level l: step 0 is x = c3 D^-1 b from x = 0
// (xdb) or, from a given x, the first operator step with (c1, c2, c3) = (1,
// 0, 1/theta); every later step x_new = c1 x + c2 x_prev + c3 D^-1 (b - A x).
struct ChebStep {
  bool xdb, has_prev;
  double c1, c2, c3;
};
std::vector<ChebStep> cheb_plan(const sipg_ctx *c, int l, int ns, bool zero_start) {
  const double lam = c->lv[l].lambda;
  const double lhi = c->prm.cheb_hi * lam, llo = c->prm.cheb_lo * lam;
  const double theta = 0.5 * (lhi + llo), delta = 0.5 * (lhi - llo);
  std::vector<ChebStep> st;
  st.push_back({zero_start, false, 1.0, 0.0, 1.0 / theta});
  double rho_prev = delta / theta;
  for (int j = 1; j < ns; ++j) {
    const double rho = 1.0 / (2.0 * theta / delta - rho_prev);
    const double sigma = rho * rho_prev, th = 2.0 * rho / delta;
    // after x_0 = 0 the first operator step has no previous iterate
    st.push_back({false, !(zero_start && j == 1), 1.0 + sigma, -sigma, th});
    rho_prev = rho;
  }
  return st;
}

// Algorithm 3 on level l: x (in/out buffer pointer) with scratch xt; the
// buffers are swapped as the iteration proceeds.
// (x0_done: the producer of b already wrote the first step, x = c3 D^-1 b)
template <typename T>
void chebyshev(sipg_ctx *c, int l, const T *b, T *&x, T *&xt, int ns, bool zero_start, bool x0_done = false) {
  constexpr int pi = pidx<T>();
  const Level &L = c->lv[l];
  const T *dinv = (const T *)L.dinv[pi];
  for (const ChebStep &q : cheb_plan(c, l, ns, zero_start)) {
    if (q.xdb) {   // x_0 = 0
      if (!x0_done) CK(launch_xdb<T>(x, (T)q.c3, dinv, b, L.ndofs, c->stream, c->nv));
      continue;
    }
    apply_level<T>(c, l, x, xt, 1, x, q.has_prev ? xt : nullptr, b, dinv, (T)q.c1, (T)q.c2, (T)q.c3);
    std::swap(x, xt);
  }
}

template <typename T>
void learned_smooth(sipg_ctx *c, const T *b, T *x, int steps, bool zero_start);

// V-cycle vector k (0 vb, 1 vx, 2 vr, 3 vt) of level l in the current work set
template <typename T>
T *lvec(sipg_ctx *c, int l, int k) {
  if (c->nv > 1) return (T *)c->mv.v[4 * l + k];
  const Level &L = c->lv[l];
  void *const *v[4] = {L.vb, L.vx, L.vr, L.vt};
  return (T *)v[k][pidx<T>()];
}

// Inexact coarse solve on level 0 (FE_1 on the coarsest mesh) when it is too
// large for the dense inverse: coarse_iters Jacobi-preconditioned CG
// iterations from x = 0 (Algorithm 1 with D^-1 as the preconditioner; the
// paper solves its coarse level inexactly with AMG-CG, Section 3.2).  Every
// scalar stays in device memory (slots 16-18 of the context's scalar array)
// and the iteration count is fixed, so the V-cycle stays capturable.  The
// iteration runs in FP64 whatever the cycle's precision (like the dense
// inverse): an FP32 cycle casts its right-hand side into level 0's FP64
// vectors, which only the FP64 cycle uses otherwise, and casts the result
// back.  With several vectors (multi-vector cycles) each is solved in turn.
void coarse_cg_fp64(sipg_ctx *c, const double *b, double *x) {
  const Level &L0 = c->lv[0];
  const int64_t n = L0.ndofs;
  const double *dinv = (const double *)L0.dinv[0];
  double *p = c->cg_p, *q = c->cg_q;
  double *g[2] = {c->scal + 16, c->scal + 17}, *pq = c->scal + 18;
  double *r = lvec<double>(c, 0, 2), *z = lvec<double>(c, 0, 3);
  CK(cudaMemsetAsync(x, 0, n * sizeof(double), c->stream));
  CK(cudaMemcpyAsync(r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  CK(launch_xdb<double>(z, 1.0, dinv, r, n, c->stream));
  CK(launch_cg_dot<double>(r, z, n, c->partials, c->counter, g[0], c->stream));
  CK(cudaMemcpyAsync(p, z, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  for (int k = 0; k < c->prm.coarse_iters; ++k) {
    apply_level<double>(c, 0, p, q, 0);
    CK(launch_cg_dot<double>(p, q, n, c->partials, c->counter, pq, c->stream));
    CK(launch_cg_update_xr<double>(x, r, p, q, n, g[k & 1], pq, c->stream));
    CK(launch_xdb<double>(z, 1.0, dinv, r, n, c->stream));
    CK(launch_cg_dot<double>(r, z, n, c->partials, c->counter, g[(k + 1) & 1], c->stream));
    CK(launch_cg_update_p<double>(p, z, n, g[(k + 1) & 1], g[k & 1], c->stream));
  }
}

template <typename T>
void coarse_cg_solve(sipg_ctx *c, const T *b_all, T *x_all) {
  const int64_t n = c->lv[0].ndofs;
  const int nv = c->nv;
  c->nv = 1;   // one vector at a time (level-0 operator on single vectors)
  try {
    for (int v = 0; v < nv; ++v) {
      auto fp64 = [&](const double *b, double *x) {
        if (c->amg) CK(amg_solve(c->amg, b, x, c->stream));
        else coarse_cg_fp64(c, b, x);
      };
      if constexpr (std::is_same<T, double>::value) {
        fp64(b_all + v * n, x_all + v * n);
      } else {
        double *bd = lvec<double>(c, 0, 0), *xd = lvec<double>(c, 0, 1);
        CK((launch_cast<double, T>(bd, b_all + v * n, n, c->stream)));
        fp64(bd, xd);
        CK((launch_cast<T, double>(x_all + v * n, xd, n, c->stream)));
      }
    }
  } catch (...) {
    c->nv = nv;
    throw;
  }
  c->nv = nv;
}

// The steps vcycle_rec(l) launches on the levels of the fused tail, in
// launch order with the same buffers and coefficients, as a program of the
// tail kernel; returns the buffer that holds x^(l) after it.
template <typename T>
T *tail_rec(sipg_ctx *c, int l, std::vector<TailStep<T>> &prog) {
  constexpr int pi = pidx<T>();
  T *b = lvec<T>(c, l, 0);
  if (l == 0) {   // the dense coarse inverse
    TailStep<T> s{};
    s.op = kTailCoarse;
    s.n = c->n0;
    s.b = b;
    s.out = lvec<T>(c, 0, 1);
    s.Ainv = c->Ainv;
    prog.push_back(s);
    return lvec<T>(c, 0, 1);
  }
  const Level &L = c->lv[l];
  T *x = lvec<T>(c, l, 1), *xt = lvec<T>(c, l, 3);
  auto level_step = [&](int op) {
    TailStep<T> s{};
    s.op = op;
    s.n = (int)L.ndofs;
    for (int d = 0; d < 3; ++d) s.grid[d] = L.grid[d];
    for (int k = 0; k < 6; ++k) s.bc[k] = c->mesh.bc[k];
    s.dinv = (const T *)L.dinv[pi];
    s.coef = (const T *)L.stencil[pi];
    s.b = b;
    return s;
  };
  auto smooth = [&](bool zero_start) {   // chebyshev()
    for (const ChebStep &q : cheb_plan(c, l, c->prm.cheb_degree, zero_start)) {
      TailStep<T> s = level_step(q.xdb ? kTailXdb : kTailStencil);
      s.c3 = (T)q.c3;
      if (q.xdb) {
        s.out = x;
        prog.push_back(s);
        continue;
      }
      s.mode = 1;
      s.u = x;
      s.out = xt;
      s.x = x;
      s.xp = q.has_prev ? xt : nullptr;
      s.c1 = (T)q.c1;
      s.c2 = (T)q.c2;
      prog.push_back(s);
      std::swap(x, xt);
    }
  };
  smooth(true);
  TailStep<T> r = level_step(kTailStencil);   // the residual
  r.mode = 2;
  r.u = x;
  r.out = lvec<T>(c, l, 2);
  prog.push_back(r);
  const XferGeom g = xfer(c, l);
  TailStep<T> rs{};
  rs.op = kTailRestrict;
  rs.g = g;
  rs.n = g.gc[0] * g.gc[1] * g.gc[2];
  rs.P1 = (const T *)L.P1[pi];
  rs.u = lvec<T>(c, l, 2);
  rs.out = lvec<T>(c, l - 1, 0);
  prog.push_back(rs);
  const T *xc = tail_rec<T>(c, l - 1, prog);
  TailStep<T> pr{};
  pr.op = kTailProlong;
  pr.g = g;
  pr.n = g.gf[0] * g.gf[1] * g.gf[2];
  pr.P1 = (const T *)L.P1[pi];
  pr.u = xc;
  pr.out = x;
  prog.push_back(pr);
  smooth(false);
  return x;
}

// Which levels the fused tail takes: from level 1 up, every degree-1 FE level
// below the finest applied by its stencil with a 2:1 transfer from the level
// below and at most kTailMaxNodes nodes, over a dense coarse level; a program
// for every top level t, so that a cycle entered at any of them (the batched
// cycle enters below its two finest levels) runs fused.
template <typename T>
void build_tail(sipg_ctx *c) {
  constexpr int pi = pidx<T>();
  if (!c->prm.fuse_tail || c->coarse_cg || !c->Ainv || c->n0 > kTailMaxCoarse || c->n0 != c->lv[0].ndofs) return;
  int top = 0;
  while (top + 1 < c->L) {
    const Level &L = c->lv[top + 1];
    if (L.kind != 1 || L.deg != 1 || !L.stencil[pi] || L.t_kind != 2 || L.ndofs > kTailMaxNodes ||
        !fe_restrict_nodes_ok(xfer(c, top + 1)) || !L.dinv[pi])
      break;
    ++top;
  }
  std::vector<void *> progs(top + 1, nullptr), xs(top + 1, nullptr);
  std::vector<int> steps(top + 1, 0);
  int built = 0;
  for (int t = 1; t <= top; ++t) {
    std::vector<TailStep<T>> prog;
    xs[t] = tail_rec<T>(c, t, prog);
    if ((int)prog.size() > kTailMaxSteps) break;
    TailStep<T> *d = dalloc<TailStep<T>>(c, (int64_t)prog.size());
    CK(cudaMemcpy(d, prog.data(), prog.size() * sizeof(TailStep<T>), cudaMemcpyHostToDevice));
    progs[t] = d;
    steps[t] = (int)prog.size();
    built = t;
  }
  if (built == 0) return;
  const int cluster = fe_tail_cluster<T>(steps[built]);
  if (cluster == 0) return;
  c->tail_top = built;
  c->tail_cluster = cluster;
  c->tail_prog = progs;
  c->tail_x = xs;
  c->tail_steps = steps;
}

// Algorithm 2 with x^(l) = 0 on entry: rhs in lv[l].vb; returns the buffer
// (vx or vt of that level) that holds x^(l).  No state changes between calls,
// so the whole cycle can be captured once and replayed.
// level l runs inside the fused tail
template <typename T>
bool in_tail(const sipg_ctx *c, int l) {
  return l >= 1 && l <= c->tail_top && c->nv == 1 && pidx<T>() == c->prm.precision;
}

// (x0_done: the restriction or the cast that wrote this level's right-hand
// side also wrote its first Chebyshev step)
template <typename T>
T *vcycle_rec(sipg_ctx *c, int l, bool x0_done = false) {
  if (in_tail<T>(c, l)) {   // the fused tail
    CK(launch_fe_tail<T>((const TailStep<T> *)c->tail_prog[l], c->tail_steps[l], c->tail_cluster, c->stream));
    return (T *)c->tail_x[l];
  }
  T *b = lvec<T>(c, l, 0);
  if (l == 0) {
    if (c->coarse_cg) coarse_cg_solve<T>(c, b, lvec<T>(c, l, 1));
    else CK((launch_dense_gemv<T, T>(c->Ainv, b, lvec<T>(c, l, 1), c->n0, c->stream, c->nv)));
    return lvec<T>(c, l, 1);
  }
  T *x = lvec<T>(c, l, 1), *xt = lvec<T>(c, l, 3);
  const int ns = c->prm.cheb_degree;
  const bool learned = (l == c->L) && c->use_learned;
  if (learned && c->net.steps_pre > 0) learned_smooth<T>(c, b, x, c->net.steps_pre, true);
  else chebyshev<T>(c, l, b, x, xt, ns, true, x0_done);   // steps_pre = 0: Chebyshev pre-smoothing
  apply_level<T>(c, l, x, lvec<T>(c, l, 2), 2, nullptr, nullptr, b);
  // the level below starts its Chebyshev smoothing from x = 0 unless it is the
  // coarse level or runs in the fused tail: its first step can ride on the restriction
  const bool x0 = c->nv == 1 && l - 1 >= 1 && !in_tail<T>(c, l - 1);
  const bool done = restrict_level<T>(c, l, lvec<T>(c, l, 2), lvec<T>(c, l - 1, 0),
                                      x0 ? lvec<T>(c, l - 1, 1) : nullptr,
                                      x0 ? (T)cheb_plan(c, l - 1, ns, true)[0].c3 : T(0));
  const T *xc = vcycle_rec<T>(c, l - 1, done);
  prolongate_level<T>(c, l, xc, x);
  if (learned) learned_smooth<T>(c, b, x, c->net.steps_post, false);
  else chebyshev<T>(c, l, b, x, xt, ns, false);
  return x;
}

// z = M^-1 r with FP64 vectors in and out
// (one vector with Chebyshev pre-smoothing on the finest level: the copy or
// cast of r into the level's right-hand side also writes its first step)
void vcycle_body(sipg_ctx *c, const double *r, double *z) {
  const int64_t n = c->lv[c->L].ndofs * c->nv;
  const bool x0 = c->nv == 1 && !(c->use_learned && c->net.steps_pre > 0);
  const Level &F = c->lv[c->L];
  const double c3 = x0 ? cheb_plan(c, c->L, c->prm.cheb_degree, true)[0].c3 : 0.0;
  if (c->prm.precision == 0) {
    if (x0)
      CK((launch_cast_xdb<double, double>(lvec<double>(c, c->L, 0), lvec<double>(c, c->L, 1), c3,
                                          (const double *)F.dinv[0], r, n, c->stream)));
    else
      CK(cudaMemcpyAsync(lvec<double>(c, c->L, 0), r, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    const double *x = vcycle_rec<double>(c, c->L, x0);
    CK(cudaMemcpyAsync(z, x, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  } else {
    if (x0)
      CK((launch_cast_xdb<float, double>(lvec<float>(c, c->L, 0), lvec<float>(c, c->L, 1), (float)c3,
                                         (const float *)F.dinv[1], r, n, c->stream)));
    else
      CK((launch_cast<float, double>(lvec<float>(c, c->L, 0), r, n, c->stream)));
    const float *x = vcycle_rec<float>(c, c->L, x0);
    CK((launch_cast<double, float>(z, x, n, c->stream)));
  }
}

void vcycle_fp64io(sipg_ctx *c, const double *r, double *z) { vcycle_body(c, r, z); }

// The solver's preconditioner z = M^-1 r on its own vectors fr -> fz.  On a
// non-default stream the cycle is captured into a CUDA graph on its second
// use and replayed afterwards (one launch instead of ~100 per cycle).
void precondition(sipg_ctx *c) {
  const int pi = c->prm.precision;
  cudaGraphExec_t *gslot = c->use_learned ? &c->vgraph_l[pi] : &c->vgraph[pi];
  int *calls = c->use_learned ? &c->vcalls_l[pi] : &c->vcalls[pi];
  const double *r = c->fr;
  double *z = c->fz;
  if (c->nv > 1) {   // the multi-vector cycle on the multi-vector flexible-CG vectors
    if (c->mv.graph && c->mv.graph_nv != c->nv) {
      cudaGraphExecDestroy(c->mv.graph);
      c->mv.graph = nullptr;
      c->mv.calls = 0;
    }
    c->mv.graph_nv = c->nv;
    gslot = &c->mv.graph;
    calls = &c->mv.calls;
    r = c->mv.r;
    z = c->mv.z;
  }
  if (*gslot) {
    CK(cudaGraphLaunch(*gslot, c->stream));
    note_kernels(c->graph_kernels[*gslot]);
    return;
  }
  if (c->stream == nullptr || (*calls)++ < 1) {
    vcycle_body(c, r, z);
    return;
  }
  cudaGraph_t g = nullptr;
  long long kernels = 0;
  CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  try {
    CaptureTally tally(&kernels);
    vcycle_body(c, r, z);
  } catch (...) {
    cudaStreamEndCapture(c->stream, &g);
    if (g) cudaGraphDestroy(g);
    throw;
  }
  CK(cudaStreamEndCapture(c->stream, &g));
  cudaGraphExec_t ex = nullptr;
  const cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  CK(e);
  *gslot = ex;
  c->graph_kernels[ex] = kernels;
  CK(cudaGraphLaunch(ex, c->stream));
  note_kernels(kernels);
}

double read_scalar(sipg_ctx *c, int slot) {
  double v;
  CK(cudaMemcpyAsync(&v, c->scal + slot, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return v;
}

double dot(sipg_ctx *c, const double *x, const double *y, int64_t n, int slot) {
  CK(launch_dot2(x, y, nullptr, nullptr, n, c->partials, c->counter, c->scal + slot, c->stream));
  return read_scalar(c, slot);
}

// lambda_max of D^-1 A on level l from Jacobi-PCG (Section 3.1: 20 CG iterations)
double estimate_lambda(sipg_ctx *c, int l) {
  Level &L = c->lv[l];
  const int64_t n = L.ndofs;
  std::vector<double> r0(n);
  for (int64_t i = 0; i < n; ++i) r0[i] = uniform_pm1(1910, (uint64_t)i);
  double *r = (double *)L.vb[0], *z = (double *)L.vx[0], *p = (double *)L.vr[0], *Ap = (double *)L.vt[0];
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaMemcpy(r, r0.data(), n * sizeof(double), cudaMemcpyHostToDevice));
  if (L.kind == 1) {   // the start vector is zero on constrained FE nodes
    std::vector<double> h(n);
    for (int64_t g = 0; g < n; ++g) {
      const int gx = (int)(g % L.grid[0]), gy = (int)((g / L.grid[0]) % L.grid[1]),
                gz = (int)(g / ((int64_t)L.grid[0] * L.grid[1]));
      const int *bc = c->mesh.bc;
      const bool cons = (gx == 0 && bc[0] == 0) || (gx == L.grid[0] - 1 && bc[1] == 0) ||
                        (gy == 0 && bc[2] == 0) || (gy == L.grid[1] - 1 && bc[3] == 0) ||
                        (gz == 0 && bc[4] == 0) || (gz == L.grid[2] - 1 && bc[5] == 0);
      h[g] = cons ? 0.0 : r0[g];
    }
    CK(cudaMemcpy(r, h.data(), n * sizeof(double), cudaMemcpyHostToDevice));
  }
  const double *dinv = (const double *)L.dinv[0];
  CK(launch_xdb<double>(z, 1.0, dinv, r, n, c->stream));
  CK(cudaMemcpyAsync(p, z, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  double rz = dot(c, r, z, n, 8);
  const double rz0 = rz;
  std::vector<double> alphas, betas;
  for (int it = 0; it < c->prm.eig_iters; ++it) {
    apply_level<double>(c, l, p, Ap, 0);
    const double pAp = dot(c, p, Ap, n, 9);
    const double alpha = rz / pAp;
    CK(launch_axpy<double>(r, -alpha, Ap, n, c->stream));
    CK(launch_xdb<double>(z, 1.0, dinv, r, n, c->stream));
    const double rz_new = dot(c, r, z, n, 10);
    alphas.push_back(alpha);
    if (!(rz_new > 1e-28 * rz0)) break;
    const double beta = rz_new / rz;
    betas.push_back(beta);
    CK(launch_xpby<double>(p, z, beta, n, c->stream));
    rz = rz_new;
  }
  const int m = (int)alphas.size();
  std::vector<double> dg(m), off(m > 1 ? m - 1 : 0);
  for (int j = 0; j < m; ++j) {
    dg[j] = 1.0 / alphas[j] + (j > 0 ? betas[j - 1] / alphas[j - 1] : 0.0);
    if (j + 1 < m) off[j] = std::sqrt(betas[j]) / alphas[j];
  }
  return tridiag_max_eig(dg, off);
}

void build_level_geometry(sipg_ctx *c, Level &L, const MeshDesc &md, bool faces) {
  Mapping map(md);
  std::vector<double> metric, wcart;
  cell_geometry(map, L.n, metric, wcart);
  upload2(c, metric, L.metric);
  upload2(c, wcart, L.wcart);
  for (int d = 0; d < 3; ++d) L.h[d] = map.h[d];
  if (faces) {
    std::vector<double> fdA[3], fc[3], fw, tau;
    face_geometry(map, L.n, fdA, fc, fw);
    for (int d = 0; d < 3; ++d) {
      void *o[2];
      upload2(c, fdA[d], o);
      L.fdA[0][d] = o[0];
      L.fdA[1][d] = o[1];
      upload2(c, fc[d], o);
      L.fc[0][d] = o[0];
      L.fc[1][d] = o[1];
    }
    upload2(c, fw, L.fwcart);
    penalty(map, L.n, c->prm.penalty_factor, tau);
    upload2(c, tau, L.tau);
  }
}

void alloc_work(sipg_ctx *c, Level &L) {
  for (int pi = 0; pi < 2; ++pi) {
    const size_t es = pi == 0 ? 8 : 4;
    void **v[4] = {&L.vb[pi], &L.vx[pi], &L.vr[pi], &L.vt[pi]};
    for (auto *pp : v) {
      void *p;
      CK(cudaMalloc(&p, std::max<size_t>(L.ndofs, 1) * es));
      c->allocs.push_back(p);
      *pp = p;
    }
  }
}

// Tile-shape autotuner.  A cell kernel's block width cb (cells per block)
// fixes how many cells an SM holds at once (the occupancy calculator's
// resident blocks times cb) and hence how full the last wave of blocks is.
// The candidates are the widths whose waves leave the fewest cell slots
// idle (weighted by the share of live lanes in the block's last warp), plus
// the compiled default; each is timed on the level and the fastest kept.
// Results are cached per (n, geometry, precision, pass, cells) for the
// process, so contexts and batch members of equal shape tune once.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int64_t>, int> g_tune;

template <typename T>
std::vector<int> tile_candidates(const Level &L, int pass, int keep) {
  int dev = 0, nsm = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int maxcb = pass < 2 ? dg_max_cells_per_block<T>(L.n) : fe_max_cells_per_block<T>(L.n);
  std::vector<std::pair<double, int>> score;
  for (int cb = 1; cb <= maxcb; ++cb) {
    int occ = 0;
    CK(pass < 2 ? dg_blocks_per_sm<T>(L.n, L.curved, pass, cb, &occ) : fe_blocks_per_sm<T>(L.n, L.curved, cb, &occ));
    if (occ <= 0) continue;
    const int threads = cb * L.n * L.n;
    const double lanes = threads / (32.0 * ((threads + 31) / 32));
    const int64_t slots = (int64_t)occ * nsm, groups = (L.ncells + cb - 1) / cb;
    const int64_t waves = (groups + slots - 1) / slots;
    score.push_back({(double)L.ncells / ((double)waves * slots * cb) * lanes, cb});
  }
  std::stable_sort(score.begin(), score.end(), [](const auto &x, const auto &y) { return x.first > y.first; });
  std::vector<int> out{dg_cells_per_block<T>(L.n)};
  for (const auto &sc : score) {
    if ((int)out.size() > keep) break;
    if (std::find(out.begin(), out.end(), sc.second) == out.end()) out.push_back(sc.second);
  }
  return out;
}

template <typename T>
void autotune_level(sipg_ctx *c, int l, int pass) {
  constexpr int pi = pidx<T>();
  Level &L = c->lv[l];
  const auto key = std::make_tuple(L.n, (int)L.curved, pi, pass, L.ncells);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      L.cb[pi][pass] = it->second;
      return;
    }
  }
  const std::vector<int> cands = tile_candidates<T>(L, pass, 4);
  const int64_t len = pass < 2 ? L.ndofs : (int64_t)L.grid[0] * L.grid[1] * L.grid[2];
  T *u = dalloc<T>(c, len), *v = dalloc<T>(c, L.ncells * (int64_t)L.n * L.n * L.n);
  CK(cudaMemsetAsync(u, 0, len * sizeof(T), c->stream));
  DGArgs<T> a{};
  FEArgs<T> f{};
  if (pass < 2) {
    a = dg_args<T>(c, L);
    a.u = u;
    a.out = v;
    a.mode = 0;
  } else {
    f = fe_args<T>(c, L);
    f.u = u;
    f.ebuf = v;   // the cell pass writes ncells n^3 values: the DG length of this mesh
  }
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_cb = cands[0];
  for (int cb : cands) {
    auto run = [&]() {
      if (pass == 0) CK(launch_dg_eval<T>(L.n, L.curved, a, c->stream, cb));
      else if (pass == 1) CK(launch_dg_integrate<T>(L.n, L.curved, a, c->stream, cb));
      else CK(launch_fe_cells<T>(L.n, L.curved, f, false, c->stream, cb));
    };
    if (pass == 1) CK(launch_dg_eval<T>(L.n, L.curved, a, c->stream, 0));   // valid scratch for the integration
    run();
    CK(cudaEventRecord(e0, c->stream));
    const int reps = 5;
    for (int r = 0; r < reps; ++r) run();
    CK(cudaEventRecord(e1, c->stream));
    CK(cudaEventSynchronize(e1));
    float ms;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best) {
      best = ms;
      best_cb = cb;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  L.cb[pi][pass] = best_cb;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = best_cb;
}

// 1D tables into every translation unit's constant memory, shared-memory
// opt-ins of the cell kernels (once per process and device use)
void init_device_tables() {
  static Tables<double> td;
  static Tables<float> tf;
  static std::once_flag built;
  std::call_once(built, [] {
    build_tables(td);
    build_tables(tf);
  });
  upload_tables_dg<double>(td);
  upload_tables_dg<float>(tf);
  upload_tables_fe<double>(td);
  upload_tables_fe<float>(tf);
  upload_tables_batch<double>(td);
  upload_tables_batch<float>(tf);
  CK(cudaGetLastError());
  CK(prepare_dg_kernels<double>());
  CK(prepare_dg_kernels<float>());
  CK(prepare_fe_kernels());
}

// Default tile widths of every level: the compiled default, lowered on
// meshes that would give fewer blocks than SMs, so that every SM gets cells
// (GB300 runs two FP64 FMAs per clock per SM: an FP64 pass over 64 cells in 4
// blocks of 16 would use 4 of the 152 SMs).
void default_tile_widths(sipg_ctx *c) {
  int dev = 0, nsm = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  for (Level &L : c->lv)
    for (int pi = 0; pi < 2; ++pi)
      for (int pass = 0; pass < 3; ++pass) {
        int cb = dg_cells_per_block<double>(L.n);
        if (nsm > 0 && (L.ncells + cb - 1) / cb < nsm) cb = (int)std::max<int64_t>(1, (L.ncells + nsm - 1) / nsm);
        L.cb[pi][pass] = L.cb0[pi][pass] = cb;
      }
}

void setup(sipg_ctx *c) {
  const sipg_mesh &M = c->mesh;
  const sipg_params &P = c->prm;
  init_device_tables();
  MeshDesc md{};
  for (int d = 0; d < 3; ++d) {
    md.m[d] = M.m[d];
    md.lo[d] = M.lo[d];
    md.hi[d] = M.hi[d];
  }
  md.deform = M.deform;
  md.amp = M.amp;
  for (int s = 0; s < 6; ++s) md.bc[s] = M.bc[s];
  c->md = md;
  bool any_dir = false;
  for (int s = 0; s < 6; ++s) any_dir |= (M.bc[s] == 0);
  c->solver = !P.operator_only && any_dir;

  // fine-to-coarse list of (kind, degree, mesh)
  struct Spec {
    int kind, deg;
    MeshDesc md;
    int t_kind;   // transfer to the next coarser level
  };
  std::vector<Spec> specs;
  specs.push_back({0, P.degree, md, -1});
  if (c->solver) {
    // coarsening steps in the order of params.coarsening (Section 3.2): 'c' DG -> FE
    // at equal h and p, 'p' all polynomial levels down to 1, 'h' all geometric
    // levels (halve while every m is even and m/2 >= 3); the coarsest level is FE
    int kind = 0, p = P.degree;
    MeshDesc cm = md;
    for (const char *o = P.coarsening; *o; ++o) {
      if (*o == 'c') {
        if (kind == 1) throw_inval("coarsening: 'c' twice");
        specs.back().t_kind = 0;
        kind = 1;
        specs.push_back({1, p, cm, -1});
      } else if (*o == 'p') {
        while (p > 1) {   // floor(p/2) (default), p-1, or straight to 1
          specs.back().t_kind = kind ? 1 : 3;
          p = P.p_coarsen == 0 ? std::max(1, p / 2) : (P.p_coarsen == 1 ? p - 1 : 1);
          specs.push_back({kind, p, cm, -1});
        }
      } else if (*o == 'h') {
        while (cm.m[0] % 2 == 0 && cm.m[1] % 2 == 0 && cm.m[2] % 2 == 0 && cm.m[0] / 2 >= 3 &&
               cm.m[1] / 2 >= 3 && cm.m[2] / 2 >= 3) {
          for (int d = 0; d < 3; ++d) cm.m[d] /= 2;
          specs.back().t_kind = kind ? 2 : 4;
          specs.push_back({kind, p, cm, -1});
        }
      } else {
        throw_inval("coarsening letters are c, p and h");
      }
    }
    if (kind != 1) throw_inval("coarsening must contain 'c' (the coarse solve works on an FE level)");
    if (p != 1) throw_inval("coarsening must contain 'p' (the coarse matrix is assembled for degree 1)");
  }
  const int nl = (int)specs.size();
  c->lv.assign(nl, Level());
  c->L = nl - 1;
  int64_t ebuf_len = 0, dg_grad_len = 0, dg_trace_len = 0;
  for (int i = 0; i < nl; ++i) {
    const Spec &s = specs[i];
    Level &L = c->lv[nl - 1 - i];
    L.kind = s.kind;
    L.deg = s.deg;
    L.n = s.deg + 1;
    L.curved = md.deform != 0;
    for (int d = 0; d < 3; ++d) {
      L.m[d] = s.md.m[d];
      L.grid[d] = s.md.m[d] * s.deg + 1;
    }
    L.ncells = (int64_t)L.m[0] * L.m[1] * L.m[2];
    const int64_t n3 = (int64_t)L.n * L.n * L.n;
    L.ndofs = s.kind == 0 ? L.ncells * n3 : (int64_t)L.grid[0] * L.grid[1] * L.grid[2];
    build_level_geometry(c, L, s.md, s.kind == 0);
    if (s.kind == 1) ebuf_len = std::max(ebuf_len, L.ncells * n3);
    if (s.kind == 0) {
      dg_grad_len = std::max(dg_grad_len, L.ncells * 3 * n3);
      dg_trace_len = std::max(dg_trace_len, L.ncells * 12 * (int64_t)L.n * L.n);
    }
    if (c->solver) alloc_work(c, L);
  }
  // transfer tables: level l (fine) from l-1 (coarse)
  for (int l = 1; l < nl; ++l) {
    Level &F = c->lv[l];
    const Spec &s = specs[nl - 1 - l];
    F.t_kind = s.t_kind;
    if (F.t_kind == 0) continue;
    const Level &C = c->lv[l - 1];
    const int nf = F.n, nc = C.n;
    const Rules1D &rf = rules(nf), &rc = rules(nc);
    const bool hk = F.t_kind == 2 || F.t_kind == 4;
    const int nch = hk ? 2 : 1;
    std::vector<double> P1((size_t)nch * nf * nc);
    for (int ch = 0; ch < nch; ++ch)
      for (int i = 0; i < nf; ++i) {
        const double x = hk ? 0.5 * (ch + rf.gl[i]) : rf.gl[i];
        const auto v = lagrange_values(rc.gl, x);
        for (int j = 0; j < nc; ++j) P1[((size_t)ch * nf + i) * nc + j] = v[j];
      }
    upload2(c, P1, F.P1);
    ebuf_len = std::max(ebuf_len, C.ncells * (int64_t)nc * nc * nc);
  }
  // DG scratch (both precisions), shared by all DG levels (used one at a time)
  c->dg_grad[0] = dalloc<double>(c, dg_grad_len);
  c->dg_trace[0] = dalloc<double>(c, dg_trace_len);
  c->dg_grad[1] = dalloc<float>(c, dg_grad_len);
  c->dg_trace[1] = dalloc<float>(c, dg_trace_len);
  CK(cudaDeviceSynchronize());   // geometry uploads (legacy stream) complete before stream work
  default_tile_widths(c);
  if (P.autotune) {
    // the finest DG level always; the other cell-kernel levels of the solver
    for (int l = c->solver ? 1 : c->L; l <= c->L; ++l) {
      const int k = c->lv[l].kind;
      if (k == 1 && c->lv[l].deg <= P.fe_assemble) continue;   // assembled stencil: no cell pass to tune
      for (int pass = k == 0 ? 0 : 2; pass <= (k == 0 ? 1 : 2); ++pass) {
        autotune_level<double>(c, l, pass);
        autotune_level<float>(c, l, pass);
      }
    }
  }
  c->scal = dalloc<double>(c, 64);
  c->partials = dalloc<double>(c, 2 * 304);
  c->counter = dalloc<unsigned>(c, 4);
  CK(cudaMemset(c->counter, 0, 4 * sizeof(unsigned)));
  if (!c->solver) {
    CK(cudaDeviceSynchronize());
    return;
  }
  c->ebuf[0] = dalloc<double>(c, ebuf_len);
  c->ebuf[1] = dalloc<float>(c, ebuf_len);
  // a coarsest level above coarse_dense_max unknowns is solved by Jacobi-PCG
  if (P.coarse_dense_max < 0 || P.coarse_iters < 1 || P.coarse_iters > 10000)
    throw_inval("coarse_dense_max must be >= 0 and coarse_iters in 1..10000");
  c->coarse_cg = c->lv[0].ndofs > P.coarse_dense_max;
  const int lfirst = c->coarse_cg ? 0 : 1;   // levels that need an operator beyond the V-cycle's smoothing
  // assembled stencils of the low-degree FE levels that get applied
  if (P.fe_assemble < 0 || P.fe_assemble > 3) throw_inval("fe_assemble must be 0, 1, 2 or 3");
  for (int l = lfirst; l < nl; ++l) {
    Level &L = c->lv[l];
    if (L.kind != 1 || L.deg > P.fe_assemble) continue;
    const int w = 2 * L.deg + 1;
    const int64_t len = (int64_t)w * w * w * L.ndofs;
    double *cd = dalloc<double>(c, len);
    float *cf = dalloc<float>(c, len);
    CK(launch_fe_stencil_setup(L.curved, fe_args<double>(c, L), cd, c->stream));
    CK((launch_cast<float, double>(cf, cd, len, c->stream)));
    L.stencil[0] = cd;
    L.stencil[1] = cf;
  }
  // inverse diagonals (smoothed levels; the coarse level too for its Jacobi-PCG)
  for (int l = lfirst; l < nl; ++l) {
    Level &L = c->lv[l];
    double *d = dalloc<double>(c, L.ndofs);
    if (L.kind == 0) {
      DGArgs<double> a = dg_args<double>(c, L);
      CK(launch_dg_diag(L.n, L.curved, a, d, c->stream));
    } else {
      FEArgs<double> a = fe_args<double>(c, L);
      CK(launch_fe_cells<double>(L.n, L.curved, a, true, c->stream));
      a.mode = 4;
      a.out = d;
      CK(launch_fe_gather<double>(a, c->stream));
    }
    CK(launch_invert(d, L.ndofs, c->stream));
    float *f = dalloc<float>(c, L.ndofs);
    CK((launch_cast<float, double>(f, d, L.ndofs, c->stream)));
    L.dinv[0] = d;
    L.dinv[1] = f;
  }
  CK(cudaStreamSynchronize(c->stream));
  // smoothing range
  for (int l = 1; l < nl; ++l)
    c->lv[l].lambda = P.lambda_override > 0 ? P.lambda_override : estimate_lambda(c, l);
  // coarse matrix and its inverse, or the work vectors of the coarse Jacobi-PCG
  if (c->coarse_cg) {
    const int64_t n0 = c->lv[0].ndofs;
    c->n0 = (int)n0;
    if (P.coarse_solver == 0) {   // AMG-CG on the FE_1 matrix of the coarsest mesh
      Csr A;
      Mapping cmap(specs.back().md);
      coarse_matrix_csr(cmap, M.bc, A);
      std::string err;
      c->amg = amg_create(A, P.coarse_rtol, P.coarse_maxit, P.cheb_lo, P.cheb_hi, &err);
      if (!c->amg) {
        if (err.find("cudaMalloc") != std::string::npos) throw std::runtime_error("AMG setup: " + err);
        throw_inval("AMG setup: " + err);
      }
    } else {
      c->cg_p = dalloc<double>(c, n0);
      c->cg_q = dalloc<double>(c, n0);
    }
  } else {
    std::vector<double> A;
    int N;
    Mapping cmap(specs.back().md);
    coarse_matrix(cmap, M.bc, A, N);
    if (!cholesky_inverse(A, N)) throw_inval("coarse matrix is not positive definite");
    c->n0 = N;
    c->Ainv = dalloc<double>(c, (int64_t)N * N);
    CK(cudaMemcpy(c->Ainv, A.data(), A.size() * sizeof(double), cudaMemcpyHostToDevice));
  }
  if (P.precision == 0) build_tail<double>(c);
  else build_tail<float>(c);
  const int64_t N = c->lv[c->L].ndofs;
  c->fr = dalloc<double>(c, N);
  c->fz = dalloc<double>(c, N);
  c->fp = dalloc<double>(c, N);
  c->fv = dalloc<double>(c, N);
  c->fx = dalloc<double>(c, N);
  c->fb = dalloc<double>(c, N);
  CK(cudaDeviceSynchronize());
}

// Operator-only context on an unstructured hexahedral mesh: one DG level with
// per-cell geometry and face neighbours (unstructured.cpp).
void setup_unstructured(sipg_ctx *c, const UMeshIn &in) {
  const sipg_params &P = c->prm;
  init_device_tables();
  UGeometry g;
  std::string err;
  if (!build_unstructured(in, P.degree + 1, P.penalty_factor, g, err)) throw_inval(err);
  c->solver = false;
  c->lv.assign(1, Level());
  c->L = 0;
  Level &L = c->lv[0];
  L.kind = 0;
  L.deg = P.degree;
  L.n = P.degree + 1;
  L.curved = true;
  L.m[0] = in.ncells;
  L.ncells = in.ncells;
  const int64_t n3 = (int64_t)L.n * L.n * L.n;
  L.ndofs = L.ncells * n3;
  upload2(c, g.metric, L.metric);
  void *o[2];
  upload2(c, g.fdA, o);
  L.fdA[0][0] = o[0];
  L.fdA[1][0] = o[1];
  upload2(c, g.fc, o);
  L.fc[0][0] = o[0];
  L.fc[1][0] = o[1];
  upload2(c, g.tau, L.tau);
  L.ufn = (int2 *)dalloc<int>(c, (int64_t)g.ufn.size());
  CK(cudaMemcpy(L.ufn, g.ufn.data(), g.ufn.size() * sizeof(int), cudaMemcpyHostToDevice));
  c->dg_grad[0] = dalloc<double>(c, L.ncells * 3 * n3);
  c->dg_trace[0] = dalloc<double>(c, L.ncells * 12 * (int64_t)L.n * L.n);
  c->dg_grad[1] = dalloc<float>(c, L.ncells * 3 * n3);
  c->dg_trace[1] = dalloc<float>(c, L.ncells * 12 * (int64_t)L.n * L.n);
  CK(cudaDeviceSynchronize());
  default_tile_widths(c);
  if (P.autotune) {
    autotune_level<double>(c, 0, 0);
    autotune_level<double>(c, 0, 1);
    autotune_level<float>(c, 0, 0);
    autotune_level<float>(c, 0, 1);
  }
  c->scal = dalloc<double>(c, 64);
  c->partials = dalloc<double>(c, 2 * 304);
  c->counter = dalloc<unsigned>(c, 4);
  CK(cudaMemset(c->counter, 0, 4 * sizeof(unsigned)));
  CK(cudaDeviceSynchronize());
}

constexpr int kFcgChunk = 8;

// a conditional IF node on the capture of s, depending on what s captured so
// far; returns its body graph (to be filled by a capture on another stream)
cudaGraph_t add_if_node(cudaStream_t s, cudaGraphConditionalHandle h) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t *deps = nullptr;
  const cudaGraphEdgeData *ed = nullptr;
  size_t nd = 0;
  CK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, &ed, &nd));
  cudaGraphNodeParams prm{};
  prm.type = cudaGraphNodeTypeConditional;
  prm.conditional.handle = h;
  prm.conditional.type = cudaGraphCondTypeIf;
  prm.conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, g, deps, ed, nd, &prm));
  CK(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  return prm.conditional.phGraph_out[0];
}

// Capture kFcgChunk flexible-CG iterations on the context's vectors (x in
// fx, r in fr, p in fp, v = A p in fv, z in fz).  Iteration i: IF A_i {
// v = A p; p.Ap; x, r update; check (sets B_i) } then IF B_i { z = M^-1 r
// (the V-cycle); r.z, z.Ap; p = z + beta p; set A_{i+1} }.  Conditions
// default to 0 at every launch, so after the check that ends the solve
// nothing more runs.
void build_fcg_chunk(sipg_ctx *c) {
  const int pi = c->prm.precision;
  if (c->fcg_graph[pi]) return;
  if (!c->cap_stream) CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  const int64_t N = c->lv[c->L].ndofs;
  cudaStream_t s = c->stream, s2 = c->cap_stream;
  cudaGraph_t G = nullptr;
  CK(cudaGraphCreate(&G, 0));
  std::vector<cudaGraphConditionalHandle> hA(kFcgChunk), hB(kFcgChunk);
  for (int i = 0; i < kFcgChunk; ++i) {
    CK(cudaGraphConditionalHandleCreate(&hA[i], G, 0, cudaGraphCondAssignDefault));
    CK(cudaGraphConditionalHandleCreate(&hB[i], G, 0, cudaGraphCondAssignDefault));
  }
  c->fcg_kA.assign(kFcgChunk, 0);
  c->fcg_kB.assign(kFcgChunk, 0);
  long long k0 = 0;
  auto body = [&](cudaGraph_t b, long long *tally, auto &&fn) {
    c->stream = s2;
    CK(cudaStreamBeginCaptureToGraph(s2, b, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    try {
      CaptureTally t(tally);
      fn();
    } catch (...) {
      cudaGraph_t o;
      cudaStreamEndCapture(s2, &o);
      c->stream = s;
      throw;
    }
    cudaGraph_t o;
    CK(cudaStreamEndCapture(s2, &o));
    c->stream = s;
  };
  CK(cudaStreamBeginCaptureToGraph(s, G, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  try {
    {
      CaptureTally t(&k0);
      CK(launch_fcg_cond(c->fcg_state, hA[0], s));
    }
    for (int i = 0; i < kFcgChunk; ++i) {
      body(add_if_node(s, hA[i]), &c->fcg_kA[i], [&]() {
        apply_level<double>(c, c->L, c->fp, c->fv, 0);
        CK(launch_dot2(c->fp, c->fv, nullptr, nullptr, N, c->partials, c->counter, c->scal + 2, s2));
        CK(launch_fcg_update_xr(c->fx, c->fr, c->fp, c->fv, N, c->scal, c->partials, c->counter, c->scal + 3, s2));
        CK(launch_fcg_check(c->scal, c->fcg_hist, c->fcg_state, c->fcg_prm, hB[i], s2));
      });
      body(add_if_node(s, hB[i]), &c->fcg_kB[i], [&]() {
        vcycle_body(c, c->fr, c->fz);
        CK(launch_dot2(c->fr, c->fz, c->fz, c->fv, N, c->partials, c->counter, c->scal + 0, s2));
        CK(launch_fcg_update_p(c->fp, c->fz, c->scal, N, s2));
        if (i + 1 < kFcgChunk) CK(launch_fcg_cond(c->fcg_state, hA[i + 1], s2));
      });
    }
  } catch (...) {
    c->stream = s;
    cudaGraph_t o;
    cudaStreamEndCapture(s, &o);
    if (o) cudaGraphDestroy(o);
    cudaGraphDestroy(G);
    throw;
  }
  cudaGraph_t out = nullptr;
  CK(cudaStreamEndCapture(s, &out));
  cudaGraphExec_t ex = nullptr;
  const cudaError_t e = cudaGraphInstantiate(&ex, out, 0);
  cudaGraphDestroy(out);
  CK(e);
  c->fcg_graph[pi] = ex;
  c->graph_kernels[ex] = k0;   // per launch; the bodies are counted as they run
}

// Flexible CG (Algorithm 1 structure) preconditioned by one V-cycle.
sipg_status solve_impl(sipg_ctx *c, const double *b, double *x, double rtol, int maxit, int fixed,
                       sipg_solve_info *info) {
  const int64_t N = c->lv[c->L].ndofs;
  cudaStream_t s = c->stream;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, s));
  // ||b||^2 and ||x||^2 in one pass; r = b - A x, or r = b for a zero start
  // vector (no operator application)
  CK(launch_dot2(b, b, x, x, N, c->partials, c->counter, c->scal + 4, s));
  double bx[2];
  CK(cudaMemcpyAsync(bx, c->scal + 4, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (bx[1] == 0.0)
    CK(cudaMemcpyAsync(c->fr, b, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  else
    apply_level<double>(c, c->L, x, c->fr, 2, nullptr, nullptr, b);
  const double bn = std::sqrt(bx[0]);
  if (!std::isfinite(bn)) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->err = "right-hand side is not finite";
    return SIPG_ENAN;
  }
  const double r0 = std::sqrt(dot(c, c->fr, c->fr, N, 3));
  std::vector<double> hist{r0};
  c->use_learned = (c->smoother >= 1 && c->net.trained) ? 1 : 0;
  const int learned_at_start = c->use_learned;
  precondition(c);
  CK(launch_dot2(c->fr, c->fz, nullptr, nullptr, N, c->partials, c->counter, c->scal + 0, s));
  CK(cudaMemcpyAsync(c->fp, c->fz, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
  int it = 0;
  sipg_status st = SIPG_OK;
  double rn = r0;
  const bool fixed_mode = fixed > 0;
  int fell_back = 0;
  // (a solve that ends before its first iteration stays on the host path)
  const bool on_device = !c->use_learned && c->nv == 1 && s != nullptr && r0 > 0.0 &&
                         (fixed_mode || (rtol < 1.0 && maxit > 0));
  if (on_device) {
    // iterations gated on the device, kFcgChunk per graph launch and host read
    if (!c->fcg_state) {
      c->fcg_state = dalloc<int>(c, 4);
      c->fcg_hist = dalloc<double>(c, 260);
      c->fcg_prm = dalloc<double>(c, 2);
    }
    struct {
      double rtol;
      int maxit, fixed;
    } prm{rtol, maxit, fixed};
    const int st0[4] = {0, 0, 0, 0};
    CK(cudaMemcpyAsync(c->fcg_prm, &prm, sizeof(prm), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->fcg_state, st0, sizeof(st0), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->scal + 20, &r0, sizeof(double), cudaMemcpyHostToDevice, s));
    if (x != c->fx) CK(cudaMemcpyAsync(c->fx, x, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    build_fcg_chunk(c);
    int hs[4] = {0, 0, 0, 0};
    // every chunk that does not end the solve advances it by kFcgChunk
    // iterations, and the device ends it at maxit: the bound below is never
    // reached unless the device state stopped moving
    const int max_launches = (fixed_mode ? fixed : maxit) / kFcgChunk + 2;
    for (int launches = 0;; ++launches) {
      if (launches >= max_launches) {
        c->err = "flexible CG on the device made no progress";
        throw Fail{SIPG_ECUDA};
      }
      CK(cudaGraphLaunch(c->fcg_graph[c->prm.precision], s));
      note_kernels(c->graph_kernels[c->fcg_graph[c->prm.precision]]);
      CK(cudaMemcpyAsync(hs, c->fcg_state, sizeof(hs), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (hs[1]) break;
    }
    if (x != c->fx) CK(cudaMemcpyAsync(x, c->fx, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    it = hs[0];
    // kernels of the bodies that ran: the first step of iterations 1..it,
    // the preconditioning step of all but the last
    for (int j = 0; j < it; ++j) note_kernels(c->fcg_kA[j % kFcgChunk] + (j + 1 < it ? c->fcg_kB[j % kFcgChunk] : 0));
    // a breakdown is counted as an iteration without a recorded residual
    const int done_it = hs[2] == 1 ? it - 1 : it;
    std::vector<double> h(std::min(done_it, 256) + 1);
    CK(cudaMemcpyAsync(h.data(), c->fcg_hist, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    double rr_last = 0;
    CK(cudaMemcpyAsync(&rr_last, c->scal + 3, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int j = 1; j < (int)h.size(); ++j) hist.push_back(h[j]);
    if (hs[2] == 1) {
      c->err = "flexible CG breakdown: p^T A p <= 0 or a non-finite scalar";
      st = SIPG_EBREAKDOWN;
      rn = hist.back();
    } else {
      rn = std::sqrt(rr_last);   // (the history stops at 256 iterations)
      if (hs[2] == 2) st = SIPG_ENOTCONV;
    }
  }
  // otherwise (the learned cycle, whose fallback the host decides per
  // iteration; the legacy default stream, which cannot be captured): one host
  // read per iteration
  while (!on_device) {
    if (fixed_mode) {
      if (it >= fixed) break;
    } else if (rn <= rtol * r0 || r0 == 0.0) {
      break;
    } else if (it >= maxit) {
      st = SIPG_ENOTCONV;
      break;
    }
    apply_level<double>(c, c->L, c->fp, c->fv, 0);
    CK(launch_dot2(c->fp, c->fv, nullptr, nullptr, N, c->partials, c->counter, c->scal + 2, s));
    CK(launch_fcg_update_xr(x, c->fr, c->fp, c->fv, N, c->scal, c->partials, c->counter, c->scal + 3, s));
    double sc[4];
    CK(cudaMemcpyAsync(sc, c->scal, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (!(sc[2] > 0) || !std::isfinite(sc[0]) || !std::isfinite(sc[3])) {
      c->err = "flexible CG breakdown: p^T A p <= 0 or a non-finite scalar";
      st = SIPG_EBREAKDOWN;
      ++it;
      break;
    }
    const double rprev = rn;
    rn = std::sqrt(sc[3]);
    ++it;
    hist.push_back(rn);
    if (!fixed_mode && rn <= rtol * r0) break;
    // the Chebyshev cycle judges the learned one: a step that reduces the
    // residual less than the Chebyshev cycle's average rate switches the rest
    // of the solve back to Chebyshev (flexible CG keeps the iteration valid)
    // (rate per unit time: a cheaper learned iteration may reduce less per step)
    const double tr = (c->net.t_iter_cheb > 0 && c->net.t_iter_learned > 0)
                          ? c->net.t_iter_learned / c->net.t_iter_cheb
                          : 1.0;
    if (c->use_learned && c->smoother == 1 && rn > std::pow(c->net.rho_cheb, tr) * rprev) {
      c->use_learned = 0;
      fell_back = 1;
    }
    precondition(c);
    CK(launch_dot2(c->fr, c->fz, c->fz, c->fv, N, c->partials, c->counter, c->scal + 0, s));   // gamma, z.Ap
    CK(launch_fcg_update_p(c->fp, c->fz, c->scal, N, s));
  }
  CK(cudaEventRecord(e1, s));
  CK(cudaEventSynchronize(e1));
  if (learned_at_start) {   // a tensor-core GEMM of the learned cycle that timed out wrote nothing
    int timed_out = 0;
    CK(mlp_tc_status(&timed_out));
    if (timed_out) {
      c->err = "a tensor-core GEMM of the learned smoother timed out waiting for its MMAs";
      st = SIPG_ETIMEOUT;
    }
  }
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->iterations = it;
    info->r0_norm = r0;
    info->r_norm = rn;
    info->converged = (r0 == 0.0 || rn <= rtol * r0) ? 1 : 0;
    info->rho = (it > 0 && r0 > 0) ? std::pow(rn / r0, 1.0 / it) : 0.0;
    info->n10 = (info->rho > 0 && info->rho < 1) ? -10.0 / std::log10(info->rho) : 0.0;
    info->seconds = ms * 1e-3;
    for (int j = 0; j < (int)hist.size() && j < 256; ++j) info->res_history[j] = hist[j];
    info->learned = learned_at_start;
    info->fell_back = fell_back;
  }
  c->use_learned = 0;
  if (st == SIPG_ENOTCONV) c->err = "flexible CG reached maxit before the tolerance";
  return st;
}


// ------------------------------------------------------------ learned smoother
// A per-cell network (input: the cell's residual and the neighbours' face
// residuals, scaled by their RMS; output: the cell's correction) that stands in
// for the Chebyshev smoother on the finest level.  Not in the paper.

// the transposed BF16 weights follow every change of the BF16 weights
inline const void *bf(const void *base, long off) { return (const uint16_t *)base + off; }
inline void *bfm(void *base, long off) { return (uint16_t *)base + off; }

void net_weights_updated(sipg_ctx *c) {
  auto &N = c->net;
  CK(mlp_transpose_weights(N.Pb, N.oW1, N.oW2, N.oW3, N.Fp, N.H, N.No, N.Pt, c->stream));
  if (N.Wc) {   // the fused forward's operand blocks (core-matrix layout, K chunks of 32)
    CK(mlp_pack_core(bf(N.Pt, N.oT1), N.Fp, N.H, N.Fp, N.H, bfm(N.Wc, N.oC1), c->stream));
    CK(mlp_pack_core(bf(N.Pt, N.oT2), N.H, N.H, N.H, N.H, bfm(N.Wc, N.oC2), c->stream));
    CK(mlp_pack_core(bf(N.Pt, N.oT3), N.H, N.No, N.H, N.No, bfm(N.Wc, N.oC3), c->stream));
  }
}

void net_setup(sipg_ctx *c, long rows) {
  auto &N = c->net;
  const Level &F = c->lv[c->L];
  if (!N.ready) {
    N.n3 = F.n * F.n * F.n;
    N.F = N.n3 + 6 * F.n * F.n;
    N.Fp = (N.F + 15) / 16 * 16;
    N.No = (N.n3 + 15) / 16 * 16;
    N.oW1 = 0;
    N.ob1 = N.oW1 + (long)N.Fp * N.H;
    N.oW2 = N.ob1 + N.H;
    N.ob2 = N.oW2 + (long)N.H * N.H;
    N.oW3 = N.ob2 + N.H;
    N.ob3 = N.oW3 + (long)N.H * N.No;
    N.np = N.ob3 + N.No;
    N.P = dalloc<float>(c, N.np);
    N.M = dalloc<float>(c, N.np);
    N.V = dalloc<float>(c, N.np);
    N.G = dalloc<float>(c, N.np);
    N.Pb = dalloc<uint16_t>(c, N.np);
    N.oT1 = 0;
    N.oT2 = (long)N.H * N.Fp;
    N.oT3 = N.oT2 + (long)N.H * N.H;
    N.Pt = dalloc<uint16_t>(c, N.oT3 + (long)N.No * N.H);
    if (N.H == 256 && N.No <= 256) {
      N.Fc = (N.Fp + 31) / 32 * 32;
      N.oC1 = 0;
      N.oC2 = (long)N.H * N.Fc;
      N.oC3 = N.oC2 + (long)N.H * N.H;
      N.Wc = dalloc<uint16_t>(c, N.oC3 + (long)N.No * N.H);
    }
    N.loss = dalloc<double>(c, 2);
    // He-uniform initial weights from the counter-based generator, zero biases
    std::vector<float> h(N.np, 0.f);
    auto fill = [&](long off, int fin, int fanin_valid, int fout, uint64_t seed) {
      const double lim = std::sqrt(6.0 / fanin_valid);
      for (int i = 0; i < fin; ++i)
        for (int j = 0; j < fout; ++j)
          h[off + (long)i * fout + j] = i < fanin_valid ? (float)(lim * uniform_pm1(seed, (uint64_t)i * fout + j)) : 0.f;
    };
    fill(N.oW1, N.Fp, N.F, N.H, 4001);
    fill(N.oW2, N.H, N.H, N.H, 4002);
    fill(N.oW3, N.H, N.H, N.No, 4003);
    CK(cudaMemcpyAsync(N.P, h.data(), N.np * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    CK(mlp_f2bf(N.P, N.Pb, N.np, c->stream));
    net_weights_updated(c);
    CK(cudaStreamSynchronize(c->stream));
    N.ready = true;
  }
  if (rows > N.rows) {
    N.X = dalloc<uint16_t>(c, rows * N.Fp);
    if (N.Wc) N.Xc = dalloc<uint16_t>(c, (rows + 127) / 128 * 128 * (long)N.Fc);
    N.H1 = dalloc<uint16_t>(c, rows * N.H);
    N.H2 = dalloc<uint16_t>(c, rows * N.H);
    N.dH = dalloc<uint16_t>(c, rows * N.H);
    N.dY = dalloc<uint16_t>(c, rows * N.No);
    N.Y = dalloc<float>(c, rows * N.No);
    N.dYf = dalloc<float>(c, rows * N.No);
    N.scale = dalloc<float>(c, rows);
    const long rp = (rows + 15) / 16 * 16;
    N.TA = dalloc<uint16_t>(c, rp * std::max(N.Fp, N.H));
    N.TB = dalloc<uint16_t>(c, rp * std::max(N.H, N.No));
    N.rows = rows;
  }
}


// Y = net(X) for B rows of X (bf16, row stride ldx elements); the hidden
// activations land in N.H1 and N.H2 when keep_hidden (the backward pass reads them)
void net_forward(sipg_ctx *c, const void *X, long ldx, int B, bool keep_hidden = true) {
  auto &N = c->net;
  cudaStream_t s = c->stream;
  if (N.Wc) {   // the whole network in one tensor-core kernel, operands packed for bulk copies
    CK(mlp_pack_core(X, ldx, B, N.Fp, 128, N.Xc, s));
    CK(mlp_forward_fused(N.Xc, B, N.Fp, N.No, N.Wc, N.oC1, N.oC2, N.oC3, N.P + N.ob1, N.P + N.ob2, N.P + N.ob3, N.Y,
                         N.No, keep_hidden ? N.H1 : nullptr, keep_hidden ? N.H2 : nullptr, s));
    return;
  }
  // one layer: out = act(in W + b) with W [K][Nout]; on the tcgen05 tensor
  // cores (transposed weights) when the output width fits one MMA tile
  auto layer = [&](const void *in, long ld, long oW, long oT, int K, int Nout, const float *bias, int relu,
                   float *Cf, void *Cb) {
    if (Nout % 16 == 0 && Nout <= 256)
      CK(mlp_gemm_tc(in, ld, bf(N.Pt, oT), K, B, Nout, K, bias, relu, Cf, Cb, Nout, s));
    else
      CK(mlp_gemm(in, ld, 1, bf(N.Pb, oW), Nout, 1, B, Nout, K, bias, relu, Cf, Cb, Nout, 0, s));
  };
  layer(X, ldx, N.oW1, N.oT1, N.Fp, N.H, N.P + N.ob1, 1, nullptr, N.H1);
  layer(N.H1, N.H, N.oW2, N.oT2, N.H, N.H, N.P + N.ob2, 1, nullptr, N.H2);
  layer(N.H2, N.H, N.oW3, N.oT3, N.H, N.No, N.P + N.ob3, 0, N.Y, nullptr);
}

// gradients of the mean squared error over B rows (X row stride ldx, T row stride ldt) into N.G
void net_backward(sipg_ctx *c, const void *X, long ldx, int B);

void net_gradients(sipg_ctx *c, const void *X, long ldx, const float *T, long ldt, int B) {
  auto &N = c->net;
  net_forward(c, X, ldx, B);
  CK(mlp_mse_grad(N.Y, T, ldt, B, N.n3, N.No, N.dY, N.dYf, N.loss, c->stream));
  net_backward(c, X, ldx, B);
}

// gradients into N.G from the output errors in N.dY (BF16) and N.dYf (FP32)
// of the last forward pass over B rows of X
void net_backward(sipg_ctx *c, const void *X, long ldx, int B) {
  auto &N = c->net;
  cudaStream_t s = c->stream;
  if (N.No <= 256) {
    // every product on the tcgen05 tensor cores: the back-propagated errors
    // dY W3^T and dH W2^T read the stored weights as K-contiguous operands;
    // the weight gradients contract over the batch rows, so both of their
    // operands are transposed (zero-padded to a multiple of 16 rows) first
    const int Bp = (B + 15) / 16 * 16;
    CK(mlp_transpose_bf16(N.H2, B, N.H, N.H, N.TA, Bp, s));
    CK(mlp_transpose_bf16(N.dY, B, N.No, N.No, N.TB, Bp, s));
    CK(mlp_gemm_tc(N.TA, Bp, N.TB, Bp, N.H, N.No, Bp, nullptr, 0, N.G + N.oW3, nullptr, N.No, s));
    CK(mlp_colsum(N.dYf, 0, B, N.No, N.No, N.G + N.ob3, s));
    CK(mlp_gemm_tc(N.dY, N.No, bf(N.Pb, N.oW3), N.No, B, N.H, N.No, nullptr, 0, nullptr, N.dH, N.H, s));
    CK(mlp_relu_mask(N.dH, N.H2, (long)B * N.H, s));
    CK(mlp_transpose_bf16(N.H1, B, N.H, N.H, N.TA, Bp, s));
    CK(mlp_transpose_bf16(N.dH, B, N.H, N.H, N.TB, Bp, s));
    CK(mlp_gemm_tc(N.TA, Bp, N.TB, Bp, N.H, N.H, Bp, nullptr, 0, N.G + N.oW2, nullptr, N.H, s));
    CK(mlp_colsum(N.dH, 1, B, N.H, N.H, N.G + N.ob2, s));
    CK(mlp_gemm_tc(N.dH, N.H, bf(N.Pb, N.oW2), N.H, B, N.H, N.H, nullptr, 0, nullptr, N.H2, N.H, s));
    CK(mlp_relu_mask(N.H2, N.H1, (long)B * N.H, s));
    CK(mlp_transpose_bf16(X, B, N.Fp, ldx, N.TA, Bp, s));
    CK(mlp_transpose_bf16(N.H2, B, N.H, N.H, N.TB, Bp, s));
    CK(mlp_gemm_tc(N.TA, Bp, N.TB, Bp, N.Fp, N.H, Bp, nullptr, 0, N.G + N.oW1, nullptr, N.H, s));
    CK(mlp_colsum(N.H2, 1, B, N.H, N.H, N.G + N.ob1, s));
    return;
  }
  // outputs wider than one tensor-core tile (degree >= 6): mma.sync products
  CK(mlp_gemm(N.H2, 1, N.H, N.dY, N.No, 1, N.H, N.No, B, nullptr, 0, N.G + N.oW3, nullptr, N.No, 0, s));
  CK(mlp_colsum(N.dYf, 0, B, N.No, N.No, N.G + N.ob3, s));
  CK(mlp_gemm(N.dY, N.No, 1, bf(N.Pb, N.oW3), 1, N.No, B, N.H, N.No, nullptr, 0, nullptr, N.dH, N.H, 0, s));
  CK(mlp_relu_mask(N.dH, N.H2, (long)B * N.H, s));
  CK(mlp_gemm(N.H1, 1, N.H, N.dH, N.H, 1, N.H, N.H, B, nullptr, 0, N.G + N.oW2, nullptr, N.H, 0, s));
  CK(mlp_colsum(N.dH, 1, B, N.H, N.H, N.G + N.ob2, s));
  CK(mlp_gemm(N.dH, N.H, 1, bf(N.Pb, N.oW2), 1, N.H, B, N.H, N.H, nullptr, 0, nullptr, N.H2, N.H, 0, s));
  CK(mlp_relu_mask(N.H2, N.H1, (long)B * N.H, s));
  CK(mlp_gemm(X, 1, ldx, N.H2, N.H, 1, N.Fp, N.H, B, nullptr, 0, N.G + N.oW1, nullptr, N.H, 0, s));
  CK(mlp_colsum(N.H2, 1, B, N.H, N.H, N.G + N.ob1, s));
}

// steps of x <- x + c s net(features(b - A x)) on the finest level
template <typename T>
void learned_smooth(sipg_ctx *c, const T *b, T *x, int steps, bool zero_start) {
  constexpr int pi = pidx<T>();
  auto &N = c->net;
  const Level &F = c->lv[c->L];
  const int E = (int)F.ncells;
  for (int st = 0; st < steps; ++st) {
    const T *r;
    if (zero_start && st == 0) {
      CK(cudaMemsetAsync(x, 0, F.ndofs * sizeof(T), c->stream));
      r = b;
    } else {
      apply_level<T>(c, c->L, x, (T *)F.vr[pi], 2, nullptr, nullptr, b);
      r = (const T *)F.vr[pi];
    }
    CK(mlp_gather<T>(r, F.n, F.m, nullptr, 0, E, N.X, N.Fp, N.scale, c->stream));
    net_forward(c, N.X, N.Fp, E, false);
    CK(mlp_correct<T>(x, N.n3, 0, E, N.Y, N.No, N.scale, N.cscale, c->stream));
  }
}
template void learned_smooth<double>(sipg_ctx *, const double *, double *, int, bool);
template void learned_smooth<float>(sipg_ctx *, const float *, float *, int, bool);

// Time of one flexible-CG iteration's work with the Chebyshev (learned = 0)
// or the learned cycle: a V-cycle on fr plus one outer operator application
// (mean of 3 after one warm-up, CUDA events on the context stream).
double iteration_ms(sipg_ctx *c, int learned) {
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const int save = c->use_learned;
  c->use_learned = learned;
  vcycle_body(c, c->fr, c->fz);
  apply_level<double>(c, c->L, c->fz, c->fv, 0);
  CK(cudaEventRecord(e0, c->stream));
  for (int r = 0; r < 3; ++r) {
    vcycle_body(c, c->fr, c->fz);
    apply_level<double>(c, c->L, c->fz, c->fv, 0);
  }
  CK(cudaEventRecord(e1, c->stream));
  CK(cudaEventSynchronize(e1));
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  c->use_learned = save;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms / 3.0;
}

sipg_status train_impl(sipg_ctx *c, int npairs, int epochs, uint64_t seed, sipg_train_info *info) {
  auto t0 = std::chrono::steady_clock::now();
  const Level &F = c->lv[c->L];
  const int E = (int)F.ncells;
  const int64_t Nd = F.ndofs;
  const int B = 256;
  const int NB = std::max(1, (npairs + B - 1) / B);
  const long R = (long)NB * B;
  net_setup(c, std::max<long>(E, B));
  auto &N = c->net;
  const int S = 4, J = 4;   // right-hand sides, iterates per right-hand side
  void *Xall = dalloc<uint16_t>(c, R * N.Fp);
  float *Tall = dalloc<float>(c, R * N.No);
  float *sall = dalloc<float>(c, R);
  int *cells = dalloc<int>(c, R);
  double *b = dalloc<double>(c, Nd), *xs = dalloc<double>(c, Nd), *xj = dalloc<double>(c, Nd),
         *r = dalloc<double>(c, Nd), *e = dalloc<double>(c, Nd);
  std::vector<int> hc(R);
  for (long i = 0; i < R; ++i) hc[i] = (int)(splitmix64(seed ^ (0x5151ull + (uint64_t)i)) % (uint64_t)E);
  // every copy below is ordered on the context stream (which may be a
  // non-blocking stream that the legacy default stream does not wait for)
  CK(cudaMemcpyAsync(cells, hc.data(), R * sizeof(int), cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  std::vector<double> hb(Nd);
  double rho_sum = 0;
  int rho_cnt = 0;
  const int save_smoother = c->smoother;
  c->smoother = 0;
  double *bv = dalloc<double>(c, Nd), *xv = dalloc<double>(c, Nd), *xx = dalloc<double>(c, Nd),
         *xt2 = dalloc<double>(c, Nd);
  if (N.nsnap != S * J) {
    N.snap_r = dalloc<double>(c, (int64_t)S * J * Nd);
    N.snap_e = dalloc<double>(c, (int64_t)S * J * Nd);
    N.nsnap = S * J;
  }
  long row = 0;
  auto add_pairs = [&](const double *res, const double *err, long cnt) {
    CK(mlp_gather<double>(res, F.n, F.m, cells, (int)row, (int)cnt, bfm(Xall, row * N.Fp), N.Fp, sall + row,
                          c->stream));
    CK(mlp_targets(err, N.n3, cells, (int)row, (int)cnt, sall + row, Tall + row * N.No, N.No, c->stream));
    row += cnt;
  };
  // Snapshots of the plain cycle at work: for FCG iterate j of a seeded random
  // right-hand side, the cycle's input b_v = r_j; its exact correction
  // x*_v = A^-1 b_v (solved to 1e-12); pairs at random cells taken after
  // pre-smoothing and the coarse-grid correction (the state the post-smoother
  // starts from): residual b_v - A x, error x*_v - x -- the high-frequency
  // error a smoother has to remove.  (The full error x*_v of the cycle's input
  // is dominated by smooth components no cell-local map can predict; pairs of
  // that kind taught the network corrections far too large.)
  for (int sidx = 0; sidx < S; ++sidx) {
    for (int64_t i = 0; i < Nd; ++i) hb[i] = uniform_pm1(seed + 1 + sidx, (uint64_t)i);
    CK(cudaStreamSynchronize(c->stream));   // the previous right-hand side is no longer read
    CK(cudaMemcpyAsync(b, hb.data(), Nd * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    for (int j = 0; j < J; ++j) {
      CK(cudaMemsetAsync(xj, 0, Nd * sizeof(double), c->stream));
      if (j > 0) solve_impl(c, b, xj, 0.0, j, j, nullptr);
      apply_level<double>(c, c->L, xj, bv, 2, nullptr, nullptr, b);           // b_v = r_j
      CK(cudaMemsetAsync(xv, 0, Nd * sizeof(double), c->stream));
      sipg_solve_info inf{};
      const sipg_status st = solve_impl(c, bv, xv, 1e-12, 500, 0, &inf);     // x*_v
      if (st != SIPG_OK) {
        c->smoother = save_smoother;
        return st;
      }
      rho_sum += inf.rho;
      ++rho_cnt;
      const long snaps = (long)S * J, cnt = (sidx * J + j == snaps - 1) ? R - row : R / snaps;
      // the cycle up to the post-smoother, in FP64
      double *x = xx, *xt = xt2;
      chebyshev<double>(c, c->L, bv, x, xt, c->prm.cheb_degree, true);
      apply_level<double>(c, c->L, x, r, 2, nullptr, nullptr, bv);
      restrict_level<double>(c, c->L, r, (double *)c->lv[c->L - 1].vb[0]);
      const double *xc = vcycle_rec<double>(c, c->L - 1);
      prolongate_level<double>(c, c->L, xc, x);
      apply_level<double>(c, c->L, x, r, 2, nullptr, nullptr, bv);
      CK(cudaMemcpyAsync(e, xv, Nd * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
      CK(launch_axpy<double>(e, -1.0, x, Nd, c->stream));
      add_pairs(r, e, cnt);
      const int64_t so = (int64_t)(sidx * J + j) * Nd;
      CK(cudaMemcpyAsync(N.snap_r + so, r, Nd * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
      CK(cudaMemcpyAsync(N.snap_e + so, e, Nd * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
      if (sidx == S - 1 && j == J - 1)   // kept for the damping below
        CK(cudaMemcpyAsync(bv, r, Nd * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    }
  }
  c->smoother = save_smoother;
  N.rho_cheb = rho_cnt ? rho_sum / rho_cnt : 1.0;
  // data statistics (targets before scaling), for the training report
  unsigned long long *bad = dalloc<unsigned long long>(c, 2);
  unsigned *mx = (unsigned *)(bad + 1);
  CK(cudaMemsetAsync(bad, 0, 2 * sizeof(unsigned long long), c->stream));
  CK(mlp_stats(Tall, R * N.No, mx, bad, c->stream));
  unsigned long long hbad = 0;
  unsigned hmx = 0;
  CK(cudaMemcpyAsync(&hbad, bad, sizeof(hbad), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(&hmx, mx, sizeof(hmx), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  float tmax;
  std::memcpy(&tmax, &hmx, sizeof(tmax));
  // output scale: RMS of the targets
  CK(cudaMemsetAsync(N.loss, 0, 2 * sizeof(double), c->stream));
  CK(mlp_sumsq(Tall, R * N.No, N.loss, c->stream));
  double ss;
  CK(cudaMemcpyAsync(&ss, N.loss, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  const double cs = std::sqrt(ss / ((double)R * N.n3)) + 1e-300;
  N.cscale = (float)cs;
  CK(mlp_scale(Tall, R * N.No, (float)(1.0 / cs), c->stream));
  // Adam over strided minibatches (rows i, i + NB, i + 2 NB, ...)
  CK(cudaMemsetAsync(N.M, 0, N.np * sizeof(float), c->stream));
  CK(cudaMemsetAsync(N.V, 0, N.np * sizeof(float), c->stream));
  double loss_first = 0, loss_last = 0;
  int step = 0;
  for (int ep = 0; ep < epochs; ++ep) {
    CK(cudaMemsetAsync(N.loss, 0, sizeof(double), c->stream));
    for (int i = 0; i < NB; ++i) {
      net_gradients(c, bf(Xall, (long)i * N.Fp), (long)NB * N.Fp, Tall + (long)i * N.No, (long)NB * N.No, B);
      ++step;
      const float lr = 1e-3f * (ep >= epochs * 2 / 3 ? 0.3f : 1.0f);
      CK(mlp_adam(N.P, N.M, N.V, N.G, N.np, lr, step, N.Pb, c->stream));
      net_weights_updated(c);
    }
    double l;
    CK(cudaMemcpyAsync(&l, N.loss, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    l /= NB;
    if (ep == 0) loss_first = l;
    loss_last = l;
    if (!std::isfinite(l)) {
      c->err = "learned smoother training diverged (non-finite loss) at epoch " + std::to_string(ep) +
               "; target max " + std::to_string(tmax) + ", non-finite targets " + std::to_string(hbad) +
               ", output scale " + std::to_string(cs) + ", first loss " + std::to_string(loss_first);
      return SIPG_ENAN;
    }
  }
  CK(cudaStreamSynchronize(c->stream));
  N.trained = true;
  // graphs of a learned cycle captured earlier hold old weights only by pointer: nothing to redo
  {
    // Damping of the learned step on the data it was trained for: on the last
    // snapshot's residual after pre-smoothing and coarse-grid correction, r,
    // take the step d = corr(r) from x = 0 and scale the output by the omega
    // minimising ||r - omega A d||, so that the step does not increase such
    // residuals.
    learned_smooth<double>(c, bv, xx, 1, true);
    apply_level<double>(c, c->L, xx, e, 0);
    const double rad = dot(c, bv, e, Nd, 11), add = dot(c, e, e, Nd, 12), rr = dot(c, bv, bv, Nd, 13);
    const double omega = (add > 0 && std::isfinite(rad / add)) ? rad / add : 0.0;
    // ||r - omega A d|| / ||r|| with the optimal omega
    N.step_reduction = rr > 0 ? std::sqrt(std::max(0.0, rr - omega * rad) / rr) : 1.0;
    N.cscale = (float)(N.cscale * std::max(0.0, omega));
    N.omega = omega;
  }
  N.t_iter_cheb = iteration_ms(c, 0);
  N.t_iter_learned = iteration_ms(c, 1);
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->npairs = (int)R;
    info->epochs = epochs;
    info->steps = step;
    info->loss_first = loss_first;
    info->loss_last = loss_last;
    info->out_scale = cs;
    info->cheb_rate = N.rho_cheb;
    info->target_max = tmax;
    info->nonfinite = (double)hbad;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    info->iter_ms_chebyshev = N.t_iter_cheb;
    info->iter_ms_learned = N.t_iter_learned;
    info->damping = N.omega;
    info->step_reduction = N.step_reduction;
  }
  return SIPG_OK;
}

// Energy-norm fine-tuning of the trained network on the full-mesh
// snapshots of training: for a snapshot's residual r and error e (A e = r)
// the step of all cells is d = c s net(features(r)) and the loss
// ||e - d||_A^2 / ||e||_A^2 = (e - d).(r - A d) / e.r; its gradient with
// respect to d is -2 (r - A d) / e.r, one operator application per step (the
// 2-norm training target e of one cell leaves what the step does to its
// neighbours' residuals out; this loss sees it).  Adam (learning rate lr) over
// all cells of one snapshot per step, `epochs` passes over the snapshots; then
// the step is damped by the energy-optimal omega = d.r / d.A d on the last
// snapshot.
sipg_status finetune_impl(sipg_ctx *c, int epochs, float lr, sipg_train_info *info) {
  auto t0 = std::chrono::steady_clock::now();
  auto &N = c->net;
  const Level &F = c->lv[c->L];
  const int E = (int)F.ncells;
  const int64_t Nd = F.ndofs;
  net_setup(c, std::max<long>(E, 256));
  double *d = dalloc<double>(c, Nd), *ad = dalloc<double>(c, Nd), *rp = dalloc<double>(c, Nd),
         *ep = dalloc<double>(c, Nd);
  double loss_first = 0, loss_last = 0;
  int step = 0;
  // Adam moments restart for the new objective
  CK(cudaMemsetAsync(N.M, 0, N.np * sizeof(float), c->stream));
  CK(cudaMemsetAsync(N.V, 0, N.np * sizeof(float), c->stream));
  auto take_step = [&](int k) {   // d, A d, r' = r - A d, e' = e - d for snapshot k
    const double *r = N.snap_r + (int64_t)k * Nd;
    CK(mlp_gather<double>(r, F.n, F.m, nullptr, 0, E, N.X, N.Fp, N.scale, c->stream));
    net_forward(c, N.X, N.Fp, E, true);
    CK(cudaMemsetAsync(d, 0, Nd * sizeof(double), c->stream));
    CK(mlp_correct<double>(d, N.n3, 0, E, N.Y, N.No, N.scale, N.cscale, c->stream));
    apply_level<double>(c, c->L, d, ad, 0);
    CK(cudaMemcpyAsync(rp, r, Nd * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    CK(launch_axpy<double>(rp, -1.0, ad, Nd, c->stream));
    CK(cudaMemcpyAsync(ep, N.snap_e + (int64_t)k * Nd, Nd * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    CK(launch_axpy<double>(ep, -1.0, d, Nd, c->stream));
  };
  for (int ep_i = 0; ep_i < epochs; ++ep_i) {
    double lsum = 0;
    for (int k = 0; k < N.nsnap; ++k) {
      take_step(k);
      const double er = dot(c, N.snap_e + (int64_t)k * Nd, N.snap_r + (int64_t)k * Nd, Nd, 11);
      const double l = dot(c, ep, rp, Nd, 12) / er;
      lsum += l;
      CK(mlp_energy_grad(rp, N.n3, E, N.scale, N.cscale, -2.0 / er, N.No, N.dY, N.dYf, c->stream));
      net_backward(c, N.X, N.Fp, E);
      ++step;
      CK(mlp_adam(N.P, N.M, N.V, N.G, N.np, lr, step, N.Pb, c->stream));
      net_weights_updated(c);
    }
    lsum /= N.nsnap;
    if (!std::isfinite(lsum)) {
      c->err = "energy-norm fine-tuning diverged (non-finite loss) at epoch " + std::to_string(ep_i);
      return SIPG_ENAN;
    }
    if (ep_i == 0) loss_first = lsum;
    loss_last = lsum;
  }
  // energy-optimal damping on the last snapshot
  take_step(N.nsnap - 1);
  const double *r = N.snap_r + (int64_t)(N.nsnap - 1) * Nd;
  const double dr = dot(c, d, r, Nd, 11), dad = dot(c, d, ad, Nd, 12);
  const double omega = (dad > 0 && std::isfinite(dr / dad)) ? dr / dad : 0.0;
  N.cscale = (float)(N.cscale * std::max(0.0, omega));
  N.omega = omega;
  N.t_iter_learned = iteration_ms(c, 1);
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->epochs = epochs;
    info->steps = step;
    info->loss_first = loss_first;
    info->loss_last = loss_last;
    info->out_scale = N.cscale;
    info->cheb_rate = N.rho_cheb;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    info->iter_ms_chebyshev = N.t_iter_cheb;
    info->iter_ms_learned = N.t_iter_learned;
    info->damping = omega;
  }
  return SIPG_OK;
}

template <typename F>
sipg_status guarded(sipg_ctx *c, F &&f) {
  std::string *prev = t_err;
  t_err = c ? &c->err : &g_create_err;
  sipg_status st;
  try {
    st = f();
  } catch (const Fail &e) {
    st = e.st;
  } catch (const std::exception &e) {
    if (t_err) *t_err = e.what();
    st = SIPG_ENOMEM;
  }
  t_err = prev;
  return st;
}

bool level_ok(const sipg_ctx *c, int l) { return c && l >= 0 && l <= c->L; }

}  // namespace

extern "C" {

void sipg_default_params(sipg_params *p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->degree = 3;
  p->penalty_factor = 1.0;
  p->precision = 0;
  p->p_coarsen = 0;
  p->cheb_degree = 5;
  p->cheb_lo = 0.06;
  p->cheb_hi = 1.2;
  p->eig_iters = 20;
  p->lambda_override = 0.0;
  p->smoother = 0;
  p->operator_only = 0;
  std::strcpy(p->coarsening, "cph");
  p->fe_assemble = 1;
  p->coarse_dense_max = 2197;
  p->coarse_iters = 50;
  p->coarse_solver = 0;
  p->coarse_rtol = 1e-3;
  p->coarse_maxit = 12;
  p->fuse_tail = 1;
  p->stream = nullptr;
}

sipg_status sipg_create(const sipg_mesh *mesh, const sipg_params *params, sipg_ctx **out) {
  if (!out) return SIPG_EINVAL;
  *out = nullptr;
  auto c = std::make_unique<sipg_ctx>();
  sipg_status st = guarded(nullptr, [&]() -> sipg_status {
    if (!mesh || !params) throw_inval("null mesh or params");
    const sipg_mesh &M = *mesh;
    const sipg_params &P = *params;
    if (P.degree < 1 || P.degree > 8) throw_inval("degree must be in 1..8");
    for (int d = 0; d < 3; ++d) {
      if (M.m[d] < 1) throw_inval("m must be >= 1");
      if (!(M.hi[d] > M.lo[d])) throw_inval("box extents must be positive");
    }
    if (M.deform && M.mapping_degree != 3) throw_inval("curved cells need mapping_degree 3");
    if (!(P.penalty_factor > 0)) throw_inval("penalty factor must be positive");
    if (P.precision != 0 && P.precision != 1) throw_inval("precision must be 0 or 1");
    if (P.cheb_degree < 1 || P.eig_iters < 1 || P.p_coarsen < 0 || P.p_coarsen > 2 || P.smoother != 0)
      throw_inval("unsupported smoother parameters");
    if (P.coarse_solver < 0 || P.coarse_solver > 1 || !(P.coarse_rtol > 0 && P.coarse_rtol < 1) ||
        P.coarse_maxit < 1 || P.coarse_maxit > 1000)
      throw_inval("coarse_solver must be 0 or 1, coarse_rtol in (0, 1) and coarse_maxit in 1..1000");
    if (P.fuse_tail != 0 && P.fuse_tail != 1) throw_inval("fuse_tail must be 0 or 1");
    for (int s = 0; s < 6; ++s)
      if (M.bc[s] != 0 && M.bc[s] != 1) throw_inval("bc must be 0 (Dirichlet) or 1 (Neumann)");
    const double cells = (double)M.m[0] * M.m[1] * M.m[2];
    if (cells * std::pow(P.degree + 1.0, 3) > 2.0e9) throw_inval("problem too large");
    c->mesh = M;
    c->prm = P;
    c->stream = (cudaStream_t)P.stream;
    t_err = &c->err;
    setup(c.get());
    return SIPG_OK;
  });
  if (st != SIPG_OK) {
    if (!c->err.empty()) g_create_err = c->err;
    amg_destroy(c->amg);
    for (void *p : c->allocs) cudaFree(p);
    return st;
  }
  *out = c.release();
  return SIPG_OK;
}

sipg_status sipg_create_unstructured(const sipg_hex_mesh *mesh, const sipg_params *params, sipg_ctx **out) {
  if (!out) return SIPG_EINVAL;
  *out = nullptr;
  auto c = std::make_unique<sipg_ctx>();
  sipg_status st = guarded(nullptr, [&]() -> sipg_status {
    if (!mesh || !params) throw_inval("null mesh or params");
    const sipg_params &P = *params;
    if (P.degree < 1 || P.degree > 8) throw_inval("degree must be in 1..8");
    if (!(P.penalty_factor > 0)) throw_inval("penalty factor must be positive");
    if (!P.operator_only) throw_inval("unstructured meshes: operator_only must be 1 (no multigrid hierarchy)");
    if (mesh->ncells < 1 || mesh->nverts < 8 || !mesh->vertices || !mesh->cells)
      throw_inval("unstructured mesh: need vertices (>= 8) and cells (>= 1)");
    for (int64_t i = 0; i < (int64_t)mesh->ncells * 8; ++i)
      if (mesh->cells[i] < 0 || mesh->cells[i] >= mesh->nverts) throw_inval("unstructured mesh: vertex id out of range");
    if (mesh->face_bc)
      for (int64_t i = 0; i < (int64_t)mesh->ncells * 6; ++i)
        if (mesh->face_bc[i] != 0 && mesh->face_bc[i] != 1)
          throw_inval("unstructured mesh: face_bc must be 0 (Dirichlet) or 1 (Neumann)");
    if (mesh->deform && !(mesh->hi[0] > mesh->lo[0] && mesh->hi[1] > mesh->lo[1] && mesh->hi[2] > mesh->lo[2]))
      throw_inval("unstructured mesh: deformation box extents must be positive");
    if ((double)mesh->ncells * std::pow(P.degree + 1.0, 3) > 2.0e9) throw_inval("problem too large");
    c->prm = P;
    c->unstructured = true;
    c->stream = (cudaStream_t)P.stream;
    for (int s = 0; s < 6; ++s) c->mesh.bc[s] = 0;
    UMeshIn in;
    in.nverts = mesh->nverts;
    in.ncells = mesh->ncells;
    in.vertices = mesh->vertices;
    in.cells = mesh->cells;
    in.face_bc = mesh->face_bc;
    in.deform = mesh->deform;
    in.amp = mesh->amp;
    for (int d = 0; d < 3; ++d) {
      in.lo[d] = mesh->lo[d];
      in.hi[d] = mesh->hi[d];
    }
    t_err = &c->err;
    setup_unstructured(c.get(), in);
    return SIPG_OK;
  });
  if (st != SIPG_OK) {
    if (!c->err.empty()) g_create_err = c->err;
    for (void *p : c->allocs) cudaFree(p);
    return st;
  }
  *out = c.release();
  return SIPG_OK;
}

sipg_status sipg_destroy(sipg_ctx *c) {
  if (!c) return SIPG_EINVAL;
  cudaStreamSynchronize(c->stream);
  for (auto &g : c->vgraph)
    if (g) cudaGraphExecDestroy(g);
  for (auto &g : c->vgraph_l)
    if (g) cudaGraphExecDestroy(g);
  for (auto &g : c->fcg_graph)
    if (g) cudaGraphExecDestroy(g);
  if (c->mv.graph) cudaGraphExecDestroy(c->mv.graph);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  amg_destroy(c->amg);
  for (void *p : c->allocs) cudaFree(p);
  delete c;
  return SIPG_OK;
}

const char *sipg_last_error(const sipg_ctx *c) { return c ? c->err.c_str() : g_create_err.c_str(); }

sipg_status sipg_num_levels(const sipg_ctx *c, int *nl) {
  if (!c || !nl) return SIPG_EINVAL;
  *nl = c->L + 1;
  return SIPG_OK;
}

sipg_status sipg_num_dofs(const sipg_ctx *c, int level, int64_t *n) {
  if (!level_ok(c, level) || !n) return SIPG_EINVAL;
  *n = c->lv[level].ndofs;
  return SIPG_OK;
}

sipg_status sipg_level_info(const sipg_ctx *c, int level, int *kind, int *degree, int m[3]) {
  if (!level_ok(c, level)) return SIPG_EINVAL;
  const Level &L = c->lv[level];
  if (kind) *kind = L.kind;
  if (degree) *degree = L.deg;
  if (m)
    for (int d = 0; d < 3; ++d) m[d] = L.m[d];
  return SIPG_OK;
}

sipg_status sipg_lambda(const sipg_ctx *c, int level, double *lambda) {
  if (!level_ok(c, level) || !lambda || !c->solver) return SIPG_EINVAL;
  *lambda = c->lv[level].lambda;
  return SIPG_OK;
}

sipg_status sipg_rhs(sipg_ctx *c, int kind, double *b) {
  if (!c || !b || kind != 0 || c->unstructured) return SIPG_EINVAL;
  return guarded(c, [&]() -> sipg_status {
    const Level &F = c->lv[c->L];
    Mapping map(c->md);
    std::vector<double> h, tau;
    manufactured_rhs(map, F.n, tau, h);
    CK(cudaMemcpyAsync(b, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return SIPG_OK;
  });
}

sipg_status sipg_l2_error(sipg_ctx *c, int kind, const double *x, double *err) {
  if (!c || !x || !err || kind != 0 || c->unstructured) return SIPG_EINVAL;
  return guarded(c, [&]() -> sipg_status {
    const Level &F = c->lv[c->L];
    std::vector<double> h(F.ndofs);
    CK(cudaMemcpyAsync(h.data(), x, F.ndofs * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    Mapping map(c->md);
    *err = l2_error_manufactured(map, F.n, h.data());
    return SIPG_OK;
  });
}

sipg_status sipg_level_apply(sipg_ctx *c, int level, int precision, const void *u, void *v) {
  if (!level_ok(c, level) || !u || !v || (precision != 0 && precision != 1)) return SIPG_EINVAL;
  if (u == v) return SIPG_EINVAL;
  if (level != c->L && !c->solver) return SIPG_EINVAL;
  return guarded(c, [&]() -> sipg_status {
    if (precision == 0)
      apply_level<double>(c, level, (const double *)u, (double *)v, 0);
    else
      apply_level<float>(c, level, (const float *)u, (float *)v, 0);
    return SIPG_OK;
  });
}

sipg_status sipg_operator_apply(sipg_ctx *c, int precision, const void *u, void *v) {
  if (!c) return SIPG_EINVAL;
  return sipg_level_apply(c, c->L, precision, u, v);
}

sipg_status sipg_inverse_diagonal(sipg_ctx *c, int level, int precision, void *d) {
  if (!level_ok(c, level) || level == 0 || !d || !c->solver || (precision != 0 && precision != 1))
    return SIPG_EINVAL;
  return guarded(c, [&]() -> sipg_status {
    const Level &L = c->lv[level];
    CK(cudaMemcpyAsync(d, L.dinv[precision], L.ndofs * (precision ? 4 : 8), cudaMemcpyDeviceToDevice, c->stream));
    return SIPG_OK;
  });
}

sipg_status sipg_smooth(sipg_ctx *c, int level, const void *b, void *x, int nsteps) {
  if (!level_ok(c, level) || level == 0 || !b || !x || nsteps < 1 || !c->solver) return SIPG_EINVAL;
  return guarded(c, [&]() -> sipg_status {
    Level &L = c->lv[level];
    const int pi = c->prm.precision;
    const size_t bytes = L.ndofs * (pi ? 4 : 8);
    CK(cudaMemcpyAsync(L.vx[pi], x, bytes, cudaMemcpyDeviceToDevice, c->stream));
    if (pi == 0) {
      double *xx = (double *)L.vx[0], *xt = (double *)L.vt[0];
      chebyshev<double>(c, level, (const double *)b, xx, xt, nsteps, false);
      CK(cudaMemcpyAsync(x, xx, bytes, cudaMemcpyDeviceToDevice, c->stream));
    } else {
      float *xx = (float *)L.vx[1], *xt = (float *)L.vt[1];
      chebyshev<float>(c, level, (const float *)b, xx, xt, nsteps, false);
      CK(cudaMemcpyAsync(x, xx, bytes, cudaMemcpyDeviceToDevice, c->stream));
    }
    return SIPG_OK;
  });
}

sipg_status sipg_restrict(sipg_ctx *c, int level, const void *r, void *rc) {
  if (!level_ok(c, level) || level == 0 || !r || !rc || !c->solver) return SIPG_EINVAL;
  return guarded(c, [&]() -> sipg_status {
    if (c->prm.precision == 0)
      restrict_level<double>(c, level, (const double *)r, (double *)rc);
    else
      restrict_level<float>(c, level, (const float *)r, (float *)rc);
    return SIPG_OK;
  });
}

sipg_status sipg_prolongate_add(sipg_ctx *c, int level, const void *xc, void *x) {
  if (!level_ok(c, level) || level == 0 || !xc || !x || !c->solver) return SIPG_EINVAL;
  return guarded(c, [&]() -> sipg_status {
    if (c->prm.precision == 0)
      prolongate_level<double>(c, level, (const double *)xc, (double *)x);
    else
      prolongate_level<float>(c, level, (const float *)xc, (float *)x);
    return SIPG_OK;
  });
}

sipg_status sipg_coarse_solve(sipg_ctx *c, const double *b, double *x) {
  if (!c || !b || !x || !c->solver) return SIPG_EINVAL;
  return guarded(c, [&]() -> sipg_status {
    if (c->coarse_cg) coarse_cg_solve<double>(c, b, x);
    else CK((launch_dense_gemv<double, double>(c->Ainv, b, x, c->n0, c->stream)));
    return SIPG_OK;
  });
}

sipg_status sipg_coarse_info(sipg_ctx *c, int *kind, int *nlevels, int sizes[10], int *last_iterations) {
  if (!c || !c->solver) return SIPG_EINVAL;
  return guarded(c, [&]() -> sipg_status {
    const int k = !c->coarse_cg ? 0 : (c->amg ? 2 : 1);
    if (kind) *kind = k;
    int nl = 0, sz[10] = {0};
    if (c->amg) nl = amg_level_sizes(c->amg, sz, 10);
    if (nlevels) *nlevels = nl;
    if (sizes)
      for (int i = 0; i < 10; ++i) sizes[i] = sz[i];
    int it = 0;
    if (c->amg && last_iterations) CK(amg_last_iterations(c->amg, &it, c->stream));
    if (last_iterations) *last_iterations = it;
    return SIPG_OK;
  });
}

sipg_status sipg_coarse_amg_vcycle(sipg_ctx *c, const double *b, double *x) {
  if (!c || !b || !x || !c->solver || !c->amg) return SIPG_EINVAL;
  return guarded(c, [&]() -> sipg_status {
    CK(amg_vcycle(c->amg, b, x, c->stream));
    return SIPG_OK;
  });
}

sipg_status sipg_vcycle(sipg_ctx *c, const double *r, double *z) {
  if (!c || !r || !z || !c->solver) return SIPG_EINVAL;
  return guarded(c, [&]() -> sipg_status {
    c->use_learned = (c->smoother >= 1 && c->net.trained) ? 1 : 0;
    vcycle_fp64io(c, r, z);
    c->use_learned = 0;
    return SIPG_OK;
  });
}

sipg_status sipg_solve(sipg_ctx *c, const double *b, double *x, double rtol, int maxit, int fixed_iters,
                       sipg_solve_info *info) {
  if (!c || !b || !x || !c->solver || maxit < 0 || fixed_iters < 0 || !(rtol >= 0)) return SIPG_EINVAL;
  return guarded(c, [&]() -> sipg_status { return solve_impl(c, b, x, rtol, maxit, fixed_iters, info); });
}

sipg_status sipg_solve_host(sipg_ctx *c, const double *bh, double *xh, double rtol, int maxit,
                            sipg_solve_info *info) {
  if (!c || !bh || !xh || !c->solver) return SIPG_EINVAL;
  return guarded(c, [&]() -> sipg_status {
    const int64_t N = c->lv[c->L].ndofs;
    CK(cudaMemcpyAsync(c->fb, bh, N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemsetAsync(c->fx, 0, N * sizeof(double), c->stream));
    const sipg_status st = solve_impl(c, c->fb, c->fx, rtol, maxit, 0, info);
    CK(cudaMemcpyAsync(xh, c->fx, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return st;
  });
}

sipg_status sipg_time_apply(sipg_ctx *c, int precision, const void *u, void *v, int repeats, float *ms_eval,
                            float *ms_int) {
  if (!c || !u || !v || repeats < 1 || (precision != 0 && precision != 1)) return SIPG_EINVAL;
  return guarded(c, [&]() -> sipg_status {
    const Level &L = c->lv[c->L];
    cudaEvent_t ev[3];
    for (auto &e : ev) CK(cudaEventCreate(&e));
    float te = 0, ti = 0;
    for (int r = 0; r < repeats; ++r) {
      CK(cudaEventRecord(ev[0], c->stream));
      if (precision == 0) {
        DGArgs<double> a = dg_args<double>(c, L);
        a.u = (const double *)u;
        a.out = (double *)v;
        CK(launch_dg_eval<double>(L.n, L.curved, a, c->stream, L.cb[0][0]));
        CK(cudaEventRecord(ev[1], c->stream));
        CK(launch_dg_integrate<double>(L.n, L.curved, a, c->stream, L.cb[0][1]));
      } else {
        DGArgs<float> a = dg_args<float>(c, L);
        a.u = (const float *)u;
        a.out = (float *)v;
        CK(launch_dg_eval<float>(L.n, L.curved, a, c->stream, L.cb[1][0]));
        CK(cudaEventRecord(ev[1], c->stream));
        CK(launch_dg_integrate<float>(L.n, L.curved, a, c->stream, L.cb[1][1]));
      }
      CK(cudaEventRecord(ev[2], c->stream));
      CK(cudaEventSynchronize(ev[2]));
      float a1, a2;
      CK(cudaEventElapsedTime(&a1, ev[0], ev[1]));
      CK(cudaEventElapsedTime(&a2, ev[1], ev[2]));
      te += a1;
      ti += a2;
    }
    for (auto &e : ev) cudaEventDestroy(e);
    if (ms_eval) *ms_eval = te / repeats;
    if (ms_int) *ms_int = ti / repeats;
    return SIPG_OK;
  });
}

sipg_status sipg_tile_shape(const sipg_ctx *c, int level, int precision, int pass, int *cells_per_block) {
  if (!c || !cells_per_block || precision < 0 || precision > 1 || pass < 0 || pass > 2 || level < 0 ||
      level > c->L || (c->lv[level].kind == 0) != (pass < 2))
    return SIPG_EINVAL;
  const int v = c->lv[level].cb[precision][pass];
  const int n = c->lv[level].n;
  *cells_per_block = v ? v : (precision == 0 ? dg_cells_per_block<double>(n) : dg_cells_per_block<float>(n));
  return SIPG_OK;
}

sipg_status sipg_set_tile_shape(sipg_ctx *c, int level, int precision, int pass, int cells_per_block) {
  if (!c || precision < 0 || precision > 1 || pass < 0 || pass > 2 || level < 0 || level > c->L ||
      (c->lv[level].kind == 0) != (pass < 2))
    return SIPG_EINVAL;
  const int n = c->lv[level].n;
  const int mx = pass < 2 ? (precision == 0 ? dg_max_cells_per_block<double>(n) : dg_max_cells_per_block<float>(n))
                          : (precision == 0 ? fe_max_cells_per_block<double>(n) : fe_max_cells_per_block<float>(n));
  if (cells_per_block < 0 || cells_per_block > mx) return SIPG_EINVAL;
  c->lv[level].cb[precision][pass] = cells_per_block ? cells_per_block : c->lv[level].cb0[precision][pass];
  // captured V-cycles hold the old launch shapes
  for (int p = 0; p < 2; ++p) {
    if (c->vgraph[p]) cudaGraphExecDestroy(c->vgraph[p]);
    if (c->vgraph_l[p]) cudaGraphExecDestroy(c->vgraph_l[p]);
    if (c->fcg_graph[p]) cudaGraphExecDestroy(c->fcg_graph[p]);
    c->vgraph[p] = c->vgraph_l[p] = c->fcg_graph[p] = nullptr;
    c->vcalls[p] = c->vcalls_l[p] = 0;
  }
  if (c->mv.graph) cudaGraphExecDestroy(c->mv.graph);
  c->mv.graph = nullptr;
  c->mv.calls = 0;
  return SIPG_OK;
}

// A tensor-core GEMM whose MMA wait ran out wrote no output: report it.
static sipg_status tc_check(sipg_ctx *c) {
  CK(cudaStreamSynchronize(c->stream));
  int timed_out = 0;
  CK(mlp_tc_status(&timed_out));
  if (timed_out) {
    c->err = "a tensor-core GEMM of the learned smoother timed out waiting for its MMAs";
    return SIPG_ETIMEOUT;
  }
  return SIPG_OK;
}

sipg_status sipg_smoother_train(sipg_ctx *c, int npairs, int epochs, uint64_t seed, sipg_train_info *info) {
  if (!c || !c->solver || npairs < 256 || npairs > 10000000 || epochs < 1) return SIPG_EINVAL;
  return guarded(c, [&]() -> sipg_status {
    const sipg_status st = train_impl(c, npairs, epochs, seed, info);
    const sipg_status tc = tc_check(c);
    return st != SIPG_OK ? st : tc;
  });
}

sipg_status sipg_smoother_finetune(sipg_ctx *c, int epochs, double lr, sipg_train_info *info) {
  if (!c || epochs < 1 || epochs > 100000 || !c->solver || !(lr >= 0.0) || lr > 1.0) return SIPG_EINVAL;
  if (!c->net.trained || c->net.nsnap < 1) {
    c->err = "the learned smoother has not been trained (sipg_smoother_train)";
    return SIPG_EINVAL;
  }
  return guarded(c, [&]() -> sipg_status {
    const sipg_status st = finetune_impl(c, epochs, lr > 0 ? (float)lr : 3e-4f, info);
    if (st == SIPG_OK) return tc_check(c);
    return st;
  });
}

sipg_status sipg_set_smoother(sipg_ctx *c, int which, int steps_pre, int steps_post) {
  if (!c || which < 0 || which > 2 || steps_pre < 0 || steps_post < 0 || steps_pre > 16 || steps_post > 16)
    return SIPG_EINVAL;
  if (which >= 1 && !c->net.trained) {
    c->err = "the learned smoother has not been trained (sipg_smoother_train)";
    return SIPG_EINVAL;
  }
  c->smoother = which;
  if (c->net.steps_pre != steps_pre || c->net.steps_post != steps_post) {
    for (auto &g : c->vgraph_l)
      if (g) {
        cudaGraphExecDestroy(g);
        g = nullptr;
      }
    c->vcalls_l[0] = c->vcalls_l[1] = 0;
  }
  const bool changed = c->net.steps_pre != steps_pre || c->net.steps_post != steps_post;
  c->net.steps_pre = steps_pre;
  c->net.steps_post = steps_post;
  if (which >= 1 && changed)   // the fallback test compares time per iteration
    return guarded(c, [&]() -> sipg_status {
      c->net.t_iter_learned = iteration_ms(c, 1);
      return SIPG_OK;
    });
  return SIPG_OK;
}

sipg_status sipg_mlp_shape(sipg_ctx *c, int *in_dim, int *in_pad, int *hidden, int *out_dim, int *out_pad,
                           int64_t *nparams) {
  if (!c || !c->solver) return SIPG_EINVAL;
  return guarded(c, [&]() -> sipg_status {
    net_setup(c, 256);
    const auto &N = c->net;
    if (in_dim) *in_dim = N.F;
    if (in_pad) *in_pad = N.Fp;
    if (hidden) *hidden = N.H;
    if (out_dim) *out_dim = N.n3;
    if (out_pad) *out_pad = N.No;
    if (nparams) *nparams = N.np;
    return SIPG_OK;
  });
}

sipg_status sipg_mlp_params(sipg_ctx *c, int set, float *host) {
  if (!c || !c->solver || !host) return SIPG_EINVAL;
  return guarded(c, [&]() -> sipg_status {
    net_setup(c, 256);
    auto &N = c->net;
    if (set) {
      CK(cudaMemcpyAsync(N.P, host, N.np * sizeof(float), cudaMemcpyHostToDevice, c->stream));
      CK(mlp_f2bf(N.P, N.Pb, N.np, c->stream));
      net_weights_updated(c);
    } else {
      CK(cudaMemcpyAsync(host, N.P, N.np * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    return SIPG_OK;
  });
}

sipg_status sipg_mlp_forward(sipg_ctx *c, const float *X, int B, float *Y) {
  if (!c || !c->solver || !X || !Y || B < 1) return SIPG_EINVAL;
  return guarded(c, [&]() -> sipg_status {
    net_setup(c, B);
    auto &N = c->net;
    CK(mlp_pad_f2bf(X, B, N.F, N.Fp, N.X, c->stream));
    net_forward(c, N.X, N.Fp, B);
    CK(cudaMemcpyAsync(Y, N.Y, (size_t)B * N.No * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
    return tc_check(c);
  });
}

sipg_status sipg_mlp_gradients(sipg_ctx *c, const float *X, const float *T, int B, float *grads_host,
                               double *loss) {
  if (!c || !c->solver || !X || !T || !grads_host || B < 1) return SIPG_EINVAL;
  return guarded(c, [&]() -> sipg_status {
    net_setup(c, B);
    auto &N = c->net;
    CK(mlp_pad_f2bf(X, B, N.F, N.Fp, N.X, c->stream));
    CK(cudaMemsetAsync(N.loss, 0, sizeof(double), c->stream));
    net_gradients(c, N.X, N.Fp, T, N.n3, B);
    CK(cudaMemcpyAsync(grads_host, N.G, N.np * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    double l = 0;
    CK(cudaMemcpyAsync(&l, N.loss, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (loss) *loss = l;
    return tc_check(c);
  });
}

sipg_status sipg_mlp_features(sipg_ctx *c, const double *r, float *feat, float *scale) {
  if (!c || !c->solver || !r || !feat || !scale) return SIPG_EINVAL;
  return guarded(c, [&]() -> sipg_status {
    const Level &F = c->lv[c->L];
    net_setup(c, F.ncells);
    auto &N = c->net;
    CK(mlp_gather<double>(r, F.n, F.m, nullptr, 0, (int)F.ncells, N.X, N.Fp, scale, c->stream));
    CK(mlp_bf2f(N.X, F.ncells * (long)N.Fp, feat, c->stream));
    return SIPG_OK;
  });
}

sipg_status sipg_launch_count(unsigned long long *n) {
  if (!n) return SIPG_EINVAL;
  *n = launch_count();
  return SIPG_OK;
}

sipg_status sipg_fma_peak(int precision, void *stream, double *flops) {
  if (!flops || precision < 0 || precision > 2) return SIPG_EINVAL;
  const cudaError_t e = fma_peak(precision, (cudaStream_t)stream, flops);
  return e == cudaSuccess ? SIPG_OK : SIPG_ECUDA;
}

}  // extern "C"

// ------------------------------------------------------------------ batches

// One V-cycle of all problems of a batch as one captured graph: the two
// finest levels of every problem (its DG level and the FE level of the same
// degree, whose operators dominate the cycle) run as shared launches, each
// Chebyshev step, residual and c-transfer one batched launch over all
// problems' cells or nodes; below them each problem's own cycle (its
// restriction, lower levels, coarse solve, prolongation) is a branch of the
// graph, the branches of different problems side by side.
struct BLaunch {
  int kind;     // 0 vector op over DG points, 1 over FE nodes, 2 DG evaluation, 3 DG integration,
                // 4 FE cell pass, 5 FE node pass, 6 c-prolongation, 7 the per-problem branches
  size_t off;   // the launch's first task in its task array (one task per problem)
};

template <typename T>
struct BatchCycle {
  int np = 0;
  bool curved = false;
  BatchPlan<T> dg;                        // DG work items of the finest levels
  WorkItem *fe_items = nullptr;           // FE cell items
  int n_fe_items = 0;
  size_t fe_smem = 0;
  NodeItem *items_d = nullptr, *items_g = nullptr;   // DG points, FE nodes
  int n_d = 0, n_g = 0;
  VecTask *vec = nullptr;
  BatchProb<T> *dgt = nullptr;
  FETask<T> *fet = nullptr;
  std::vector<BLaunch> prog;
  std::vector<T *> br_r, br_x;            // per problem: FE residual to restrict, FE iterate to correct
  std::vector<char> solo;                 // problems that fill the GPU alone: own cycle, beside the rest
  cudaGraphExec_t graph = nullptr;
  long long kernels = 0;
  ~BatchCycle() {
    if (graph) cudaGraphExecDestroy(graph);
    batch_plan_free(dg);
    for (void *q : {(void *)fe_items, (void *)items_d, (void *)items_g, (void *)vec, (void *)dgt, (void *)fet})
      cudaFree(q);
  }
};

struct sipg_batch {
  std::vector<sipg_ctx *> ctx;
  std::vector<cudaStream_t> streams;   // one per problem (created here)
  cudaStream_t stream = nullptr;       // caller's stream for the batched kernels
  BatchPlan<double> plan;
  std::vector<Seg> segs;
  Seg *d_segs = nullptr;
  SegGrid sg;                      // block map of the batched vector kernels
  std::vector<void *> sg_allocs;
  double *sc = nullptr, *partials = nullptr;
  unsigned *counters = nullptr;
  cudaEvent_t ev_start = nullptr, ev_branch = nullptr;
  std::vector<cudaEvent_t> ev_done;
  std::string err;
  // the batched cycle (state 0 not tried, 1 built, -1 not applicable)
  int cyc_state = 0;
  std::unique_ptr<BatchCycle<double>> cyc_d;
  std::unique_ptr<BatchCycle<float>> cyc_f;
  // flexible CG gated on the device: chunk graph, state and descriptors
  cudaGraphExec_t fcg_graph = nullptr;
  long long fcg_k0 = 0;
  std::vector<long long> fcg_kA, fcg_kB;
  cudaStream_t cap_stream = nullptr;
  BatchProb<double> *d_app = nullptr;   // v = A p descriptors
  int *d_it = nullptr, *d_status = nullptr, *d_any = nullptr;
  double *d_hist = nullptr, *d_rn = nullptr, *d_r0 = nullptr, *d_prm = nullptr;
};

namespace {

void batch_free(sipg_batch *B) {
  if (!B) return;
  if (B->stream) cudaStreamSynchronize(B->stream);
  B->cyc_d.reset();
  B->cyc_f.reset();
  if (B->fcg_graph) cudaGraphExecDestroy(B->fcg_graph);
  if (B->cap_stream) cudaStreamDestroy(B->cap_stream);
  for (void *q : {(void *)B->d_app, (void *)B->d_it, (void *)B->d_status, (void *)B->d_any, (void *)B->d_hist,
                  (void *)B->d_rn, (void *)B->d_r0, (void *)B->d_prm})
    cudaFree(q);
  for (auto *c : B->ctx)
    if (c) sipg_destroy(c);
  for (auto s : B->streams) cudaStreamDestroy(s);
  batch_plan_free(B->plan);
  cudaFree(B->d_segs);
  cudaFree(B->sc);
  cudaFree(B->partials);
  for (void *q : B->sg_allocs) cudaFree(q);
  cudaFree(B->counters);
  if (B->ev_start) cudaEventDestroy(B->ev_start);
  if (B->ev_branch) cudaEventDestroy(B->ev_branch);
  for (auto e : B->ev_done) cudaEventDestroy(e);
  delete B;
}

template <typename T>
BatchCycle<T> *batch_cycle(sipg_batch *B);

// all problems' preconditioners z = M^-1 r: the batched cycle's graph, else
// each problem's cycle on its own stream, overlapping
void batch_precondition(sipg_batch *B) {
  if (B->cyc_state == 1) {
    const long long k = B->cyc_d ? B->cyc_d->kernels : B->cyc_f->kernels;
    CK(cudaGraphLaunch(B->cyc_d ? B->cyc_d->graph : B->cyc_f->graph, B->stream));
    note_kernels(k);
    return;
  }
  CK(cudaEventRecord(B->ev_start, B->stream));
  for (size_t p = 0; p < B->ctx.size(); ++p) {
    if (!B->segs[p].active) continue;
    CK(cudaStreamWaitEvent(B->streams[p], B->ev_start, 0));
    precondition(B->ctx[p]);
    CK(cudaEventRecord(B->ev_done[p], B->streams[p]));
    CK(cudaStreamWaitEvent(B->stream, B->ev_done[p], 0));
  }
}

void batch_set_plan(sipg_batch *B, int mode, const double *const *u, double *const *out) {
  for (size_t p = 0; p < B->ctx.size(); ++p) {
    DGArgs<double> &a = B->plan.probs[p].a;
    a.mode = mode;
    a.u = u[p];
    a.out = out[p];
    a.b = B->segs[p].b;
    B->plan.probs[p].active = B->segs[p].active;
  }
}

// Flexible CG (Section 3, Algorithm 1 with Notay's beta) for np systems in
// lockstep: every step runs on all active systems at once, the scalars of
// system p sit at sc[p * kSegSlots + slot] (0 gamma, 1 z.Ap, 2 p.Ap, 3 r.r,
// 4 b.b, 5 r0.r0); a system leaves the iteration when it converges, breaks
// down or reaches maxit.  residual(): r = b - A x; apply(): v = A p;
// precondition(): z = M^-1 r, each for all systems.
struct Lockstep {
  cudaStream_t s;
  std::vector<Seg> &segs;
  Seg *d_segs;
  const SegGrid &g;
  double *sc, *partials;
  unsigned *counters;
  std::string &err;
};

template <typename FR, typename FA, typename FP>
sipg_status lockstep_fcg(Lockstep K, FR residual, FA apply, FP precondition_all, double rtol, int maxit,
                         sipg_solve_info *infos) {
  const int np = (int)K.segs.size();
  cudaStream_t s = K.s;
  auto upload_segs = [&]() {
    CK(cudaMemcpyAsync(K.d_segs, K.segs.data(), np * sizeof(Seg), cudaMemcpyHostToDevice, s));
  };
  const int st = kSegSlots;
  std::vector<double> hsc((size_t)np * st);
  auto read_sc = [&]() {
    CK(cudaMemcpyAsync(hsc.data(), K.sc, hsc.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  };
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, s));
  upload_segs();
  residual();
  CK(seg_dot(K.d_segs, K.g, 0, K.partials, K.counters, K.sc, st, 4, s));
  precondition_all();
  CK(seg_dot(K.d_segs, K.g, 1, K.partials, K.counters, K.sc, st, 0, s));
  CK(seg_update_p(K.d_segs, K.g, K.sc, st, 1, s));
  read_sc();
  std::vector<double> r0(np), rn(np);
  std::vector<int> it(np, 0);
  std::vector<std::vector<double>> hist(np);
  sipg_status status = SIPG_OK;
  for (int p = 0; p < np; ++p) {
    if (!std::isfinite(hsc[p * st + 4])) {
      K.err = "a right-hand side is not finite";
      status = SIPG_ENAN;
    }
    r0[p] = rn[p] = std::sqrt(hsc[p * st + 5]);
    hist[p].push_back(r0[p]);
    if (r0[p] == 0.0) K.segs[p].active = 0;
  }
  if (status != SIPG_OK) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return status;
  }
  upload_segs();
  while (true) {
    int nact = 0;
    for (int p = 0; p < np; ++p) {
      if (K.segs[p].active && it[p] >= maxit) {
        K.segs[p].active = 0;
        status = SIPG_ENOTCONV;
      }
      nact += K.segs[p].active;
    }
    if (nact == 0) break;
    upload_segs();
    apply();
    CK(seg_dot(K.d_segs, K.g, 2, K.partials, K.counters, K.sc, st, 2, s));
    CK(seg_update_xr(K.d_segs, K.g, K.partials, K.counters, K.sc, st, s));
    read_sc();
    for (int p = 0; p < np; ++p) {
      if (!K.segs[p].active) continue;
      const double *q = &hsc[p * st];
      ++it[p];
      if (!(q[2] > 0) || !std::isfinite(q[3])) {
        K.segs[p].active = 0;
        status = SIPG_EBREAKDOWN;
        K.err = "flexible CG breakdown in one of the systems solved together";
        continue;
      }
      rn[p] = std::sqrt(q[3]);
      hist[p].push_back(rn[p]);
      if (rn[p] <= rtol * r0[p]) K.segs[p].active = 0;
    }
    upload_segs();
    int still = 0;
    for (int p = 0; p < np; ++p) still += K.segs[p].active;
    if (still == 0) break;
    precondition_all();
    CK(seg_dot(K.d_segs, K.g, 3, K.partials, K.counters, K.sc, st, 0, s));
    CK(seg_update_p(K.d_segs, K.g, K.sc, st, 0, s));
  }
  CK(cudaEventRecord(e1, s));
  CK(cudaEventSynchronize(e1));
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (infos)
    for (int p = 0; p < np; ++p) {
      sipg_solve_info &I = infos[p];
      std::memset(&I, 0, sizeof(I));
      I.iterations = it[p];
      I.r0_norm = r0[p];
      I.r_norm = rn[p];
      I.converged = (r0[p] == 0.0 || rn[p] <= rtol * r0[p]) ? 1 : 0;
      I.rho = (it[p] > 0 && r0[p] > 0) ? std::pow(rn[p] / r0[p], 1.0 / it[p]) : 0.0;
      I.n10 = (I.rho > 0 && I.rho < 1) ? -10.0 / std::log10(I.rho) : 0.0;
      I.seconds = ms * 1e-3;
      for (int j = 0; j < (int)hist[p].size() && j < 256; ++j) I.res_history[j] = hist[p][j];
    }
  if (status == SIPG_ENOTCONV) K.err = "a system reached maxit before the tolerance";
  return status;
}

// ------------------------------------------------ the batched V-cycle
// Applicable when every problem has a DG finest level above a matrix-free FE
// level of the same degree (the cph hierarchy's c-transfer first), one
// vector, the batch's common precision and Chebyshev degree, and the batch
// runs on a non-default stream (the cycle is captured).
bool batch_cycle_applicable(const sipg_batch *B) {
  if (!B->stream) return false;
  const sipg_ctx *c0 = B->ctx[0];
  for (const sipg_ctx *c : B->ctx) {
    const int L = c->L;
    if (c->nv != 1 || L < 2 || c->prm.precision != c0->prm.precision ||
        c->prm.cheb_degree != c0->prm.cheb_degree)
      return false;
    const Level &D = c->lv[L], &F = c->lv[L - 1];
    if (D.kind != 0 || F.kind != 1 || D.t_kind != 0 || F.deg != D.deg || D.ufn || D.curved != c0->lv[c0->L].curved ||
        F.stencil[c->prm.precision])
      return false;
  }
  return true;
}

// Issue the batched cycle's launches on s (inside a stream capture): the
// problems that fill the GPU alone run their own cycle on their own stream,
// beside the shared launches of the others.
template <typename T>
void batch_cycle_emit(sipg_batch *B, BatchCycle<T> &C, cudaStream_t s) {
  const Seg *segs = B->d_segs;
  bool forked = false;
  for (int p = 0; p < C.np; ++p) {
    if (!C.solo[p]) continue;
    if (!forked) CK(cudaEventRecord(B->ev_start, s));
    forked = true;
    CK(cudaStreamWaitEvent(B->streams[p], B->ev_start, 0));
    vcycle_body(B->ctx[p], B->ctx[p]->fr, B->ctx[p]->fz);   // on the problem's own stream
    CK(cudaEventRecord(B->ev_done[p], B->streams[p]));
  }
  for (const BLaunch &r : C.prog) {
    switch (r.kind) {
      case 0:
        CK(launch_vec_batched(C.vec + r.off, C.items_d, C.n_d, segs, s));
        break;
      case 1:
        CK(launch_vec_batched(C.vec + r.off, C.items_g, C.n_g, segs, s));
        break;
      case 2:
      case 3:
        CK(batch_dg_pass<T>(C.dg, C.dgt + r.off, r.kind == 3, segs, s));
        break;
      case 4:
        CK(launch_fe_cells_batched<T>(C.curved, C.fet + r.off, C.fe_items, C.n_fe_items, C.fe_smem, segs, s));
        break;
      case 5:
        CK(launch_fe_nodes_batched<T>(C.fet + r.off, C.items_g, C.n_g, segs, 0, s));
        break;
      case 6:
        CK(launch_fe_nodes_batched<T>(C.fet + r.off, C.items_d, C.n_d, segs, 1, s));
        break;
      default: {   // each problem's cycle below its two finest levels, side by side
        CK(cudaEventRecord(B->ev_branch, s));
        for (int p = 0; p < C.np; ++p) {
          if (C.solo[p]) continue;
          sipg_ctx *c = B->ctx[p];
          cudaStream_t own = c->stream;
          CK(cudaStreamWaitEvent(B->streams[p], B->ev_branch, 0));
          c->stream = B->streams[p];
          try {
            const int L = c->L;
            restrict_level<T>(c, L - 1, C.br_r[p], lvec<T>(c, L - 2, 0));
            const T *xc = vcycle_rec<T>(c, L - 2);
            prolongate_level<T>(c, L - 1, xc, C.br_x[p]);
          } catch (...) {
            c->stream = own;
            throw;
          }
          c->stream = own;
          CK(cudaEventRecord(B->ev_done[p], B->streams[p]));
          CK(cudaStreamWaitEvent(s, B->ev_done[p], 0));
        }
      }
    }
  }
  for (int p = 0; p < C.np; ++p)
    if (C.solo[p]) CK(cudaStreamWaitEvent(s, B->ev_done[p], 0));
}

template <typename T>
T *upload_vec(const std::vector<T> &h) {
  T *d = nullptr;
  CK(cudaMalloc(&d, std::max<size_t>(1, h.size()) * sizeof(T)));
  if (!h.empty()) CK(cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  return d;
}

// The program of one cycle (the mirror of vcycle_rec on the two finest
// levels, vcycle_body's conversions around it), its device arrays and its graph.
template <typename T>
std::unique_ptr<BatchCycle<T>> batch_cycle_build(sipg_batch *B) {
  constexpr int pi = pidx<T>();
  auto C = std::make_unique<BatchCycle<T>>();
  const int np = (int)B->ctx.size();
  C->np = np;
  C->curved = B->ctx[0]->lv[B->ctx[0]->L].curved;
  const int ns = B->ctx[0]->prm.cheb_degree;
  std::vector<DGArgs<T>> a0;
  std::vector<int> nn;
  std::vector<WorkItem> fei;
  std::vector<NodeItem> nd, ng;
  // a problem of at least kSoloDofs DoF keeps its own cycle (its launches
  // fill the GPU; in lockstep with small problems it would wait for their
  // lower levels at every shared step)
  constexpr int64_t kSoloDofs = int64_t(1) << 21;
  C->solo.assign(np, 0);
  for (int p = 0; p < np; ++p) {
    sipg_ctx *c = B->ctx[p];
    const Level &D = c->lv[c->L], &F = c->lv[c->L - 1];
    a0.push_back(dg_args<T>(c, D));
    nn.push_back(D.n);
    if (np > 1 && D.ndofs >= kSoloDofs) {
      C->solo[p] = 1;
      a0.back().ncells = 0;   // no DG items
      continue;
    }
    const int cb = kBatchCellThreads / (F.n * F.n);
    C->fe_smem = std::max(C->fe_smem, (size_t)cb * tile_values(F.n) * sizeof(T));
    for (int q = 0; q < F.ncells; q += cb) fei.push_back({p, q, (int)std::min<int64_t>(cb, F.ncells - q)});
    for (int64_t q = 0; q * kBatchNodeThreads < D.ndofs; ++q) nd.push_back({p, (int)q});
    for (int64_t q = 0; q * kBatchNodeThreads < F.ndofs; ++q) ng.push_back({p, (int)q});
  }
  CK(batch_plan_build<T>(C->dg, a0, nn));
  C->dg.curved = C->curved;
  CK(prep_fe_cells_batched<T>(C->fe_smem));
  C->n_fe_items = (int)fei.size();
  C->n_d = (int)nd.size();
  C->n_g = (int)ng.size();
  // the program, task by task
  std::vector<VecTask> hv;
  std::vector<BatchProb<T>> hd;
  std::vector<FETask<T>> hf;
  std::vector<T *> bL(np), xL(np), rL(np), tL(np), bF(np), xF(np), rF(np), tF(np);
  for (int p = 0; p < np; ++p) {
    sipg_ctx *c = B->ctx[p];
    const int L = c->L;
    bL[p] = lvec<T>(c, L, 0), xL[p] = lvec<T>(c, L, 1), rL[p] = lvec<T>(c, L, 2), tL[p] = lvec<T>(c, L, 3);
    bF[p] = lvec<T>(c, L - 1, 0), xF[p] = lvec<T>(c, L - 1, 1), rF[p] = lvec<T>(c, L - 1, 2);
    tF[p] = lvec<T>(c, L - 1, 3);
  }
  auto vec = [&](int kind, auto task) {
    C->prog.push_back({kind, hv.size()});
    for (int p = 0; p < np; ++p) hv.push_back(task(p));
  };
  auto dgapply = [&](auto args) {
    C->prog.push_back({2, hd.size()});
    C->prog.push_back({3, hd.size()});
    for (int p = 0; p < np; ++p) {
      BatchProb<T> q{};
      q.a = args(p);
      q.n = nn[p];
      q.active = 1;
      hd.push_back(q);
    }
  };
  auto fetask = [&](int kind, auto args) {   // kind 4: cell and node pass; 5: node pass; 6: c-prolongation
    if (kind == 4) C->prog.push_back({4, hf.size()});
    C->prog.push_back({kind == 4 ? 5 : kind, hf.size()});
    for (int p = 0; p < np; ++p) hf.push_back(args(p));
  };
  auto dga = [&](int p, const T *u, T *out, int mode, const T *x, const T *xp, const T *b, const ChebStep *q) {
    sipg_ctx *c = B->ctx[p];
    const Level &D = c->lv[c->L];
    DGArgs<T> a = dg_args<T>(c, D);
    a.u = u, a.out = out, a.mode = mode, a.x = x, a.xp = xp, a.b = b;
    if (q) a.dinv = (const T *)D.dinv[pi], a.c1 = (T)q->c1, a.c2 = (T)q->c2, a.c3 = (T)q->c3;
    return a;
  };
  auto fea = [&](int p, const T *u, T *out, int mode, const T *x, const T *xp, const T *b, const ChebStep *q) {
    sipg_ctx *c = B->ctx[p];
    const Level &F = c->lv[c->L - 1];
    FETask<T> t{};
    t.a = fe_args<T>(c, F);
    t.a.u = u, t.a.out = out, t.a.mode = mode, t.a.x = x, t.a.xp = xp, t.a.b = b;
    if (q) t.a.dinv = (const T *)F.dinv[pi], t.a.c1 = (T)q->c1, t.a.c2 = (T)q->c2, t.a.c3 = (T)q->c3;
    return t;
  };
  // Algorithm 3 on the DG (dg) or FE level of every problem, as chebyshev()
  auto cheb = [&](bool dg, bool zero_start) {
    std::vector<std::vector<ChebStep>> plan(np);
    for (int p = 0; p < np; ++p) plan[p] = cheb_plan(B->ctx[p], B->ctx[p]->L - (dg ? 0 : 1), ns, zero_start);
    std::vector<T *> &x = dg ? xL : xF, &xt = dg ? tL : tF, &b = dg ? bL : bF;
    for (int j = 0; j < ns; ++j) {
      if (plan[0][j].xdb) {
        vec(dg ? 0 : 1, [&](int p) {
          const Level &l = B->ctx[p]->lv[B->ctx[p]->L - (dg ? 0 : 1)];
          VecTask v;
          v.op = pi == 1 ? 2 : 3;
          v.n = (long)l.ndofs;
          v.y = x[p], v.x = b[p], v.d = l.dinv[pi], v.c = (double)(T)plan[p][j].c3;
          return v;
        });
        continue;
      }
      if (dg)
        dgapply([&](int p) {
          return dga(p, x[p], xt[p], 1, x[p], plan[p][j].has_prev ? xt[p] : nullptr, b[p], &plan[p][j]);
        });
      else
        fetask(4, [&](int p) {
          return fea(p, x[p], xt[p], 1, x[p], plan[p][j].has_prev ? xt[p] : nullptr, b[p], &plan[p][j]);
        });
      for (int p = 0; p < np; ++p) std::swap(x[p], xt[p]);
    }
  };
  // r (FP64, the solver's fr) -> b of the DG level
  vec(0, [&](int p) {
    VecTask v;
    v.op = pi == 1 ? 0 : 4;
    v.n = (long)B->ctx[p]->lv[B->ctx[p]->L].ndofs;
    v.y = bL[p], v.x = B->ctx[p]->fr;
    return v;
  });
  cheb(true, true);
  dgapply([&](int p) { return dga(p, xL[p], rL[p], 2, nullptr, nullptr, bL[p], nullptr); });
  fetask(5, [&](int p) {   // c-restriction: the DG residual is the FE level's element buffer
    FETask<T> t = fea(p, nullptr, bF[p], 3, nullptr, nullptr, nullptr, nullptr);
    t.a.ebuf = rL[p];
    return t;
  });
  cheb(false, true);
  fetask(4, [&](int p) { return fea(p, xF[p], rF[p], 2, nullptr, nullptr, bF[p], nullptr); });
  C->prog.push_back({7, 0});
  C->br_r = rF;
  C->br_x = xF;
  cheb(false, false);
  fetask(6, [&](int p) {
    FETask<T> t = fea(p, nullptr, nullptr, 0, nullptr, nullptr, nullptr, nullptr);
    t.xc = xF[p];
    t.xdg = xL[p];
    return t;
  });
  cheb(true, false);
  vec(0, [&](int p) {   // the DG level's x -> z (FP64, the solver's fz)
    VecTask v;
    v.op = pi == 1 ? 1 : 4;
    v.n = (long)B->ctx[p]->lv[B->ctx[p]->L].ndofs;
    v.y = B->ctx[p]->fz, v.x = xL[p];
    return v;
  });
  C->fe_items = upload_vec(fei);
  C->items_d = upload_vec(nd);
  C->items_g = upload_vec(ng);
  C->vec = upload_vec(hv);
  C->dgt = upload_vec(hd);
  C->fet = upload_vec(hf);
  // capture
  cudaStream_t s = B->stream;
  cudaGraph_t g = nullptr;
  long long kernels = 0;
  CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  try {
    CaptureTally tally(&kernels);
    batch_cycle_emit<T>(B, *C, s);
  } catch (...) {
    cudaStreamEndCapture(s, &g);
    if (g) cudaGraphDestroy(g);
    throw;
  }
  CK(cudaStreamEndCapture(s, &g));
  const cudaError_t e = cudaGraphInstantiate(&C->graph, g, 0);
  cudaGraphDestroy(g);
  CK(e);
  C->kernels = kernels;
  return C;
}

// Build the batched cycle once, on the first preconditioning of a batch
// whose problems allow it.
void batch_cycle_prepare(sipg_batch *B) {
  if (B->cyc_state != 0) return;
  B->cyc_state = -1;
  if (!batch_cycle_applicable(B)) return;
  if (B->ctx[0]->prm.precision == 0) B->cyc_d = batch_cycle_build<double>(B);
  else B->cyc_f = batch_cycle_build<float>(B);
  B->cyc_state = 1;
}

// ------------------------------------ lockstep flexible CG gated on the device
// Chunks of kFcgChunk lockstep iterations captured with conditional nodes:
// iteration i is IF A_i { v = A p (batched), p.v, x and r update, check (per
// system: iteration count, ||r||, leaving on convergence, breakdown or
// maxit; sets B_i = some system active) } IF B_i { the batched cycle, r.z
// and z.v, p update, A_{i+1} = B_i }.  The host reads the state once per chunk.
void batch_build_fcg_chunk(sipg_batch *B) {
  if (B->fcg_graph) return;
  const int np = (int)B->ctx.size();
  if (!B->cap_stream) CK(cudaStreamCreateWithFlags(&B->cap_stream, cudaStreamNonBlocking));
  cudaStream_t s = B->stream, s2 = B->cap_stream;
  cudaGraph_t G = nullptr;
  CK(cudaGraphCreate(&G, 0));
  std::vector<cudaGraphConditionalHandle> hA(kFcgChunk), hB(kFcgChunk);
  for (int i = 0; i < kFcgChunk; ++i) {
    CK(cudaGraphConditionalHandleCreate(&hA[i], G, 0, cudaGraphCondAssignDefault));
    CK(cudaGraphConditionalHandleCreate(&hB[i], G, 0, cudaGraphCondAssignDefault));
  }
  B->fcg_kA.assign(kFcgChunk, 0);
  B->fcg_kB.assign(kFcgChunk, 0);
  B->fcg_k0 = 0;
  auto body = [&](cudaGraph_t b, long long *tally, auto &&fn) {
    CK(cudaStreamBeginCaptureToGraph(s2, b, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    try {
      CaptureTally t(tally);
      fn();
    } catch (...) {
      cudaGraph_t o;
      cudaStreamEndCapture(s2, &o);
      throw;
    }
    cudaGraph_t o;
    CK(cudaStreamEndCapture(s2, &o));
  };
  const int st = kSegSlots;
  CK(cudaStreamBeginCaptureToGraph(s, G, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  try {
    {
      CaptureTally t(&B->fcg_k0);
      CK(launch_batch_fcg_cond(B->d_any, hA[0], s));
    }
    for (int i = 0; i < kFcgChunk; ++i) {
      body(add_if_node(s, hA[i]), &B->fcg_kA[i], [&]() {
        CK(batch_dg_pass<double>(B->plan, B->d_app, false, B->d_segs, s2));
        CK(batch_dg_pass<double>(B->plan, B->d_app, true, B->d_segs, s2));
        CK(seg_dot(B->d_segs, B->sg, 2, B->partials, B->counters, B->sc, st, 2, s2));
        CK(seg_update_xr(B->d_segs, B->sg, B->partials, B->counters, B->sc, st, s2));
        CK(launch_batch_fcg_check(B->sc, st, B->d_segs, np, B->d_it, B->d_status, B->d_hist, B->d_rn, B->d_r0,
                                  B->d_prm, B->d_any, hB[i], s2));
      });
      body(add_if_node(s, hB[i]), &B->fcg_kB[i], [&]() {
        if (B->cyc_d) batch_cycle_emit<double>(B, *B->cyc_d, s2);
        else batch_cycle_emit<float>(B, *B->cyc_f, s2);
        CK(seg_dot(B->d_segs, B->sg, 3, B->partials, B->counters, B->sc, st, 0, s2));
        CK(seg_update_p(B->d_segs, B->sg, B->sc, st, 0, s2));
        if (i + 1 < kFcgChunk) CK(launch_batch_fcg_cond(B->d_any, hA[i + 1], s2));
      });
    }
  } catch (...) {
    cudaGraph_t o = nullptr;
    cudaStreamEndCapture(s, &o);
    if (o) cudaGraphDestroy(o);
    cudaGraphDestroy(G);
    throw;
  }
  cudaGraph_t out = nullptr;
  CK(cudaStreamEndCapture(s, &out));
  cudaGraphExec_t ex = nullptr;
  const cudaError_t e = cudaGraphInstantiate(&ex, out, 0);
  cudaGraphDestroy(out);
  CK(e);
  B->fcg_graph = ex;
}

// The lockstep flexible CG with the iteration gated on the device (the
// batched cycle is built): the host reads the state once per chunk of
// kFcgChunk iterations instead of the scalars every iteration.  Same
// kernels, same order and the same tests as lockstep_fcg.
sipg_status batch_solve_device(sipg_batch *B, const double *const *b, double *const *x, double rtol, int maxit,
                               sipg_solve_info *infos) {
  const int np = (int)B->ctx.size();
  const int st = kSegSlots;
  cudaStream_t s = B->stream;
  std::vector<const double *> xu(np);
  std::vector<double *> rout(np);
  for (int p = 0; p < np; ++p) {
    sipg_ctx *c = B->ctx[p];
    B->segs[p] = Seg{x[p], c->fr, c->fp, c->fv, c->fz, b[p], (long)c->lv[c->L].ndofs, 1};
    xu[p] = x[p];
    rout[p] = c->fr;
  }
  if (!B->d_app) {   // device state, and the v = A p descriptors (fixed per context)
    std::vector<BatchProb<double>> app(np);
    for (int p = 0; p < np; ++p) {
      sipg_ctx *c = B->ctx[p];
      app[p].a = dg_args<double>(c, c->lv[c->L]);
      app[p].a.u = c->fp;
      app[p].a.out = c->fv;
      app[p].a.mode = 0;
      app[p].n = c->lv[c->L].n;
      app[p].active = 1;
    }
    B->d_app = upload_vec(app);
    CK(cudaMalloc(&B->d_it, np * sizeof(int)));
    CK(cudaMalloc(&B->d_status, np * sizeof(int)));
    CK(cudaMalloc(&B->d_any, sizeof(int)));
    CK(cudaMalloc(&B->d_hist, (size_t)np * 257 * sizeof(double)));
    CK(cudaMalloc(&B->d_rn, np * sizeof(double)));
    CK(cudaMalloc(&B->d_r0, np * sizeof(double)));
    CK(cudaMalloc(&B->d_prm, 2 * sizeof(double)));
  }
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  struct EvGuard {
    cudaEvent_t a, b;
    ~EvGuard() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } evg{e0, e1};
  CK(cudaEventRecord(e0, s));
  CK(cudaMemcpyAsync(B->d_segs, B->segs.data(), np * sizeof(Seg), cudaMemcpyHostToDevice, s));
  batch_set_plan(B, 2, xu.data(), rout.data());   // r = b - A x
  CK(batch_apply(B->plan, s));
  CK(seg_dot(B->d_segs, B->sg, 0, B->partials, B->counters, B->sc, st, 4, s));
  batch_precondition(B);
  CK(seg_dot(B->d_segs, B->sg, 1, B->partials, B->counters, B->sc, st, 0, s));
  CK(seg_update_p(B->d_segs, B->sg, B->sc, st, 1, s));
  std::vector<double> hsc((size_t)np * st);
  CK(cudaMemcpyAsync(hsc.data(), B->sc, hsc.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  std::vector<double> r0(np);
  int any = 0;
  for (int p = 0; p < np; ++p) {
    if (!std::isfinite(hsc[p * st + 4])) {
      B->err = "a right-hand side is not finite";
      return SIPG_ENAN;
    }
    r0[p] = std::sqrt(hsc[p * st + 5]);
    if (r0[p] == 0.0) B->segs[p].active = 0;
    any |= B->segs[p].active;
  }
  const double prm[2] = {rtol, (double)maxit};
  CK(cudaMemcpyAsync(B->d_segs, B->segs.data(), np * sizeof(Seg), cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(B->d_it, 0, np * sizeof(int), s));
  CK(cudaMemsetAsync(B->d_status, 0, np * sizeof(int), s));
  CK(cudaMemcpyAsync(B->d_r0, r0.data(), np * sizeof(double), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(B->d_rn, r0.data(), np * sizeof(double), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(B->d_prm, prm, sizeof(prm), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(B->d_any, &any, sizeof(int), cudaMemcpyHostToDevice, s));
  int global_it = 0;
  if (any) {
    batch_build_fcg_chunk(B);
    // every chunk that does not end the solve advances all active systems by
    // kFcgChunk iterations, and the device ends each at maxit
    const int max_launches = maxit / kFcgChunk + 2;
    for (int launches = 0;; ++launches) {
      if (launches >= max_launches) {
        B->err = "the batched flexible CG on the device made no progress";
        throw Fail{SIPG_ECUDA};
      }
      CK(cudaGraphLaunch(B->fcg_graph, s));
      note_kernels(B->fcg_k0);
      int h_any = 0;
      CK(cudaMemcpyAsync(&h_any, B->d_any, sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (!h_any) break;
    }
  }
  std::vector<int> it(np), status(np);
  std::vector<double> rn(np), hist((size_t)np * 257);
  CK(cudaMemcpyAsync(it.data(), B->d_it, np * sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(status.data(), B->d_status, np * sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(rn.data(), B->d_rn, np * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(hist.data(), B->d_hist, hist.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaEventRecord(e1, s));
  CK(cudaEventSynchronize(e1));
  for (int p = 0; p < np; ++p) global_it = std::max(global_it, it[p]);
  // kernels of the bodies that ran: the first step of iterations 1..G, the
  // second of all but the last (G = the most iterations of any system)
  for (int j = 0; j < global_it; ++j)
    note_kernels(B->fcg_kA[j % kFcgChunk] + (j + 1 < global_it ? B->fcg_kB[j % kFcgChunk] : 0));
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  sipg_status status_all = SIPG_OK;
  for (int p = 0; p < np; ++p) {
    if (status[p] == 1) status_all = SIPG_EBREAKDOWN;
    else if (status[p] == 2 && status_all == SIPG_OK) status_all = SIPG_ENOTCONV;
  }
  if (infos)
    for (int p = 0; p < np; ++p) {
      sipg_solve_info &I = infos[p];
      std::memset(&I, 0, sizeof(I));
      I.iterations = it[p];
      I.r0_norm = r0[p];
      I.r_norm = rn[p];
      I.converged = (r0[p] == 0.0 || rn[p] <= rtol * r0[p]) ? 1 : 0;
      I.rho = (it[p] > 0 && r0[p] > 0) ? std::pow(rn[p] / r0[p], 1.0 / it[p]) : 0.0;
      I.n10 = (I.rho > 0 && I.rho < 1) ? -10.0 / std::log10(I.rho) : 0.0;
      I.seconds = ms * 1e-3;
      I.res_history[0] = r0[p];
      const int nh = std::min(status[p] == 1 ? it[p] - 1 : it[p], 255);
      for (int j = 1; j <= nh; ++j) I.res_history[j] = hist[(size_t)p * 257 + j];
    }
  if (status_all == SIPG_EBREAKDOWN) B->err = "flexible CG breakdown in one of the systems solved together";
  if (status_all == SIPG_ENOTCONV) B->err = "a system reached maxit before the tolerance";
  return status_all;
}

sipg_status batch_solve_impl(sipg_batch *B, const double *const *b, double *const *x, double rtol, int maxit,
                             sipg_solve_info *infos) {
  batch_cycle_prepare(B);
  if (B->cyc_state == 1 && maxit > 0) return batch_solve_device(B, b, x, rtol, maxit, infos);
  const int np = (int)B->ctx.size();
  std::vector<const double *> xu(np), pu(np);
  std::vector<double *> rout(np), vout(np);
  for (int p = 0; p < np; ++p) {
    sipg_ctx *c = B->ctx[p];
    B->segs[p] = Seg{x[p], c->fr, c->fp, c->fv, c->fz, b[p], (long)c->lv[c->L].ndofs, 1};
    xu[p] = x[p];
    pu[p] = c->fp;
    rout[p] = c->fr;
    vout[p] = c->fv;
  }
  Lockstep K{B->stream, B->segs, B->d_segs, B->sg, B->sc, B->partials, B->counters, B->err};
  return lockstep_fcg(
      K,
      [&]() {   // r = b - A x
        batch_set_plan(B, 2, xu.data(), rout.data());
        CK(batch_apply(B->plan, B->stream));
      },
      [&]() {   // v = A p
        batch_set_plan(B, 0, pu.data(), vout.data());
        CK(batch_apply(B->plan, B->stream));
      },
      [&]() { batch_precondition(B); }, rtol, maxit, infos);
}

// ------------------------------------------------ many right-hand sides
// Work set for nv vectors of the context's problem: every level's V-cycle
// vectors (V-cycle precision), the cell-kernel scratch (both precisions),
// the flexible-CG vectors and the per-system scalars.  Grown on demand;
// growing drops the captured multi-vector cycle.
void ensure_multi(sipg_ctx *c, int nv) {
  auto &M = c->mv;
  if (M.cap >= nv) return;
  CK(cudaStreamSynchronize(c->stream));
  if (M.graph) cudaGraphExecDestroy(M.graph);
  M.graph = nullptr;
  M.calls = 0;
  M.graph_nv = 0;
  std::vector<void *> old;
  for (void *q : M.v) old.push_back(q);
  for (void *q : M.sg_allocs) old.push_back(q);
  for (void *q : {M.grad[0], M.grad[1], M.trace[0], M.trace[1], M.ebuf[0], M.ebuf[1], (void *)M.r, (void *)M.z,
                  (void *)M.p, (void *)M.v_, (void *)M.d_segs, (void *)M.sc, (void *)M.partials,
                  (void *)M.counters})
    old.push_back(q);
  for (void *q : old) {
    if (!q) continue;
    auto it = std::find(c->allocs.begin(), c->allocs.end(), q);
    if (it != c->allocs.end()) c->allocs.erase(it);
    cudaFree(q);
  }
  M = sipg_ctx::Multi{};   // no pointer survives a regrowth
  const int pi = c->prm.precision;
  const size_t es = pi == 0 ? sizeof(double) : sizeof(float);
  const int nl = (int)c->lv.size();
  M.v.assign(4 * nl, nullptr);
  int64_t grad = 0, trace = 0, ebuf = 0;
  for (int l = 0; l < nl; ++l) {
    const Level &L = c->lv[l];
    for (int k = 0; k < 4; ++k) M.v[4 * l + k] = dalloc<char>(c, (int64_t)(L.ndofs * nv * es));
    const int64_t n3 = (int64_t)L.n * L.n * L.n;
    if (L.kind == 0) {
      grad = std::max(grad, L.ncells * 3 * n3);
      trace = std::max(trace, L.ncells * 12 * (int64_t)L.n * L.n);
    }
    ebuf = std::max(ebuf, L.ncells * n3);
  }
  M.grad[0] = dalloc<double>(c, grad * nv);
  M.trace[0] = dalloc<double>(c, trace * nv);
  M.ebuf[0] = dalloc<double>(c, ebuf * nv);
  if (pi == 1) {
    M.grad[1] = dalloc<float>(c, grad * nv);
    M.trace[1] = dalloc<float>(c, trace * nv);
    M.ebuf[1] = dalloc<float>(c, ebuf * nv);
  }
  const int64_t N = c->lv[c->L].ndofs * nv;
  M.r = dalloc<double>(c, N);
  M.z = dalloc<double>(c, N);
  M.p = dalloc<double>(c, N);
  M.v_ = dalloc<double>(c, N);
  M.d_segs = (Seg *)dalloc<char>(c, (int64_t)(nv * sizeof(Seg)));
  M.sc = dalloc<double>(c, (int64_t)nv * kSegSlots);
  {
    std::vector<void *> al;
    CK(seg_grid_build(std::vector<long>(nv, (long)c->lv[c->L].ndofs), M.sg, al));
    for (void *q : al) c->allocs.push_back(q);
    M.sg_allocs = al;
  }
  M.partials = dalloc<double>(c, (int64_t)M.sg.blocks * 2);
  M.counters = dalloc<unsigned>(c, nv);
  CK(cudaMemset(M.counters, 0, nv * sizeof(unsigned)));
  M.cap = nv;
}

// restores the single-vector work set on every exit
struct MultiScope {
  sipg_ctx *c;
  MultiScope(sipg_ctx *c_, int nv) : c(c_) { c->nv = nv; }
  ~MultiScope() { c->nv = 1; }
};

sipg_status solve_multi_impl(sipg_ctx *c, int nrhs, const double *B, double *X, double rtol, int maxit,
                             sipg_solve_info *infos) {
  ensure_multi(c, nrhs);
  MultiScope scope(c, nrhs);
  auto &M = c->mv;
  const int64_t N = c->lv[c->L].ndofs;
  M.segs.resize(nrhs);
  for (int r = 0; r < nrhs; ++r)
    M.segs[r] = Seg{X + r * N, M.r + r * N, M.p + r * N, M.v_ + r * N, M.z + r * N, B + r * N, (long)N, 1};
  c->use_learned = 0;   // the multi-vector cycle smooths with Chebyshev
  Lockstep K{c->stream, M.segs, M.d_segs, M.sg, M.sc, M.partials, M.counters, c->err};
  return lockstep_fcg(
      K, [&]() { apply_level<double>(c, c->L, X, M.r, 2, nullptr, nullptr, B); },
      [&]() { apply_level<double>(c, c->L, M.p, M.v_, 0); }, [&]() { precondition(c); }, rtol, maxit, infos);
}

template <typename F>
sipg_status bguarded(sipg_batch *B, F &&f) {
  std::string *prev = t_err;
  t_err = B ? &B->err : &g_create_err;
  sipg_status st;
  try {
    st = f();
  } catch (const Fail &e) {
    st = e.st;
  } catch (const std::exception &e) {
    if (t_err) *t_err = e.what();
    st = SIPG_ENOMEM;
  }
  t_err = prev;
  return st;
}

}  // namespace

sipg_status sipg_solve_multi(sipg_ctx *c, int nrhs, const double *B, double *X, double rtol, int maxit,
                             sipg_solve_info *infos) {
  if (!c || !B || !X || !c->solver || nrhs < 1 || nrhs > 4096 || maxit < 0 || !(rtol >= 0)) return SIPG_EINVAL;
  if (nrhs == 1) return sipg_solve(c, B, X, rtol, maxit, 0, infos);
  return guarded(c, [&]() -> sipg_status { return solve_multi_impl(c, nrhs, B, X, rtol, maxit, infos); });
}

sipg_status sipg_operator_apply_multi(sipg_ctx *c, int precision, int nv, const void *U, void *V) {
  if (!c || !U || !V || U == V || nv < 1 || nv > 4096 || (precision != 0 && precision != 1)) return SIPG_EINVAL;
  if (nv == 1) return sipg_operator_apply(c, precision, U, V);
  if (!c->solver) return SIPG_EINVAL;
  return guarded(c, [&]() -> sipg_status {
    ensure_multi(c, nv);
    if (precision == 1 && !c->mv.grad[1]) {   // FP32 scratch of a context whose cycle runs in FP64
      int64_t grad = 0, trace = 0;
      for (const Level &L : c->lv)
        if (L.kind == 0) {
          grad = std::max(grad, L.ncells * 3 * (int64_t)L.n * L.n * L.n);
          trace = std::max(trace, L.ncells * 12 * (int64_t)L.n * L.n);
        }
      c->mv.grad[1] = dalloc<float>(c, grad * c->mv.cap);
      c->mv.trace[1] = dalloc<float>(c, trace * c->mv.cap);
    }
    MultiScope scope(c, nv);
    if (precision == 0)
      apply_level<double>(c, c->L, (const double *)U, (double *)V, 0);
    else
      apply_level<float>(c, c->L, (const float *)U, (float *)V, 0);
    return SIPG_OK;
  });
}

extern "C" {

sipg_status sipg_batch_create(int nprob, const sipg_mesh *meshes, const sipg_params *params, sipg_batch **out) {
  if (!out || nprob < 1 || nprob > 4096 || !meshes || !params) return SIPG_EINVAL;
  *out = nullptr;
  sipg_batch *B = new sipg_batch();
  B->stream = (cudaStream_t)params[0].stream;
  sipg_status st = SIPG_OK;
  bool curved = false;
  for (int p = 0; p < nprob && st == SIPG_OK; ++p) {
    cudaStream_t ps;
    if (cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking) != cudaSuccess) {
      st = SIPG_ECUDA;
      break;
    }
    B->streams.push_back(ps);
    sipg_params prm = params[p];
    prm.stream = ps;
    prm.operator_only = 0;
    if (prm.precision != params[0].precision) {
      g_create_err = "all problems of a batch must use the same precision";
      st = SIPG_EINVAL;
      break;
    }
    if (p > 0 && (meshes[p].deform != 0) != (meshes[0].deform != 0)) {
      g_create_err = "a batch holds either only affine or only curved meshes";
      st = SIPG_EINVAL;
      break;
    }
    curved = meshes[0].deform != 0;
    sipg_ctx *c = nullptr;
    st = sipg_create(&meshes[p], &prm, &c);
    if (st == SIPG_OK && !c->solver) {
      g_create_err = "every batched problem needs a Dirichlet side";
      sipg_destroy(c);
      st = SIPG_EINVAL;
    }
    if (st == SIPG_OK) B->ctx.push_back(c);
  }
  if (st == SIPG_OK)
    st = bguarded(nullptr, [&]() -> sipg_status {
      std::vector<DGArgs<double>> args;
      std::vector<int> ns;
      for (auto *c : B->ctx) {
        args.push_back(dg_args<double>(c, c->lv[c->L]));
        ns.push_back(c->lv[c->L].n);
      }
      CK(batch_plan_build(B->plan, args, ns));
      B->plan.curved = curved;
      B->segs.assign(nprob, Seg{});
      CK(cudaMalloc(&B->d_segs, nprob * sizeof(Seg)));
      CK(cudaMalloc(&B->sc, (size_t)nprob * kSegSlots * sizeof(double)));
      std::vector<long> sizes;
      for (auto *c : B->ctx) sizes.push_back((long)c->lv[c->L].ndofs);
      CK(seg_grid_build(sizes, B->sg, B->sg_allocs));
      CK(cudaMalloc(&B->partials, (size_t)B->sg.blocks * 2 * sizeof(double)));
      CK(cudaMalloc(&B->counters, (size_t)nprob * sizeof(unsigned)));
      CK(cudaMemset(B->counters, 0, (size_t)nprob * sizeof(unsigned)));
      CK(cudaEventCreateWithFlags(&B->ev_start, cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&B->ev_branch, cudaEventDisableTiming));
      B->ev_done.resize(nprob);
      for (auto &e : B->ev_done) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      CK(cudaDeviceSynchronize());
      return SIPG_OK;
    });
  if (st != SIPG_OK) {
    batch_free(B);
    return st;
  }
  *out = B;
  return SIPG_OK;
}

sipg_status sipg_batch_destroy(sipg_batch *B) {
  if (!B) return SIPG_EINVAL;
  batch_free(B);
  return SIPG_OK;
}

const char *sipg_batch_last_error(const sipg_batch *B) { return B ? B->err.c_str() : g_create_err.c_str(); }

sipg_status sipg_batch_context(sipg_batch *B, int i, sipg_ctx **ctx) {
  if (!B || !ctx || i < 0 || i >= (int)B->ctx.size()) return SIPG_EINVAL;
  *ctx = B->ctx[i];
  return SIPG_OK;
}

sipg_status sipg_batch_apply(sipg_batch *B, const double *const *u, double *const *v) {
  if (!B || !u || !v) return SIPG_EINVAL;
  for (size_t p = 0; p < B->ctx.size(); ++p)
    if (!u[p] || !v[p] || u[p] == v[p]) return SIPG_EINVAL;
  return bguarded(B, [&]() -> sipg_status {
    for (size_t p = 0; p < B->ctx.size(); ++p) B->segs[p].active = 1;
    batch_set_plan(B, 0, u, v);
    CK(batch_apply(B->plan, B->stream));
    return SIPG_OK;
  });
}

sipg_status sipg_batch_vcycle(sipg_batch *B, const double *const *r, double *const *z) {
  if (!B || !r || !z) return SIPG_EINVAL;
  for (size_t p = 0; p < B->ctx.size(); ++p)
    if (!r[p] || !z[p]) return SIPG_EINVAL;
  return bguarded(B, [&]() -> sipg_status {
    batch_cycle_prepare(B);
    cudaStream_t s = B->stream;
    for (size_t p = 0; p < B->ctx.size(); ++p) {
      sipg_ctx *c = B->ctx[p];
      B->segs[p] = Seg{nullptr, c->fr, nullptr, nullptr, c->fz, nullptr, (long)c->lv[c->L].ndofs, 1};
      CK(cudaMemcpyAsync(c->fr, r[p], c->lv[c->L].ndofs * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    CK(cudaMemcpyAsync(B->d_segs, B->segs.data(), B->segs.size() * sizeof(Seg), cudaMemcpyHostToDevice, s));
    batch_precondition(B);
    for (size_t p = 0; p < B->ctx.size(); ++p) {
      sipg_ctx *c = B->ctx[p];
      CK(cudaMemcpyAsync(z[p], c->fz, c->lv[c->L].ndofs * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    CK(cudaStreamSynchronize(s));
    return SIPG_OK;
  });
}

sipg_status sipg_batch_solve(sipg_batch *B, const double *const *b, double *const *x, double rtol, int maxit,
                             sipg_solve_info *infos) {
  if (!B || !b || !x || maxit < 0 || !(rtol >= 0)) return SIPG_EINVAL;
  for (size_t p = 0; p < B->ctx.size(); ++p)
    if (!b[p] || !x[p]) return SIPG_EINVAL;
  return bguarded(B, [&]() -> sipg_status { return batch_solve_impl(B, b, x, rtol, maxit, infos); });
}

}  // extern "C"
