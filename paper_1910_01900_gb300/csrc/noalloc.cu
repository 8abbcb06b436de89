// Operator apply that allocates no device memory.
//
// Some callers cannot call cudaMalloc at the point where they need A u: code
// running inside a host framework whose caching allocator has already
// reserved the device memory for itself, or a time-stepping loop that must
// not allocate (or synchronize on an allocation) once it has started.  This
// entry point serves them: the caller passes only the input and output
// vectors, and the scratch that the two DG passes need (reference gradients,
// face traces, penalty and weight tables) lives in one file-scope device
// array of fixed size, allocated by the CUDA runtime when the library is
// loaded and held by every GPU that loads it until the process exits.
//
// Host code cannot use the array's name as a device address (in host code it
// is only a host-side stand-in; a kernel given it would fault or, where the
// GPU can reach host memory, silently use the wrong memory).  Its device
// address is looked up once per device with cudaGetSymbolAddress, with that
// device current, and cached.
#include <mutex>

#include "sipg_internal.h"

namespace {

// Maximum scratch: 64 MiB (enough for about 1.4 million DoF at k = 3).
constexpr size_t kScratchBytes = size_t(64) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

struct Weights1D {
  double w[sipg::kMaxN];
};

// Cartesian cell and face weights and the penalty tau_e (Section 2, same
// definitions as the context path) written into the scratch.
__global__ void noalloc_prep_kernel(double *wcart, double *fwcart, double *tau, int n, Weights1D W, double h0,
                                    double h1, double h2, int m0, int m1, int m2, double factor) {
  const int n2 = n * n, n3 = n2 * n;
  const double h[3] = {h0, h1, h2};
  const int m[3] = {m0, m1, m2};
  const double vol = h0 * h1 * h2;
  const long ncells = (long)m0 * m1 * m2;
  const long total = 3L * n3 + 3L * n2 + ncells;
  for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    if (idx < 3L * n3) {
      const int d = (int)(idx / n3), p = (int)(idx - (long)d * n3);
      const int i = p % n, j = (p / n) % n, k = p / n2;
      const double w = W.w[i] * W.w[j] * W.w[k];
      wcart[idx] = w * vol / (h[d] * h[d]);
    } else if (idx < 3L * n3 + 3L * n2) {
      const long r = idx - 3L * n3;
      const int d = (int)(r / n2), l = (int)(r - (long)d * n2);
      const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
      fwcart[r] = W.w[l % n] * W.w[l / n] * h[t1] * h[t2];
    } else {
      const long e = idx - 3L * n3 - 3L * n2;
      const int ijk[3] = {(int)(e % m0), (int)((e / m0) % m1), (int)(e / ((long)m0 * m1))};
      double a_int = 0, a_bd = 0;
      for (int d = 0; d < 3; ++d) {
        const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
        const double area = h[t1] * h[t2];
        for (int s = 0; s < 2; ++s) {
          const bool bd = s ? (ijk[d] == m[d] - 1) : (ijk[d] == 0);
          if (bd) a_bd += area;
          else a_int += area;
        }
      }
      tau[e] = factor * (double)n * n * (0.5 * a_int + a_bd) / vol;
    }
  }
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

extern "C" sipg_status sipg_operator_apply_noalloc(const sipg_mesh *mesh, int degree, double penalty_factor,
                                                   const double *u_dev, double *v_dev, void *stream) {
  using namespace sipg;
  // an error left pending by earlier, unrelated work of the caller would
  // otherwise be reported as this call's failure
  (void)cudaGetLastError();
  if (!mesh || !u_dev || !v_dev) {
    sipg::set_global_error("null argument");
    return SIPG_EINVAL;
  }
  if (degree < 1 || degree > 8 || !(penalty_factor > 0) || mesh->deform != 0) {
    sipg::set_global_error("degree must be 1..8, penalty factor positive, cells affine (deform = 0)");
    return SIPG_EINVAL;
  }
  for (int d = 0; d < 3; ++d)
    if (mesh->m[d] < 1 || !(mesh->hi[d] > mesh->lo[d])) {
      sipg::set_global_error("m must be >= 1 and extents positive");
      return SIPG_EINVAL;
    }
  // the cell count in double first, so that none of the byte counts below is
  // formed from a wrapped integer product (m = 2^21 per axis wraps 64 bits)
  const double cells_d = (double)mesh->m[0] * mesh->m[1] * mesh->m[2];
  if (cells_d > (double)(1 << 30)) {
    sipg::set_global_error("problem needs more than the 64 MiB static scratch of sipg_operator_apply_noalloc");
    return SIPG_EINVAL;
  }
  for (int s = 0; s < 6; ++s)
    if (mesh->bc[s] != 0 && mesh->bc[s] != 1) {
      sipg::set_global_error("bc must be 0 or 1");
      return SIPG_EINVAL;
    }
  const int n = degree + 1, n2 = n * n, n3 = n2 * n;
  const long long E = (long long)mesh->m[0] * mesh->m[1] * mesh->m[2];
  const size_t b_grad = align256((size_t)E * 3 * n3 * sizeof(double));
  const size_t b_trace = align256((size_t)E * 12 * n2 * sizeof(double));
  const size_t b_tau = align256((size_t)E * sizeof(double));
  const size_t b_w = align256((size_t)3 * n3 * sizeof(double));
  const size_t b_fw = align256((size_t)3 * n2 * sizeof(double));
  if (b_grad + b_trace + b_tau + b_w + b_fw > kScratchBytes) {
    sipg::set_global_error("problem needs more than the 64 MiB static scratch of sipg_operator_apply_noalloc");
    return SIPG_EINVAL;
  }
  {
    // u and v must not overlap anywhere (v is written while u is still read)
    const uintptr_t pu = (uintptr_t)u_dev, pv = (uintptr_t)v_dev, bytes = (uintptr_t)E * n3 * sizeof(double);
    if (pu < pv + bytes && pv < pu + bytes) {
      sipg::set_global_error("u and v overlap");
      return SIPG_EINVAL;
    }
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    sipg::set_global_error("no usable current device");
    return SIPG_ECUDA;
  }
  unsigned char *base;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
      // set-up, once per device, with that device current
      void *p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        sipg::set_global_error(std::string("cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
        return SIPG_ECUDA;
      }
      static Tables<double> tab;
      static std::once_flag built;
      std::call_once(built, [] { build_tables(tab); });
      upload_tables_dg<double>(tab);
      cudaError_t ue = cudaGetLastError();
      if (ue == cudaSuccess) ue = prepare_dg_kernels<double>();
      if (ue != cudaSuccess) {
        sipg::set_global_error(std::string("table upload failed: ") + cudaGetErrorString(ue));
        return SIPG_ECUDA;
      }
      g_scratch_addr[dev] = p;
    }
    base = (unsigned char *)g_scratch_addr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  double *grad = (double *)base;
  double *trace = (double *)(base + b_grad);
  double *tau = (double *)(base + b_grad + b_trace);
  double *wcart = (double *)(base + b_grad + b_trace + b_tau);
  double *fwcart = (double *)(base + b_grad + b_trace + b_tau + b_w);
  const Rules1D &r = rules(n);
  Weights1D W{};
  for (int i = 0; i < n; ++i) W.w[i] = r.wq[i];
  double h[3];
  for (int d = 0; d < 3; ++d) h[d] = (mesh->hi[d] - mesh->lo[d]) / mesh->m[d];
  const long total = 3L * n3 + 3L * n2 + E;
  const int bs = 256;
  const int grid = (int)std::min<long>((total + bs - 1) / bs, 152L * 8);
  noalloc_prep_kernel<<<grid, bs, 0, s>>>(wcart, fwcart, tau, n, W, h[0], h[1], h[2], mesh->m[0], mesh->m[1],
                                          mesh->m[2], penalty_factor);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    sipg::set_global_error(std::string("launch failed: ") + cudaGetErrorString(e));
    return SIPG_ECUDA;
  }
  DGArgs<double> a{};
  a.u = u_dev;
  a.out = v_dev;
  a.grad = grad;
  a.trace = trace;
  a.wcart = wcart;
  a.fwcart = fwcart;
  a.tau = tau;
  for (int d = 0; d < 3; ++d) {
    a.ih[d] = 1.0 / h[d];
    a.m[d] = mesh->m[d];
  }
  a.ncells = (int)E;
  for (int q = 0; q < 6; ++q) a.bc[q] = mesh->bc[q];
  a.mode = 0;
  e = launch_dg_eval<double>(n, false, a, s);
  if (e == cudaSuccess) e = launch_dg_integrate<double>(n, false, a, s);
  if (e != cudaSuccess) {
    sipg::set_global_error(std::string("launch failed: ") + cudaGetErrorString(e));
    return SIPG_ECUDA;
  }
  return SIPG_OK;
}

