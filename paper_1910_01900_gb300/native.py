"""ctypes binding of libsipg (include/sipg.h): argument marshalling only.

Every computation runs in the CUDA library.  Vectors are torch tensors on the
context's device (or numpy arrays for the *_host calls); this module only
passes their pointers and checks their sizes and dtypes.  Loading fails
loudly when the shared library has not been built.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsipg.so")

OK, EINVAL, ECUDA, ENOMEM, ENOTCONV, EBREAKDOWN, ETIMEOUT, ENAN = range(8)
STATUS_NAMES = ["OK", "EINVAL", "ECUDA", "ENOMEM", "ENOTCONV", "EBREAKDOWN", "ETIMEOUT", "ENAN"]

# every entry point the header declares (checked by the CPU test suite)
EXPORTS = [
    "sipg_default_params", "sipg_create", "sipg_create_unstructured", "sipg_destroy", "sipg_last_error", "sipg_num_levels",
    "sipg_num_dofs", "sipg_level_info", "sipg_lambda", "sipg_rhs", "sipg_operator_apply",
    "sipg_level_apply", "sipg_inverse_diagonal", "sipg_smooth", "sipg_restrict", "sipg_prolongate_add",
    "sipg_coarse_solve", "sipg_coarse_info", "sipg_coarse_amg_vcycle", "sipg_vcycle", "sipg_solve", "sipg_solve_host", "sipg_time_apply", "sipg_fma_peak",
    "sipg_operator_apply_noalloc", "sipg_launch_count", "sipg_batch_create", "sipg_batch_destroy",
    "sipg_batch_last_error", "sipg_batch_context", "sipg_batch_apply", "sipg_batch_vcycle", "sipg_batch_solve", "sipg_tile_shape", "sipg_set_tile_shape", "sipg_solve_multi",
    "sipg_operator_apply_multi",
    "sipg_smoother_train", "sipg_smoother_finetune", "sipg_set_smoother", "sipg_mlp_shape", "sipg_mlp_params", "sipg_mlp_forward",
    "sipg_mlp_gradients", "sipg_mlp_features", "sipg_l2_error",
]


class TrainInfo(ctypes.Structure):
    _fields_ = [("npairs", ctypes.c_int), ("epochs", ctypes.c_int), ("steps", ctypes.c_int),
                ("loss_first", ctypes.c_double), ("loss_last", ctypes.c_double), ("out_scale", ctypes.c_double),
                ("cheb_rate", ctypes.c_double), ("seconds", ctypes.c_double), ("target_max", ctypes.c_double),
                ("nonfinite", ctypes.c_double), ("iter_ms_chebyshev", ctypes.c_double),
                ("iter_ms_learned", ctypes.c_double), ("damping", ctypes.c_double),
                ("step_reduction", ctypes.c_double)]


class Mesh(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int * 3), ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("deform", ctypes.c_int), ("amp", ctypes.c_double), ("mapping_degree", ctypes.c_int),
                ("bc", ctypes.c_int * 6)]


class HexMesh(ctypes.Structure):
    _fields_ = [("nverts", ctypes.c_int), ("vertices", ctypes.c_void_p), ("ncells", ctypes.c_int),
                ("cells", ctypes.c_void_p), ("face_bc", ctypes.c_void_p), ("deform", ctypes.c_int),
                ("amp", ctypes.c_double), ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3)]


class Params(ctypes.Structure):
    _fields_ = [("degree", ctypes.c_int), ("penalty_factor", ctypes.c_double), ("precision", ctypes.c_int),
                ("p_coarsen", ctypes.c_int), ("cheb_degree", ctypes.c_int), ("cheb_lo", ctypes.c_double),
                ("cheb_hi", ctypes.c_double), ("eig_iters", ctypes.c_int), ("lambda_override", ctypes.c_double),
                ("smoother", ctypes.c_int), ("operator_only", ctypes.c_int), ("coarsening", ctypes.c_char * 8),
                ("autotune", ctypes.c_int), ("fe_assemble", ctypes.c_int),
                ("coarse_dense_max", ctypes.c_int), ("coarse_iters", ctypes.c_int),
                ("coarse_solver", ctypes.c_int), ("coarse_rtol", ctypes.c_double), ("coarse_maxit", ctypes.c_int),
                ("fuse_tail", ctypes.c_int), ("stream", ctypes.c_void_p)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("r0_norm", ctypes.c_double),
                ("r_norm", ctypes.c_double), ("rho", ctypes.c_double), ("n10", ctypes.c_double),
                ("seconds", ctypes.c_double), ("res_history", ctypes.c_double * 256), ("learned", ctypes.c_int),
                ("fell_back", ctypes.c_int)]


_lib = None


def lib():
    """The loaded libsipg (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libsipg.so is not built: run __graft_entry__.build() "
                               "(python -m paper_1910_01900_gb300.build)")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        L.sipg_default_params.argtypes = [ctypes.POINTER(Params)]
        L.sipg_default_params.restype = None
        L.sipg_create.argtypes = [ctypes.POINTER(Mesh), ctypes.POINTER(Params), ctypes.POINTER(vp)]
        L.sipg_create_unstructured.argtypes = [ctypes.POINTER(HexMesh), ctypes.POINTER(Params), ctypes.POINTER(vp)]
        L.sipg_destroy.argtypes = [vp]
        L.sipg_last_error.argtypes = [vp]
        L.sipg_last_error.restype = ctypes.c_char_p
        L.sipg_num_levels.argtypes = [vp, ctypes.POINTER(i32)]
        L.sipg_num_dofs.argtypes = [vp, i32, ctypes.POINTER(i64)]
        L.sipg_level_info.argtypes = [vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32 * 3)]
        L.sipg_lambda.argtypes = [vp, i32, ctypes.POINTER(dbl)]
        L.sipg_rhs.argtypes = [vp, i32, vp]
        L.sipg_operator_apply.argtypes = [vp, i32, vp, vp]
        L.sipg_level_apply.argtypes = [vp, i32, i32, vp, vp]
        L.sipg_inverse_diagonal.argtypes = [vp, i32, i32, vp]
        L.sipg_smooth.argtypes = [vp, i32, vp, vp, i32]
        L.sipg_restrict.argtypes = [vp, i32, vp, vp]
        L.sipg_prolongate_add.argtypes = [vp, i32, vp, vp]
        L.sipg_coarse_solve.argtypes = [vp, vp, vp]
        L.sipg_coarse_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                       ctypes.POINTER(i32)]
        L.sipg_coarse_amg_vcycle.argtypes = [vp, vp, vp]
        L.sipg_vcycle.argtypes = [vp, vp, vp]
        L.sipg_solve.argtypes = [vp, vp, vp, dbl, i32, i32, ctypes.POINTER(SolveInfo)]
        L.sipg_solve_host.argtypes = [vp, vp, vp, dbl, i32, ctypes.POINTER(SolveInfo)]
        L.sipg_solve_multi.argtypes = [vp, i32, vp, vp, dbl, i32, ctypes.POINTER(SolveInfo)]
        L.sipg_operator_apply_multi.argtypes = [vp, i32, i32, vp, vp]
        L.sipg_time_apply.argtypes = [vp, i32, vp, vp, i32, ctypes.POINTER(ctypes.c_float),
                                      ctypes.POINTER(ctypes.c_float)]
        L.sipg_fma_peak.argtypes = [i32, vp, ctypes.POINTER(dbl)]
        L.sipg_launch_count.argtypes = [ctypes.POINTER(ctypes.c_ulonglong)]
        L.sipg_tile_shape.argtypes = [vp, i32, i32, i32, ctypes.POINTER(i32)]
        L.sipg_set_tile_shape.argtypes = [vp, i32, i32, i32, i32]
        L.sipg_smoother_train.argtypes = [vp, i32, i32, ctypes.c_uint64, ctypes.POINTER(TrainInfo)]
        L.sipg_smoother_finetune.argtypes = [vp, i32, dbl, ctypes.POINTER(TrainInfo)]
        L.sipg_set_smoother.argtypes = [vp, i32, i32, i32]
        ip = ctypes.POINTER(i32)
        L.sipg_mlp_shape.argtypes = [vp, ip, ip, ip, ip, ip, ctypes.POINTER(i64)]
        L.sipg_mlp_params.argtypes = [vp, i32, vp]
        L.sipg_mlp_forward.argtypes = [vp, vp, i32, vp]
        L.sipg_mlp_gradients.argtypes = [vp, vp, vp, i32, vp, ctypes.POINTER(dbl)]
        L.sipg_mlp_features.argtypes = [vp, vp, vp, vp]
        L.sipg_l2_error.argtypes = [vp, i32, vp, ctypes.POINTER(dbl)]
        L.sipg_batch_create.argtypes = [i32, ctypes.POINTER(Mesh), ctypes.POINTER(Params), ctypes.POINTER(vp)]
        L.sipg_batch_destroy.argtypes = [vp]
        L.sipg_batch_last_error.argtypes = [vp]
        L.sipg_batch_last_error.restype = ctypes.c_char_p
        L.sipg_batch_context.argtypes = [vp, i32, ctypes.POINTER(vp)]
        L.sipg_batch_apply.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp)]
        L.sipg_batch_vcycle.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp)]
        L.sipg_batch_solve.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), dbl, i32, ctypes.POINTER(SolveInfo)]
        L.sipg_operator_apply_noalloc.argtypes = [ctypes.POINTER(Mesh), i32, dbl, vp, vp, vp]
        for name in EXPORTS:
            if name not in ("sipg_default_params", "sipg_last_error", "sipg_batch_last_error"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


class SipgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < 8 else status, msg))
        self.status = status


def _ptr(t, dtype=None, numel=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA torch tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError("expected dtype %s, got %s" % (dtype, t.dtype))
    if numel is not None and t.numel() != numel:
        raise ValueError("expected %d elements, got %d" % (numel, t.numel()))
    return ctypes.c_void_p(t.data_ptr())


def make_mesh(m, deform=0, amp=0.1, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), bc=(0,) * 6):
    mesh = Mesh()
    mm = tuple(m) if hasattr(m, "__len__") else (m, m, m)
    for d in range(3):
        mesh.m[d], mesh.lo[d], mesh.hi[d] = int(mm[d]), float(lo[d]), float(hi[d])
    mesh.deform, mesh.amp, mesh.mapping_degree = int(deform), float(amp), 3
    for s in range(6):
        mesh.bc[s] = int(bc[s])
    return mesh, mm


def make_params(degree, precision=0, penalty_factor=1.0, cheb_degree=5, eig_iters=20, lambda_override=0.0,
                operator_only=False, stream=None, autotune=False, p_coarsen=0, coarsening="cph", fe_assemble=None,
                coarse_dense_max=None, coarse_iters=None, coarse_solver=None, coarse_rtol=None, coarse_maxit=None,
                fuse_tail=None):
    prm = Params()
    lib().sipg_default_params(ctypes.byref(prm))
    prm.degree, prm.precision, prm.penalty_factor = int(degree), int(precision), float(penalty_factor)
    prm.cheb_degree, prm.eig_iters = int(cheb_degree), int(eig_iters)
    prm.lambda_override, prm.operator_only = float(lambda_override), int(bool(operator_only))
    prm.autotune = int(bool(autotune))
    prm.p_coarsen = int(p_coarsen)
    prm.coarsening = coarsening.encode()
    if fe_assemble is not None:
        prm.fe_assemble = int(fe_assemble)
    if coarse_dense_max is not None:
        prm.coarse_dense_max = int(coarse_dense_max)
    if coarse_iters is not None:
        prm.coarse_iters = int(coarse_iters)
    if coarse_solver is not None:
        prm.coarse_solver = int(coarse_solver)
    if coarse_rtol is not None:
        prm.coarse_rtol = float(coarse_rtol)
    if coarse_maxit is not None:
        prm.coarse_maxit = int(coarse_maxit)
    if fuse_tail is not None:
        prm.fuse_tail = int(bool(fuse_tail))
    prm.stream = ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)
    return prm


class Context:
    """One SIPG problem: mesh, degree, level hierarchy, device data (sipg_create)."""

    def __init__(self, m, degree, deform=0, amp=0.1, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), bc=(0,) * 6,
                 precision=0, penalty_factor=1.0, cheb_degree=5, eig_iters=20, lambda_override=0.0,
                 operator_only=False, stream=None, autotune=False, p_coarsen=0, coarsening="cph", fe_assemble=None,
                 coarse_dense_max=None, coarse_iters=None, coarse_solver=None, coarse_rtol=None, coarse_maxit=None,
                 fuse_tail=None, _handle=None):
        L = lib()
        mesh, mm = make_mesh(m, deform, amp, lo, hi, bc)
        self.degree, self.precision = int(degree), int(precision)
        self.m = mm
        self.stream = stream
        self._owned = _handle is None
        if _handle is not None:
            self.h = _handle
            return
        prm = make_params(degree, precision, penalty_factor, cheb_degree, eig_iters, lambda_override,
                          operator_only, stream, autotune, p_coarsen, coarsening, fe_assemble,
                          coarse_dense_max, coarse_iters, coarse_solver, coarse_rtol, coarse_maxit, fuse_tail)
        h = ctypes.c_void_p()
        st = L.sipg_create(ctypes.byref(mesh), ctypes.byref(prm), ctypes.byref(h))
        if st != OK:
            raise SipgError(st, L.sipg_last_error(None).decode())
        self.h = h

    def _check(self, st):
        if st != OK:
            raise SipgError(st, lib().sipg_last_error(self.h).decode())

    def close(self):
        if getattr(self, "_owned", False) and getattr(self, "h", None) is not None and self.h.value:
            lib().sipg_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ queries
    @property
    def num_levels(self):
        n = ctypes.c_int()
        self._check(lib().sipg_num_levels(self.h, ctypes.byref(n)))
        return n.value

    def num_dofs(self, level=None):
        level = self.num_levels - 1 if level is None else level
        n = ctypes.c_int64()
        self._check(lib().sipg_num_dofs(self.h, level, ctypes.byref(n)))
        return n.value

    def level_info(self, level):
        kind, deg, m = ctypes.c_int(), ctypes.c_int(), (ctypes.c_int * 3)()
        self._check(lib().sipg_level_info(self.h, level, ctypes.byref(kind), ctypes.byref(deg), ctypes.byref(m)))
        return kind.value, deg.value, tuple(m)

    def lam(self, level):
        v = ctypes.c_double()
        self._check(lib().sipg_lambda(self.h, level, ctypes.byref(v)))
        return v.value

    # ------------------------------------------------------------ hot path
    def rhs(self, b, kind=0):
        import torch
        self._check(lib().sipg_rhs(self.h, kind, _ptr(b, torch.float64, self.num_dofs())))

    def l2_error(self, x, kind=0):
        import torch
        e = ctypes.c_double()
        self._check(lib().sipg_l2_error(self.h, int(kind), _ptr(x, torch.float64, self.num_dofs()),
                                        ctypes.byref(e)))
        return e.value

    def apply(self, u, v, precision=None):
        import torch
        precision = (0 if u.dtype == torch.float64 else 1) if precision is None else precision
        dt = torch.float64 if precision == 0 else torch.float32
        n = self.num_dofs()
        self._check(lib().sipg_operator_apply(self.h, precision, _ptr(u, dt, n), _ptr(v, dt, n)))

    def level_apply(self, level, u, v):
        import torch
        precision = 0 if u.dtype == torch.float64 else 1
        n = self.num_dofs(level)
        self._check(lib().sipg_level_apply(self.h, level, precision, _ptr(u, u.dtype, n), _ptr(v, u.dtype, n)))

    def inverse_diagonal(self, level, d):
        import torch
        precision = 0 if d.dtype == torch.float64 else 1
        self._check(lib().sipg_inverse_diagonal(self.h, level, precision, _ptr(d, d.dtype, self.num_dofs(level))))

    def smooth(self, level, b, x, nsteps):
        n = self.num_dofs(level)
        self._check(lib().sipg_smooth(self.h, level, _ptr(b, x.dtype, n), _ptr(x, x.dtype, n), int(nsteps)))

    def restrict(self, level, r, rc):
        self._check(lib().sipg_restrict(self.h, level, _ptr(r, r.dtype, self.num_dofs(level)),
                                        _ptr(rc, r.dtype, self.num_dofs(level - 1))))

    def prolongate_add(self, level, xc, x):
        self._check(lib().sipg_prolongate_add(self.h, level, _ptr(xc, x.dtype, self.num_dofs(level - 1)),
                                              _ptr(x, x.dtype, self.num_dofs(level))))

    def coarse_solve(self, b, x):
        import torch
        n = self.num_dofs(0)
        self._check(lib().sipg_coarse_solve(self.h, _ptr(b, torch.float64, n), _ptr(x, torch.float64, n)))

    def coarse_info(self):
        """(kind, AMG level sizes, CG iterations of the last coarse solve); kind 0 dense
        inverse, 1 Jacobi-PCG, 2 AMG-CG."""
        kind, nl, it = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        sizes = (ctypes.c_int * 10)()
        self._check(lib().sipg_coarse_info(self.h, ctypes.byref(kind), ctypes.byref(nl), sizes, ctypes.byref(it)))
        return kind.value, [sizes[i] for i in range(min(nl.value, 10))], it.value

    def coarse_amg_vcycle(self, b, x):
        import torch
        n = self.num_dofs(0)
        self._check(lib().sipg_coarse_amg_vcycle(self.h, _ptr(b, torch.float64, n), _ptr(x, torch.float64, n)))

    def vcycle(self, r, z):
        import torch
        n = self.num_dofs()
        self._check(lib().sipg_vcycle(self.h, _ptr(r, torch.float64, n), _ptr(z, torch.float64, n)))

    def solve(self, b, x, rtol=1e-10, maxit=200, fixed_iters=0, allow_notconv=False):
        import torch
        n = self.num_dofs()
        info = SolveInfo()
        st = lib().sipg_solve(self.h, _ptr(b, torch.float64, n), _ptr(x, torch.float64, n), float(rtol),
                              int(maxit), int(fixed_iters), ctypes.byref(info))
        if not (allow_notconv and st == ENOTCONV):
            self._check(st)
        return info

    def solve_multi(self, B, X, rtol=1e-10, maxit=200, allow_notconv=False):
        """Solve for every row of B (shape (nrhs, num_dofs), FP64, device) at once; X holds the
        start vectors and receives the solutions.  Returns one SolveInfo per right-hand side."""
        import torch
        nrhs, n = B.shape
        assert n == self.num_dofs() and tuple(X.shape) == (nrhs, n)
        infos = (SolveInfo * nrhs)()
        st = lib().sipg_solve_multi(self.h, nrhs, _ptr(B, torch.float64, nrhs * n), _ptr(X, torch.float64, nrhs * n),
                                    float(rtol), int(maxit), infos)
        if not (allow_notconv and st == ENOTCONV):
            self._check(st)
        return list(infos)

    def apply_multi(self, U, V):
        """V = A U for every row of U (shape (nv, num_dofs), FP64 or FP32, device)."""
        import torch
        precision = 0 if U.dtype == torch.float64 else 1
        nv, n = U.shape
        assert n == self.num_dofs() and tuple(V.shape) == (nv, n)
        self._check(lib().sipg_operator_apply_multi(self.h, precision, nv, _ptr(U, U.dtype, nv * n),
                                                    _ptr(V, U.dtype, nv * n)))

    def solve_host(self, b_host, x_host, rtol=1e-10, maxit=200):
        import numpy as np
        n = self.num_dofs()
        for a in (b_host, x_host):
            if a.dtype != np.float64 or a.size != n or not a.flags["C_CONTIGUOUS"]:
                raise ValueError("host vectors must be contiguous float64 of length %d" % n)
        info = SolveInfo()
        self._check(lib().sipg_solve_host(self.h, ctypes.c_void_p(b_host.ctypes.data),
                                          ctypes.c_void_p(x_host.ctypes.data), float(rtol), int(maxit),
                                          ctypes.byref(info)))
        return info

    # ------------------------------------------------------ learned smoother
    def train_smoother(self, npairs=100000, epochs=20, seed=2024):
        info = TrainInfo()
        self._check(lib().sipg_smoother_train(self.h, int(npairs), int(epochs), int(seed), ctypes.byref(info)))
        return info

    def finetune_smoother(self, epochs=20, lr=0.0):
        """Energy-norm fine-tuning of the trained network (sipg_smoother_finetune; lr 0: 3e-4)."""
        info = TrainInfo()
        self._check(lib().sipg_smoother_finetune(self.h, int(epochs), float(lr), ctypes.byref(info)))
        return info

    def set_smoother(self, which, steps_pre=0, steps_post=1):
        """0 Chebyshev; 1 learned: steps_pre network pre-steps (0 = Chebyshev pre-smoothing) and
        steps_post network post-steps (0 = no post-smoothing: the cycle without the network)."""
        self._check(lib().sipg_set_smoother(self.h, int(which), int(steps_pre), int(steps_post)))

    def mlp_shape(self):
        v = [ctypes.c_int() for _ in range(5)]
        n = ctypes.c_int64()
        self._check(lib().sipg_mlp_shape(self.h, *[ctypes.byref(x) for x in v], ctypes.byref(n)))
        keys = ("in_dim", "in_pad", "hidden", "out_dim", "out_pad")
        d = {k: x.value for k, x in zip(keys, v)}
        d["nparams"] = n.value
        return d

    def mlp_params(self, values=None):
        import numpy as np
        n = self.mlp_shape()["nparams"]
        if values is None:
            out = np.empty(n, dtype=np.float32)
            self._check(lib().sipg_mlp_params(self.h, 0, ctypes.c_void_p(out.ctypes.data)))
            return out
        a = np.ascontiguousarray(values, dtype=np.float32)
        assert a.size == n
        self._check(lib().sipg_mlp_params(self.h, 1, ctypes.c_void_p(a.ctypes.data)))

    def mlp_forward(self, X, Y):
        import torch
        sh = self.mlp_shape()
        B = X.shape[0]
        self._check(lib().sipg_mlp_forward(self.h, _ptr(X, torch.float32, B * sh["in_dim"]), B,
                                           _ptr(Y, torch.float32, B * sh["out_pad"])))

    def mlp_gradients(self, X, T):
        import numpy as np
        import torch
        sh = self.mlp_shape()
        B = X.shape[0]
        g = np.empty(sh["nparams"], dtype=np.float32)
        loss = ctypes.c_double()
        self._check(lib().sipg_mlp_gradients(self.h, _ptr(X, torch.float32, B * sh["in_dim"]),
                                             _ptr(T, torch.float32, B * sh["out_dim"]), B,
                                             ctypes.c_void_p(g.ctypes.data), ctypes.byref(loss)))
        return g, loss.value

    def mlp_features(self, r, feat, scale):
        import torch
        self._check(lib().sipg_mlp_features(self.h, _ptr(r, torch.float64, self.num_dofs()),
                                            _ptr(feat, torch.float32), _ptr(scale, torch.float32)))

    def tile_shape(self, precision, pass_, level=None):
        """Cells per block of a cell kernel (pass 0/1 DG evaluation/integration, 2 FE cells)."""
        v = ctypes.c_int()
        lvl = self.num_levels - 1 if level is None else int(level)
        self._check(lib().sipg_tile_shape(self.h, lvl, int(precision), int(pass_), ctypes.byref(v)))
        return v.value

    def set_tile_shape(self, precision, pass_, cells_per_block, level=None):
        lvl = self.num_levels - 1 if level is None else int(level)
        self._check(lib().sipg_set_tile_shape(self.h, lvl, int(precision), int(pass_), int(cells_per_block)))

    def time_apply(self, u, v, repeats=20):
        import torch
        precision = 0 if u.dtype == torch.float64 else 1
        te, ti = ctypes.c_float(), ctypes.c_float()
        n = self.num_dofs()
        self._check(lib().sipg_time_apply(self.h, precision, _ptr(u, u.dtype, n), _ptr(v, u.dtype, n),
                                          int(repeats), ctypes.byref(te), ctypes.byref(ti)))
        return te.value, ti.value


def create_unstructured(vertices, cells, degree, face_bc=None, deform=0, amp=0.1, lo=(0.0, 0.0, 0.0),
                        hi=(1.0, 1.0, 1.0), penalty_factor=1.0, stream=None, autotune=False):
    """Operator context on an unstructured hexahedral mesh (sipg_create_unstructured).

    vertices (nv, 3) float64, cells (E, 8) int (local vertex i + 2j + 4k at reference
    corner (i, j, k)), face_bc (E, 6) int or None.  Returns a Context whose apply,
    level_apply(0, ...), time_apply and tile-shape calls work; the solver calls do not.
    """
    import numpy as np
    V = np.ascontiguousarray(vertices, dtype=np.float64)
    C = np.ascontiguousarray(cells, dtype=np.int32)
    if V.ndim != 2 or V.shape[1] != 3 or C.ndim != 2 or C.shape[1] != 8:
        raise ValueError("vertices must be (nv, 3) and cells (E, 8)")
    F = None if face_bc is None else np.ascontiguousarray(face_bc, dtype=np.int32)
    if F is not None and F.shape != (C.shape[0], 6):
        raise ValueError("face_bc must be (E, 6)")
    hm = HexMesh()
    hm.nverts, hm.vertices = V.shape[0], V.ctypes.data
    hm.ncells, hm.cells = C.shape[0], C.ctypes.data
    hm.face_bc = F.ctypes.data if F is not None else None
    hm.deform, hm.amp = int(deform), float(amp)
    for d in range(3):
        hm.lo[d], hm.hi[d] = float(lo[d]), float(hi[d])
    prm = make_params(degree, 0, penalty_factor, operator_only=True, stream=stream, autotune=autotune)
    h = ctypes.c_void_p()
    st = lib().sipg_create_unstructured(ctypes.byref(hm), ctypes.byref(prm), ctypes.byref(h))
    if st != OK:
        raise SipgError(st, lib().sipg_last_error(None).decode())
    ctx = Context(1, degree, stream=stream, _handle=h)
    ctx._owned = True
    return ctx


def operator_apply_noalloc(m, degree, u, v, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), bc=(0,) * 6,
                           penalty_factor=1.0, stream=None):
    """v = A u (FP64, affine cells) through sipg_operator_apply_noalloc.

    For callers that cannot allocate device memory when they need A u: the
    library uses its static 64 MiB device scratch instead of allocating.
    Calls that overlap on the GPU race (they share that scratch).
    """
    import torch
    mesh = Mesh()
    mm = tuple(m) if hasattr(m, "__len__") else (m, m, m)
    for d in range(3):
        mesh.m[d], mesh.lo[d], mesh.hi[d] = int(mm[d]), float(lo[d]), float(hi[d])
    mesh.deform, mesh.amp, mesh.mapping_degree = 0, 0.0, 3
    for s in range(6):
        mesh.bc[s] = int(bc[s])
    n = mm[0] * mm[1] * mm[2] * (int(degree) + 1) ** 3
    pu, pv = u.data_ptr(), v.data_ptr()
    if pu < pv + 8 * n and pv < pu + 8 * n:
        raise ValueError("u and v overlap")
    st = lib().sipg_operator_apply_noalloc(ctypes.byref(mesh), int(degree), float(penalty_factor),
                                           _ptr(u, torch.float64, n), _ptr(v, torch.float64, n),
                                           ctypes.c_void_p(stream.cuda_stream if stream is not None else 0))
    if st != OK:
        raise SipgError(st, lib().sipg_last_error(None).decode())


class Batch:
    """Many independent problems solved together (sipg_batch_*).

    problems: list of dicts with keys m, k and optionally deform, bc, lo, hi.
    """

    def __init__(self, problems, precision=0, stream=None, **kw):
        L = lib()
        n = len(problems)
        meshes = (Mesh * n)()
        prms = (Params * n)()
        for i, p in enumerate(problems):
            meshes[i], _ = make_mesh(p["m"], p.get("deform", 0), p.get("amp", 0.1), p.get("lo", (0.0,) * 3),
                                     p.get("hi", (1.0,) * 3), p.get("bc", (0,) * 6))
            prms[i] = make_params(p["k"], precision, stream=stream, **kw)
        h = ctypes.c_void_p()
        st = L.sipg_batch_create(n, meshes, prms, ctypes.byref(h))
        if st != OK:
            raise SipgError(st, L.sipg_batch_last_error(None).decode())
        self.h, self.n, self.stream = h, n, stream
        self.contexts = []
        for i, p in enumerate(problems):
            c = ctypes.c_void_p()
            L.sipg_batch_context(h, i, ctypes.byref(c))
            self.contexts.append(Context(p["m"], p["k"], deform=p.get("deform", 0), precision=precision,
                                         stream=stream, _handle=c))

    def _check(self, st):
        if st != OK:
            raise SipgError(st, lib().sipg_batch_last_error(self.h).decode())

    def num_dofs(self, i):
        return self.contexts[i].num_dofs()

    def apply(self, us, vs):
        import torch
        U = (ctypes.c_void_p * self.n)(*[_ptr(u, torch.float64, self.num_dofs(i)).value for i, u in enumerate(us)])
        V = (ctypes.c_void_p * self.n)(*[_ptr(v, torch.float64, self.num_dofs(i)).value for i, v in enumerate(vs)])
        self._check(lib().sipg_batch_apply(self.h, U, V))

    def vcycle(self, rs, zs):
        """zs[i] = M_i^-1 rs[i]: one V-cycle of every problem (FP64 device vectors)."""
        import torch
        R = (ctypes.c_void_p * self.n)(*[_ptr(r, torch.float64, self.num_dofs(i)).value for i, r in enumerate(rs)])
        Z = (ctypes.c_void_p * self.n)(*[_ptr(z, torch.float64, self.num_dofs(i)).value for i, z in enumerate(zs)])
        self._check(lib().sipg_batch_vcycle(self.h, R, Z))

    def solve(self, bs, xs, rtol=1e-10, maxit=200, allow_notconv=False):
        import torch
        B = (ctypes.c_void_p * self.n)(*[_ptr(b, torch.float64, self.num_dofs(i)).value for i, b in enumerate(bs)])
        X = (ctypes.c_void_p * self.n)(*[_ptr(x, torch.float64, self.num_dofs(i)).value for i, x in enumerate(xs)])
        infos = (SolveInfo * self.n)()
        st = lib().sipg_batch_solve(self.h, B, X, float(rtol), int(maxit), infos)
        if not (allow_notconv and st == ENOTCONV):
            self._check(st)
        return list(infos)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().sipg_batch_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def launch_count():
    """Kernel and graph launches issued by libsipg so far in this process."""
    n = ctypes.c_ulonglong()
    lib().sipg_launch_count(ctypes.byref(n))
    return n.value


def fma_peak(precision, stream=None):
    v = ctypes.c_double()
    st = lib().sipg_fma_peak(int(precision), ctypes.c_void_p(stream.cuda_stream if stream else 0), ctypes.byref(v))
    if st != OK:
        raise SipgError(st, "fma peak probe failed")
    return v.value
