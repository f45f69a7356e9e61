"""Thin ctypes binding of the C ABI in ``include/aao.h``.

Argument marshalling only: every step of the solver runs in ``libaao.so``
(hand-written sm_103a kernels).  Device buffers are passed as torch CUDA
tensors (float64, contiguous, shape (Nt, M)); the binding checks shapes and
dtypes and forwards raw pointers and the current torch stream.  There is no
CPU fallback: if the library is missing, loading raises.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libaao.so")

AAO_OK, AAO_EINVAL, AAO_ENOMEM, AAO_ECUDA, AAO_ENOCONV, AAO_EBREAKDOWN, AAO_ENONFINITE = range(7)
AAO_PREC_FP64, AAO_PREC_MIXED = 0, 1
AAO_INNER_STRANG, AAO_INNER_TAU, AAO_INNER_TAU_DIRECT = 0, 1, 2
AAO_MATVEC_FFT64, AAO_MATVEC_NTT = 0, 1
AAO_COCG_TMEM = -1  # aao_opts.cocg_threads: the Step (b) kernel with its vectors in tensor memory
STATUS_NAMES = {0: "AAO_OK", 1: "AAO_EINVAL", 2: "AAO_ENOMEM", 3: "AAO_ECUDA", 4: "AAO_ENOCONV",
                5: "AAO_EBREAKDOWN", 6: "AAO_ENONFINITE"}

# Every symbol the header declares (checked by the CPU test suite).
EXPORTED = ("aao_default_opts", "aao_setup_coeffs", "aao_plan_create", "aao_plan_destroy",
            "aao_plan_workspace_bytes", "aao_build_rhs", "aao_matvec", "aao_bc_precond_apply",
            "aao_gmres_solve", "aao_gmres_solve_host", "aao_plan_set_profiling", "aao_plan_get_profile",
            "aao_bc_precond_apply_noalloc", "aao_solve_batched", "aao_last_error",
            "aao_fno_num_params", "aao_fno_create", "aao_fno_destroy", "aao_fno_set_params",
            "aao_fno_get_params", "aao_fno_save", "aao_fno_load", "aao_fno_predict", "aao_fno_loss_grad",
            "aao_fno_train_step", "aao_fno_train", "aao_plan_set_warm_start", "aao_plan_record_pairs",
            "aao_plan_recorded_pairs", "aao_plan_get_tuning", "aao_bicgstab_solve", "aao_solve_windows",
            "aao_plan_get_inner_record")
STAGES = ("matvec", "tdft_fwd", "cocg", "tdft_inv", "vector", "fno")


class AaoProblem(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("M", ctypes.c_int64), ("Nt", ctypes.c_int64), ("T", ctypes.c_double),
                ("alpha", ctypes.c_double), ("kappa", ctypes.c_double), ("eps", ctypes.c_double),
                ("My", ctypes.c_int64), ("alpha_y", ctypes.c_double), ("kappa_y", ctypes.c_double)]


class AaoOpts(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int), ("max_cycles", ctypes.c_int), ("tol", ctypes.c_double),
                ("inner_tol", ctypes.c_double), ("inner_maxit", ctypes.c_int), ("prec", ctypes.c_int),
                ("inner", ctypes.c_int), ("use_graphs", ctypes.c_int), ("matvec", ctypes.c_int),
                ("cocg_threads", ctypes.c_int), ("poly_m", ctypes.c_int)]


class AaoInfo(ctypes.Structure):
    _fields_ = [("outer_iters", ctypes.c_int), ("cycles", ctypes.c_int), ("inner_iters_max", ctypes.c_int),
                ("matvecs", ctypes.c_int), ("true_rel_res", ctypes.c_double), ("status_detail", ctypes.c_int),
                ("inner_iters_sum", ctypes.c_int64), ("warm_accepted", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class AaoError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


_lib = None


def load():
    """Loads libaao.so (built by ``__graft_entry__.build()``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libaao.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    vp, i64, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
    lib.aao_default_opts.argtypes = [ctypes.POINTER(AaoOpts), ctypes.c_int]
    lib.aao_default_opts.restype = None
    lib.aao_setup_coeffs.argtypes = [dbl, i64, vp]
    lib.aao_plan_create.argtypes = [ctypes.POINTER(AaoProblem), ctypes.POINTER(AaoOpts), vp,
                                    ctypes.POINTER(vp)]
    lib.aao_plan_destroy.argtypes = [vp]
    lib.aao_plan_workspace_bytes.argtypes = [vp]
    lib.aao_plan_workspace_bytes.restype = ctypes.c_size_t
    lib.aao_build_rhs.argtypes = [vp, vp, vp, vp]
    lib.aao_matvec.argtypes = [vp, vp, vp]
    lib.aao_bc_precond_apply.argtypes = [vp, vp, vp]
    lib.aao_gmres_solve.argtypes = [vp, vp, vp, ctypes.POINTER(AaoInfo)]
    lib.aao_gmres_solve_host.argtypes = [vp, vp, vp, ctypes.POINTER(AaoInfo)]
    lib.aao_bicgstab_solve.argtypes = [vp, vp, vp, ctypes.POINTER(AaoInfo)]
    lib.aao_solve_windows.argtypes = [vp, ctypes.c_int, vp, vp, vp, ctypes.POINTER(AaoInfo)]
    lib.aao_plan_set_profiling.argtypes = [vp, ctypes.c_int]
    lib.aao_plan_get_profile.argtypes = [vp, vp, vp, ctypes.c_int]
    lib.aao_solve_batched.argtypes = [ctypes.c_int, vp, vp, vp, vp, ctypes.c_int]
    lib.aao_bc_precond_apply_noalloc.argtypes = [ctypes.POINTER(AaoProblem), ctypes.POINTER(AaoOpts), vp, vp, vp]
    lib.aao_last_error.argtypes = [vp]
    lib.aao_last_error.restype = ctypes.c_char_p
    lib.aao_fno_num_params.argtypes = []
    lib.aao_fno_num_params.restype = i64
    lib.aao_fno_create.argtypes = [i64, ctypes.c_int, ctypes.c_uint64, ctypes.POINTER(vp)]
    lib.aao_fno_destroy.argtypes = [vp]
    lib.aao_fno_set_params.argtypes = [vp, vp]
    lib.aao_fno_get_params.argtypes = [vp, vp, ctypes.c_int]
    lib.aao_fno_save.argtypes = [vp, ctypes.c_char_p]
    lib.aao_fno_load.argtypes = [vp, ctypes.c_char_p]
    lib.aao_fno_predict.argtypes = [vp, ctypes.c_int, vp, vp, vp, vp, vp]
    lib.aao_fno_loss_grad.argtypes = [vp, ctypes.c_int, vp, vp, vp, vp, ctypes.POINTER(dbl), vp, vp]
    lib.aao_fno_train_step.argtypes = [vp, ctypes.c_int, vp, vp, vp, vp, ctypes.c_float, ctypes.POINTER(dbl), vp]
    lib.aao_fno_train.argtypes = [vp, i64, vp, vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                                  ctypes.c_uint64, vp, vp]
    lib.aao_plan_set_warm_start.argtypes = [vp, vp]
    lib.aao_plan_record_pairs.argtypes = [vp, i64, vp, vp, vp]
    lib.aao_plan_recorded_pairs.argtypes = [vp, ctypes.POINTER(i64)]
    lib.aao_plan_get_tuning.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    lib.aao_plan_get_inner_record.argtypes = [vp, ctypes.c_int, vp, vp]
    for name in EXPORTED:
        if name not in ("aao_default_opts", "aao_plan_workspace_bytes", "aao_last_error", "aao_fno_num_params"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(status, plan_handle=None):
    if status != AAO_OK:
        msg = load().aao_last_error(plan_handle)
        raise AaoError(status, msg.decode() if msg else "")


def aao_setup_coeffs(alpha, n):
    """g_0 .. g_{n-1} (Eq. 2.4) computed by the library on the host, FP64."""
    g = np.empty(int(n), dtype=np.float64)
    _check(load().aao_setup_coeffs(float(alpha), int(n), g.ctypes.data_as(ctypes.c_void_p)))
    return g


def default_opts(prec=AAO_PREC_MIXED, **kw):
    o = AaoOpts()
    load().aao_default_opts(ctypes.byref(o), int(prec))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Plan:
    """An ``aao_plan``: one 1D problem with its device workspace."""

    def __init__(self, M, Nt, alpha, kappa=1.0, T=1.0, eps=0.0, opts=None, stream=None, My=None, alpha_y=None,
                 kappa_y=None, **opt_kw):
        """1D: M interior points.  2D (My given): M x My interior points, x fastest; alpha_y and kappa_y
        default to alpha and kappa."""
        lib = load()
        self.M, self.Nt = int(M), int(Nt)
        dim = 1 if My is None else 2
        self.My = 1 if My is None else int(My)
        self.problem = AaoProblem(dim, self.M, self.Nt, float(T), float(alpha), float(kappa), float(eps),
                                  self.My if dim == 2 else 0, float(alpha if alpha_y is None else alpha_y),
                                  float(kappa if kappa_y is None else kappa_y))
        self.opts = opts if opts is not None else default_opts(**opt_kw)
        self._stream = stream
        h = ctypes.c_void_p()
        _check(lib.aao_plan_create(ctypes.byref(self.problem), ctypes.byref(self.opts),
                                   _stream_ptr(stream), ctypes.byref(h)))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            load().aao_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def workspace_bytes(self):
        return load().aao_plan_workspace_bytes(self.handle)

    @property
    def cocg_threads(self):
        """CTA size of the Step (b) kernel chosen at plan creation (0: shared-memory kernel)."""
        v = ctypes.c_int()
        _check(load().aao_plan_get_tuning(self.handle, ctypes.byref(v)), self.handle)
        return v.value

    def inner_record(self):
        """(iterations, flags) of each shifted system in the most recent Step (b), as int32 arrays of
        Nt/2 + 1 entries (flags: 0 converged, 1 cap, 2 breakdown, 3 non-finite, + 4 warm start accepted)."""
        n = self.Nt // 2 + 1
        it = np.zeros(n, dtype=np.int32)
        fl = np.zeros(n, dtype=np.int32)
        _check(load().aao_plan_get_inner_record(self.handle, n, it.ctypes.data_as(ctypes.c_void_p),
                                                fl.ctypes.data_as(ctypes.c_void_p)), self.handle)
        return it, fl

    def _vec(self, t, name):
        if not (t.is_cuda and t.dtype.is_floating_point and t.element_size() == 8 and t.is_contiguous()):
            raise ValueError("%s must be a contiguous float64 CUDA tensor" % name)
        if t.numel() != self.M * self.My * self.Nt:
            raise ValueError("%s must have Nt*M*My = %d elements" % (name, self.M * self.My * self.Nt))
        return ctypes.c_void_p(t.data_ptr())

    def set_profiling(self, on=True):
        """Bracket every kernel launch with CUDA events on the plan's stream."""
        _check(load().aao_plan_set_profiling(self.handle, int(bool(on))), self.handle)

    def get_profile(self, reset=True):
        """{stage: (milliseconds, kernel launches)} accumulated since the last reset."""
        ms = np.zeros(len(STAGES))
        ln = np.zeros(len(STAGES), dtype=np.int64)
        _check(load().aao_plan_get_profile(self.handle, ms.ctypes.data_as(ctypes.c_void_p),
                                           ln.ctypes.data_as(ctypes.c_void_p), int(bool(reset))), self.handle)
        return {s: (float(ms[i]), int(ln[i])) for i, s in enumerate(STAGES)}

    def build_rhs(self, u0, f, F):
        if not (u0.is_cuda and u0.numel() == self.M * self.My):
            raise ValueError("u0 must be a CUDA tensor of M*My elements")
        _check(load().aao_build_rhs(self.handle, ctypes.c_void_p(u0.data_ptr()), self._vec(f, "f"),
                                    self._vec(F, "F")), self.handle)

    def matvec(self, v, w):
        _check(load().aao_matvec(self.handle, self._vec(v, "v"), self._vec(w, "w")), self.handle)

    def bc_precond_apply(self, v, z):
        _check(load().aao_bc_precond_apply(self.handle, self._vec(v, "v"), self._vec(z, "z")), self.handle)

    def gmres_solve(self, F, U, raise_on_noconv=True):
        info = AaoInfo()
        st = load().aao_gmres_solve(self.handle, self._vec(F, "F"), self._vec(U, "U"), ctypes.byref(info))
        if st != AAO_OK and (raise_on_noconv or st != AAO_ENOCONV):
            _check(st, self.handle)
        return info.as_dict()

    def bicgstab_solve(self, F, U, raise_on_noconv=True):
        """aao_bicgstab_solve: left-preconditioned BiCGSTAB; U is the initial guess on entry."""
        info = AaoInfo()
        st = load().aao_bicgstab_solve(self.handle, self._vec(F, "F"), self._vec(U, "U"), ctypes.byref(info))
        if st != AAO_OK and (raise_on_noconv or st != AAO_ENOCONV):
            _check(st, self.handle)
        return info.as_dict()

    def solve_windows(self, u0, f, U):
        """aao_solve_windows: f and U hold n_windows * Nt time levels (shape (n_windows * Nt, ...))."""
        n = self.M * self.My * self.Nt
        for t, name in ((f, "f"), (U, "U")):
            if not (t.is_cuda and t.dtype.is_floating_point and t.element_size() == 8 and t.is_contiguous()
                    and t.numel() % n == 0 and t.numel() > 0):
                raise ValueError("%s must be a contiguous float64 CUDA tensor of n_windows * Nt * M elements" % name)
        if f.numel() != U.numel() or not (u0.is_cuda and u0.numel() == self.M * self.My):
            raise ValueError("f and U must match and u0 must hold one time level")
        info = AaoInfo()
        _check(load().aao_solve_windows(self.handle, f.numel() // n, ctypes.c_void_p(u0.data_ptr()),
                                        ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(U.data_ptr()),
                                        ctypes.byref(info)), self.handle)
        return info.as_dict()

    def gmres_solve_host(self, F_host, U_host, raise_on_noconv=True):
        """F_host, U_host: float64 host arrays/tensors of Nt*M elements (pinned preferred)."""
        def ptr(a, name):
            n = self.M * self.My * self.Nt
            if hasattr(a, "data_ptr"):  # torch tensor
                if a.is_cuda or a.element_size() != 8 or not a.is_contiguous() or a.numel() != n:
                    raise ValueError("%s must be a contiguous float64 host tensor of Nt*M elements" % name)
                return ctypes.c_void_p(a.data_ptr())
            if a.dtype != np.float64 or not a.flags.c_contiguous or a.size != n:
                raise ValueError("%s must be a contiguous float64 array of Nt*M elements" % name)
            return a.ctypes.data_as(ctypes.c_void_p)
        info = AaoInfo()
        st = load().aao_gmres_solve_host(self.handle, ptr(F_host, "F_host"), ptr(U_host, "U_host"),
                                         ctypes.byref(info))
        if st != AAO_OK and (raise_on_noconv or st != AAO_ENOCONV):
            _check(st, self.handle)
        return info.as_dict()

    def set_warm_start(self, fno):
        """Attach a learned warm-start model (an :class:`Fno`), or detach it with None."""
        _check(load().aao_plan_set_warm_start(self.handle, None if fno is None else fno.handle), self.handle)
        self._fno = fno  # keep the model alive while attached

    def record_pairs(self, b, x, lam):
        """Record (rhs, solution, lambda) of every later shifted solve into b, x (complex64 CUDA tensors
        [capacity, M]) and lam (complex128 [capacity]); None stops recording."""
        lib = load()
        if b is None:
            _check(lib.aao_plan_record_pairs(self.handle, 0, None, None, None), self.handle)
            self._rec = None
            return
        cap = b.shape[0]
        for t, dt, shape in ((b, "complex64", (cap, self.M)), (x, "complex64", (cap, self.M)),
                             (lam, "complex128", (cap,))):
            if not (t.is_cuda and t.is_contiguous() and str(t.dtype).endswith(dt) and tuple(t.shape) == shape):
                raise ValueError("record buffers: b, x complex64 [capacity, M], lam complex128 [capacity]")
        _check(lib.aao_plan_record_pairs(self.handle, cap, ctypes.c_void_p(b.data_ptr()),
                                         ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(lam.data_ptr())),
               self.handle)
        self._rec = (b, x, lam)

    def recorded_pairs(self):
        n = ctypes.c_int64()
        _check(load().aao_plan_recorded_pairs(self.handle, ctypes.byref(n)), self.handle)
        return n.value


def fno_num_params():
    return load().aao_fno_num_params()


class Fno:
    """An ``aao_fno``: the learned warm start (Fourier neural operator) for grid size M."""

    def __init__(self, M, max_batch, seed=0):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.aao_fno_create(int(M), int(max_batch), int(seed), ctypes.byref(h)))
        self.handle, self.M, self.max_batch = h, int(M), int(max_batch)

    def close(self):
        if getattr(self, "handle", None):
            load().aao_fno_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_params(self, theta):
        a = np.ascontiguousarray(theta, dtype=np.float32)
        if a.size != fno_num_params():
            raise ValueError("need %d parameters" % fno_num_params())
        _check(load().aao_fno_set_params(self.handle, a.ctypes.data_as(ctypes.c_void_p)))

    def get_params(self, bf16_rounded=False):
        a = np.empty(fno_num_params(), dtype=np.float32)
        _check(load().aao_fno_get_params(self.handle, a.ctypes.data_as(ctypes.c_void_p), int(bool(bf16_rounded))))
        return a

    def save(self, path):
        _check(load().aao_fno_save(self.handle, os.fsencode(path)))

    def load(self, path):
        _check(load().aao_fno_load(self.handle, os.fsencode(path)))

    def _args(self, b, lam, alpha):
        B = b.shape[0]
        if not (b.is_cuda and b.is_contiguous() and str(b.dtype).endswith("complex64") and tuple(b.shape) == (B, self.M)):
            raise ValueError("b must be a contiguous complex64 CUDA tensor [B, M]")
        if not (lam.is_cuda and lam.is_contiguous() and str(lam.dtype).endswith("complex128") and lam.numel() == B):
            raise ValueError("lam must be a contiguous complex128 CUDA tensor [B]")
        if not (alpha.is_cuda and alpha.is_contiguous() and str(alpha.dtype).endswith("float32") and alpha.numel() == B):
            raise ValueError("alpha must be a contiguous float32 CUDA tensor [B]")
        return B, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(lam.data_ptr()), ctypes.c_void_p(alpha.data_ptr())

    def predict(self, b, lam, alpha, x0, stream=None):
        B, pb, pl, pa = self._args(b, lam, alpha)
        if not (x0.is_cuda and x0.is_contiguous() and x0.shape == b.shape and x0.dtype == b.dtype):
            raise ValueError("x0 must be like b")
        _check(load().aao_fno_predict(self.handle, B, pb, pl, pa, ctypes.c_void_p(x0.data_ptr()), _stream_ptr(stream)))

    def loss_grad(self, b, lam, alpha, x, want_grad=True, stream=None):
        B, pb, pl, pa = self._args(b, lam, alpha)
        if not (x.is_cuda and x.is_contiguous() and x.shape == b.shape and x.dtype == b.dtype):
            raise ValueError("x must be like b")
        loss = ctypes.c_double()
        g = np.empty(fno_num_params(), dtype=np.float32) if want_grad else None
        _check(load().aao_fno_loss_grad(self.handle, B, pb, pl, pa, ctypes.c_void_p(x.data_ptr()), ctypes.byref(loss),
                                        None if g is None else g.ctypes.data_as(ctypes.c_void_p), _stream_ptr(stream)))
        return loss.value, g

    def train_step(self, b, lam, alpha, x, lr=1e-3, stream=None):
        B, pb, pl, pa = self._args(b, lam, alpha)
        if not (x.is_cuda and x.is_contiguous() and x.shape == b.shape and x.dtype == b.dtype):
            raise ValueError("x must be like b")
        loss = ctypes.c_double()
        _check(load().aao_fno_train_step(self.handle, B, pb, pl, pa, ctypes.c_void_p(x.data_ptr()), float(lr),
                                         ctypes.byref(loss), _stream_ptr(stream)))
        return loss.value


    def train(self, b, lam, alpha, x, steps, batch=128, lr0=2e-3, seed=0, stream=None):
        """aao_fno_train over all pairs in b, lam, alpha, x; returns the per-step batch losses."""
        n, pb, pl, pa = self._args(b, lam, alpha)
        if not (x.is_cuda and x.is_contiguous() and x.shape == b.shape and x.dtype == b.dtype):
            raise ValueError("x must be like b")
        losses = np.zeros(int(steps), dtype=np.float64)
        _check(load().aao_fno_train(self.handle, n, pb, pl, pa, ctypes.c_void_p(x.data_ptr()), int(steps), int(batch),
                                    float(lr0), int(seed), losses.ctypes.data_as(ctypes.c_void_p),
                                    _stream_ptr(stream)))
        return losses


def solve_batched(plans, Fs, Us, max_workers=0, raise_on_error=True):
    """aao_solve_batched: all problems at once; returns the list of info dicts.  max_workers <= 0: lockstep
    restart cycles with one Step (b) launch per Arnoldi step for all instances (when the plans allow it);
    max_workers > 0: one stream per instance driven by that many host threads."""
    n = len(plans)
    P = (ctypes.c_void_p * n)(*[p.handle.value for p in plans])
    Fp = (ctypes.c_void_p * n)(*[F.data_ptr() for F in Fs])
    Up = (ctypes.c_void_p * n)(*[U.data_ptr() for U in Us])
    for p, F, U in zip(plans, Fs, Us):
        p._vec(F, "F")
        p._vec(U, "U")
    infos = (AaoInfo * n)()
    st = load().aao_solve_batched(n, P, Fp, Up, infos, int(max_workers))
    if st != AAO_OK and raise_on_error:
        _check(st, None)
    return [i.as_dict() for i in infos]


# Module-level aliases with the C names, for callers that prefer them.
def aao_plan_create(M, Nt, alpha, **kw):
    return Plan(M, Nt, alpha, **kw)


def aao_plan_destroy(plan):
    plan.close()


def aao_build_rhs(plan, u0, f, F):
    plan.build_rhs(u0, f, F)


def aao_matvec(plan, v, w):
    plan.matvec(v, w)


def aao_bc_precond_apply(plan, v, z):
    plan.bc_precond_apply(v, z)


def aao_gmres_solve(plan, F, U):
    return plan.gmres_solve(F, U)


def aao_gmres_solve_host(plan, F_host, U_host):
    return plan.gmres_solve_host(F_host, U_host)
