"""Python binding of libst.so (the C ABI in include/st.h).

Argument marshalling only: every step runs in the library's CUDA kernels.
Vectors are torch CUDA tensors (contiguous, float64 or float32); their device
pointers and the current torch CUDA stream are handed to the library.  There
is no CPU path: if the library or a CUDA device is missing, calls raise.
"""
import ctypes
import os

from . import build as _build

ST_OK, ST_EINVAL, ST_ECUDA, ST_ENOMEM, ST_NOT_CONVERGED, ST_LINESEARCH_FAILED, ST_SINGULAR_PATCH, \
    ST_DEVICE_TIMEOUT = range(8)
ST_PIC, ST_EXN, ST_MODN = 0, 1, 2
ST_FP64, ST_FP32 = 0, 1
TANGENTS = {"pic": ST_PIC, "exn": ST_EXN, "modn": ST_MODN}
STATUS = {0: "ST_OK", 1: "ST_EINVAL", 2: "ST_ECUDA", 3: "ST_ENOMEM", 4: "ST_NOT_CONVERGED",
          5: "ST_LINESEARCH_FAILED", 6: "ST_SINGULAR_PATCH", 7: "ST_DEVICE_TIMEOUT"}

EXPORTED = ["st_setup_mesh", "st_destroy", "st_num_dofs", "st_residual", "st_linearize", "st_jacobian_apply",
            "st_mnorm", "st_precond_setup", "st_vanka_smooth", "st_vcycle", "st_newton_step", "st_last_error",
            "st_mnorm_noalloc", "st_fgmres_solve", "st_batch_setup", "st_batch_destroy", "st_batch_num_dofs", "st_batch_linearize",
            "st_batch_jacobian_apply", "st_batch_residual", "st_batch_newton_step", "st_batch_last_error",
            "st_autotune_report", "st_batch_fgmres_solve"]


class StParams(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("Lx", ctypes.c_double), ("Ly", ctypes.c_double), ("Lz", ctypes.c_double),
                ("k", ctypes.c_int), ("t0", ctypes.c_double), ("dt", ctypes.c_double),
                ("p", ctypes.c_double), ("delta", ctypes.c_double), ("nu", ctypes.c_double),
                ("nu_inf", ctypes.c_double), ("sigma_max", ctypes.c_double),
                ("gamma1", ctypes.c_double), ("gamma2", ctypes.c_double),
                ("dirichlet_mask", ctypes.c_uint), ("inflow_profile", ctypes.c_int),
                ("vbar", ctypes.c_double), ("q_sign", ctypes.c_double),
                ("levels", ctypes.c_int), ("pre_smooth", ctypes.c_int), ("post_smooth", ctypes.c_int),
                ("omega", ctypes.c_double), ("rho_refresh", ctypes.c_double),
                ("fgmres_restart", ctypes.c_int), ("fgmres_maxit", ctypes.c_int), ("newton_maxit", ctypes.c_int),
                ("tol_abs", ctypes.c_double), ("tol_rel", ctypes.c_double), ("lin_rtol", ctypes.c_double),
                ("ew_gamma", ctypes.c_double), ("ew_alpha", ctypes.c_double), ("ew_max", ctypes.c_double),
                ("armijo_c", ctypes.c_double), ("lambda_min", ctypes.c_double),
                ("coarse_sweeps", ctypes.c_int), ("gamma_cip", ctypes.c_double), ("finest_patches", ctypes.c_int),
                ("coarse_solve", ctypes.c_int), ("pressure_space", ctypes.c_int),
                ("smoother", ctypes.c_int), ("patch_type", ctypes.c_int), ("omega_coarse", ctypes.c_double)]


class StNewtonInfo(ctypes.Structure):
    _fields_ = [("newton_iters", ctypes.c_int), ("fgmres_iters_total", ctypes.c_int),
                ("fgmres_iters_last", ctypes.c_int), ("patch_rebuilds", ctypes.c_int),
                ("lambda_last", ctypes.c_double), ("res_norm_initial", ctypes.c_double),
                ("res_norm_final", ctypes.c_double), ("status", ctypes.c_int)]


class StLinsolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("res_norm", ctypes.c_double), ("rhs_norm", ctypes.c_double)]


class StError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


_lib = None


def library_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load libst.so (building it first when missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError("libst.so not built: run paper_2603_28706_gb300.build.build()")
    lib = ctypes.CDLL(_build.LIB)
    vp, P = ctypes.c_void_p, ctypes.POINTER(StParams)
    lib.st_setup_mesh.argtypes = [P, vp, ctypes.POINTER(vp)]
    lib.st_destroy.argtypes = [vp]
    lib.st_num_dofs.argtypes = [vp, ctypes.c_int]
    lib.st_num_dofs.restype = ctypes.c_size_t
    lib.st_residual.argtypes = [vp, ctypes.c_int, vp, vp, vp, vp]
    lib.st_linearize.argtypes = [vp, ctypes.c_int, vp]
    lib.st_jacobian_apply.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp, vp]
    lib.st_mnorm.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_double)]
    lib.st_precond_setup.argtypes = [vp, ctypes.c_int]
    lib.st_vanka_smooth.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp]
    lib.st_vcycle.argtypes = [vp, ctypes.c_int, vp, vp]
    lib.st_newton_step.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp, vp, ctypes.POINTER(StNewtonInfo)]
    lib.st_fgmres_solve.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.c_double, ctypes.c_int,
                                    ctypes.POINTER(StLinsolveInfo)]
    lib.st_last_error.argtypes = [vp]
    lib.st_last_error.restype = ctypes.c_char_p
    lib.st_mnorm_noalloc.argtypes = [P, vp, vp, ctypes.POINTER(ctypes.c_double)]
    lib.st_mnorm_noalloc.restype = ctypes.c_int
    vpp = ctypes.POINTER(vp)
    lib.st_batch_setup.argtypes = [P, ctypes.c_int, vp, ctypes.POINTER(vp)]
    lib.st_batch_destroy.argtypes = [vp]
    lib.st_batch_num_dofs.argtypes = [vp, ctypes.c_int]
    lib.st_batch_num_dofs.restype = ctypes.c_size_t
    lib.st_batch_linearize.argtypes = [vp, ctypes.c_int, vpp]
    lib.st_batch_jacobian_apply.argtypes = [vp, ctypes.c_int, ctypes.c_int, vpp, vpp]
    lib.st_batch_residual.argtypes = [vp, ctypes.c_int, vpp, vpp, vpp, vpp]
    lib.st_batch_newton_step.argtypes = [vp, ctypes.c_int, ctypes.c_int, vpp, vpp, vpp, ctypes.POINTER(StNewtonInfo)]
    lib.st_batch_fgmres_solve.argtypes = [vp, ctypes.c_int, vpp, vpp, ctypes.c_double, ctypes.c_int,
                                          ctypes.POINTER(StLinsolveInfo)]
    lib.st_batch_fgmres_solve.restype = ctypes.c_int
    lib.st_autotune_report.argtypes = [ctypes.c_char_p, ctypes.c_size_t]
    lib.st_autotune_report.restype = ctypes.c_size_t
    lib.st_batch_last_error.argtypes = [vp]
    lib.st_batch_last_error.restype = ctypes.c_char_p
    for name in ("st_batch_setup", "st_batch_destroy", "st_batch_linearize", "st_batch_jacobian_apply",
                 "st_batch_residual", "st_batch_newton_step"):
        getattr(lib, name).restype = ctypes.c_int
    for name in EXPORTED:
        getattr(lib, name)
    for name in ("st_setup_mesh", "st_destroy", "st_residual", "st_linearize", "st_jacobian_apply", "st_mnorm",
                 "st_precond_setup", "st_vanka_smooth", "st_vcycle", "st_newton_step", "st_fgmres_solve"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


_OPTIONAL = {"gamma_cip": 0.0, "finest_patches": 0, "coarse_solve": 0, "pressure_space": 0, "smoother": 0,
             "patch_type": 0, "omega_coarse": 0.0}


def params(p):
    return StParams(*[p.get(name, _OPTIONAL[name]) if name in _OPTIONAL else p[name] for name, _ in StParams._fields_])


def _ptr(t, dtype=None, n=None, name="vector"):
    if t is None:
        return None
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise TypeError("%s must be a CUDA tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if dtype is not None and t.dtype != dtype:
        raise TypeError("%s must have dtype %s (got %s)" % (name, dtype, t.dtype))
    if n is not None and t.numel() != n:
        raise ValueError("%s must have %d entries (got %d)" % (name, n, t.numel()))
    return ctypes.c_void_p(t.data_ptr())


def _prec_dtype(prec):
    import torch
    return torch.float64 if prec == ST_FP64 else torch.float32


def slab_dofs(p):
    """(k+1)(d (2nx+1)(2ny+1)(2nz+1) + (nx+1)(ny+1)(nz+1)): the length of a
    finest-level slab vector for the parameter dict p (Q2/Q1, eq. slab-system)."""
    d = p["dim"]
    n = [p["nx"], p["ny"], p["nz"] if d == 3 else 0]
    nq2 = nq1 = 1
    for a in range(d):
        nq2 *= 2 * n[a] + 1
        nq1 *= n[a] + 1
    return (p["k"] + 1) * (d * nq2 + nq1)


def mnorm_noalloc(p, r, stream=None):
    """|r|_M without a handle and without any device allocation (st_mnorm_noalloc).

    For callers that cannot allocate device memory; the library keeps a static
    16 MiB scratch array per GPU, which limits the slab to 1 047 552 dofs.
    Calls that overlap on the GPU share that array and must be serialised.
    r must live on the current CUDA device (the one whose copy of the array
    the call uses) and hold exactly slab_dofs(p) doubles."""
    import torch
    if p.get("pressure_space", 0) != 0:
        raise ValueError("st_mnorm_noalloc implements the Q2/Q1 pair only (pressure_space = 0)")
    lib = load()
    P = params(p)
    ptr = _ptr(r, torch.float64, slab_dofs(p), "r")
    if r.device.index != torch.cuda.current_device():
        raise ValueError("r is on cuda:%d but the current device is cuda:%d"
                         % (r.device.index, torch.cuda.current_device()))
    if stream is None:
        stream = torch.cuda.current_stream()
    elif stream.device.index != r.device.index:
        raise ValueError("the stream is not on r's device")
    v = ctypes.c_double()
    st = lib.st_mnorm_noalloc(ctypes.byref(P), ctypes.c_void_p(stream.cuda_stream), ptr, ctypes.byref(v))
    if st != ST_OK:
        raise StError(st, "st_mnorm_noalloc failed (see stderr)")
    return v.value


def autotune_report():
    """The launch shapes the library's autotuner chose in this process (st_autotune_report)."""
    lib = load()
    n = lib.st_autotune_report(None, 0)
    buf = ctypes.create_string_buffer(int(n))
    lib.st_autotune_report(buf, n)
    return buf.value.decode()


class Problem:
    """One slab problem on the current CUDA device (st_setup_mesh handle)."""

    def __init__(self, p, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU path)")
        self.lib = load()
        self.p = dict(p)
        self._P = params(p)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        st = self.lib.st_setup_mesh(ctypes.byref(self._P), ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h))
        if st != ST_OK:
            raise StError(st, "st_setup_mesh failed")
        self.h = h
        d = p["dim"]
        self.levels = p["levels"]

    def close(self):
        if getattr(self, "h", None):
            self.lib.st_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != ST_OK:
            raise StError(st, "%s: %s" % (what, self.lib.st_last_error(self.h).decode()))
        return st

    def num_dofs(self, level=None):
        if level is None:
            level = self.levels - 1
        return int(self.lib.st_num_dofs(self.h, level))

    def velocity_size(self, level=None):
        if level is None:
            level = self.levels - 1
        sh = self.levels - 1 - level
        n = [self.p["nx"] >> sh, self.p["ny"] >> sh, (self.p["nz"] >> sh) if self.p["dim"] == 3 else 0]
        g = 1
        for a in range(self.p["dim"]):
            g *= 2 * n[a] + 1
        return self.p["dim"] * g

    # -- entry points (same names as the C ABI) --
    def residual(self, U, v_prev, f=None, R=None, prec=ST_FP64):
        import torch
        dt = _prec_dtype(prec)
        n = self.num_dofs()
        if R is None:
            R = torch.empty(n, dtype=dt, device=U.device)
        self._check(self.lib.st_residual(self.h, prec, _ptr(U, dt, n, "U"),
                                         _ptr(v_prev, dt, self.velocity_size(), "v_prev"),
                                         _ptr(f, dt, (self.p["k"] + 1) * self.velocity_size(), "f"),
                                         _ptr(R, dt, n, "R")), "st_residual")
        return R

    def linearize(self, tangent, U):
        import torch
        self._check(self.lib.st_linearize(self.h, tangent, _ptr(U, torch.float64, self.num_dofs(), "U")),
                    "st_linearize")

    def jacobian_apply(self, tangent, dU, out=None, U_state=None, prec=ST_FP64):
        import torch
        dt = _prec_dtype(prec)
        n = self.num_dofs()
        if out is None:
            out = torch.empty(n, dtype=dt, device=dU.device)
        self._check(self.lib.st_jacobian_apply(self.h, tangent, prec, _ptr(U_state, torch.float64, n, "U_state"),
                                               _ptr(dU, dt, n, "dU"), _ptr(out, dt, n, "out")),
                    "st_jacobian_apply")
        return out

    def mnorm(self, r):
        import torch
        v = ctypes.c_double()
        self._check(self.lib.st_mnorm(self.h, _ptr(r, torch.float64, self.num_dofs(), "r"), ctypes.byref(v)),
                    "st_mnorm")
        return v.value

    def precond_setup(self, prec=ST_FP32):
        self._check(self.lib.st_precond_setup(self.h, prec), "st_precond_setup")

    def vanka_smooth(self, level, sweeps, r, d, prec=ST_FP32):
        dt = _prec_dtype(prec)
        n = self.num_dofs(level)
        self._check(self.lib.st_vanka_smooth(self.h, level, sweeps, prec, _ptr(r, dt, n, "r"), _ptr(d, dt, n, "d")),
                    "st_vanka_smooth")
        return d

    def vcycle(self, r, d=None, prec=ST_FP32):
        import torch
        dt = _prec_dtype(prec)
        n = self.num_dofs()
        if d is None:
            d = torch.empty(n, dtype=dt, device=r.device)
        self._check(self.lib.st_vcycle(self.h, prec, _ptr(r, dt, n, "r"), _ptr(d, dt, n, "d")), "st_vcycle")
        return d

    def fgmres_solve(self, b, x=None, rtol=1e-8, maxit=200, vcycle_prec=ST_FP32, raise_on_fail=True):
        import torch
        n = self.num_dofs()
        if x is None:
            x = torch.empty(n, dtype=torch.float64, device=b.device)
        info = StLinsolveInfo()
        st = self.lib.st_fgmres_solve(self.h, vcycle_prec, _ptr(b, torch.float64, n, "b"),
                                      _ptr(x, torch.float64, n, "x"), float(rtol), int(maxit), ctypes.byref(info))
        if raise_on_fail and st != ST_OK:
            raise StError(st, "st_fgmres_solve: %s" % self.lib.st_last_error(self.h).decode())
        return st, x, {name: getattr(info, name) for name, _ in StLinsolveInfo._fields_}

    def newton_step(self, tangent, U, v_prev, f=None, vcycle_prec=ST_FP32, raise_on_fail=True):
        import torch
        info = StNewtonInfo()
        n = self.num_dofs()
        st = self.lib.st_newton_step(self.h, tangent, vcycle_prec, _ptr(U, torch.float64, n, "U"),
                                     _ptr(v_prev, torch.float64, self.velocity_size(), "v_prev"),
                                     _ptr(f, torch.float64, (self.p["k"] + 1) * self.velocity_size(), "f"),
                                     ctypes.byref(info))
        if raise_on_fail and st not in (ST_OK,):
            raise StError(st, "st_newton_step: %s" % self.lib.st_last_error(self.h).decode())
        return st, {name: getattr(info, name) for name, _ in StNewtonInfo._fields_}


def _ptr_array(ts, dtype, sizes, name):
    arr = (ctypes.c_void_p * len(ts))()
    for i, t in enumerate(ts):
        arr[i] = _ptr(t, dtype, sizes[i], "%s[%d]" % (name, i)).value
    return arr


class Batch:
    """Independent slab problems (same dim and k) handled together (st_batch_*):
    the operator calls share one persistent volume launch over all instances'
    cells; Newton steps run concurrently, one host thread and stream each."""

    def __init__(self, plist, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU path)")
        self.lib = load()
        self.plist = [dict(p) for p in plist]
        arr = (StParams * len(plist))(*[params(p) for p in plist])
        self._arr = arr
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        b = ctypes.c_void_p()
        st = self.lib.st_batch_setup(arr, len(plist), ctypes.c_void_p(stream.cuda_stream), ctypes.byref(b))
        if st != ST_OK:
            raise StError(st, "st_batch_setup failed")
        self.b = b
        self.n = len(plist)

    def close(self):
        if getattr(self, "b", None):
            self.lib.st_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != ST_OK:
            raise StError(st, "%s: %s" % (what, self.lib.st_batch_last_error(self.b).decode()))
        return st

    def num_dofs(self, i):
        return int(self.lib.st_batch_num_dofs(self.b, i))

    def velocity_size(self, i):
        p = self.plist[i]
        g = 1
        for a, key in enumerate(("nx", "ny", "nz")[:p["dim"]]):
            g *= 2 * p[key] + 1
        return p["dim"] * g

    # -- entry points (same names as the C ABI) --
    def linearize(self, tangent, Us):
        import torch
        self._check(self.lib.st_batch_linearize(
            self.b, tangent, _ptr_array(Us, torch.float64, [self.num_dofs(i) for i in range(self.n)], "U")),
            "st_batch_linearize")

    def jacobian_apply(self, tangent, dUs, outs=None, prec=ST_FP64):
        import torch
        dt = _prec_dtype(prec)
        if outs is None:
            outs = [torch.empty(self.num_dofs(i), dtype=dt, device=dUs[i].device) for i in range(self.n)]
        sz = [self.num_dofs(i) for i in range(self.n)]
        self._check(self.lib.st_batch_jacobian_apply(self.b, tangent, prec, _ptr_array(dUs, dt, sz, "dU"),
                                                     _ptr_array(outs, dt, sz, "out")), "st_batch_jacobian_apply")
        return outs

    def residual(self, Us, v_prevs, fs=None, Rs=None, prec=ST_FP64):
        import torch
        dt = _prec_dtype(prec)
        if Rs is None:
            Rs = [torch.empty(self.num_dofs(i), dtype=dt, device=Us[i].device) for i in range(self.n)]
        sz = [self.num_dofs(i) for i in range(self.n)]
        vs = [self.velocity_size(i) for i in range(self.n)]
        fa = None
        if fs is not None:
            fa = (ctypes.c_void_p * self.n)()
            for i, f in enumerate(fs):
                fa[i] = None if f is None else _ptr(f, dt, (self.plist[i]["k"] + 1) * vs[i], "f[%d]" % i).value
        self._check(self.lib.st_batch_residual(self.b, prec, _ptr_array(Us, dt, sz, "U"),
                                               _ptr_array(v_prevs, dt, vs, "v_prev"), fa,
                                               _ptr_array(Rs, dt, sz, "R")), "st_batch_residual")
        return Rs

    def fgmres_solve(self, rhs, xs=None, rtol=1e-8, maxit=200, vcycle_prec=ST_FP32, raise_on_fail=True):
        import torch
        sz = [self.num_dofs(i) for i in range(self.n)]
        if xs is None:
            xs = [torch.empty(sz[i], dtype=torch.float64, device=rhs[i].device) for i in range(self.n)]
        infos = (StLinsolveInfo * self.n)()
        st = self.lib.st_batch_fgmres_solve(self.b, vcycle_prec, _ptr_array(rhs, torch.float64, sz, "rhs"),
                                            _ptr_array(xs, torch.float64, sz, "x"), float(rtol), int(maxit), infos)
        if raise_on_fail and st != ST_OK:
            raise StError(st, "st_batch_fgmres_solve: %s" % self.lib.st_batch_last_error(self.b).decode())
        return st, xs, [{name: getattr(infos[i], name) for name, _ in StLinsolveInfo._fields_} for i in range(self.n)]

    def newton_step(self, tangent, Us, v_prevs, fs=None, vcycle_prec=ST_FP32, raise_on_fail=True):
        import torch
        infos = (StNewtonInfo * self.n)()
        sz = [self.num_dofs(i) for i in range(self.n)]
        vs = [self.velocity_size(i) for i in range(self.n)]
        fa = None
        if fs is not None:
            fa = (ctypes.c_void_p * self.n)()
            for i, f in enumerate(fs):
                fa[i] = None if f is None else _ptr(f, torch.float64, (self.plist[i]["k"] + 1) * vs[i],
                                                    "f[%d]" % i).value
        st = self.lib.st_batch_newton_step(self.b, tangent, vcycle_prec, _ptr_array(Us, torch.float64, sz, "U"),
                                           _ptr_array(v_prevs, torch.float64, vs, "v_prev"), fa, infos)
        if raise_on_fail and st != ST_OK:
            raise StError(st, "st_batch_newton_step: %s" % self.lib.st_batch_last_error(self.b).decode())
        return st, [{name: getattr(infos[i], name) for name, _ in StNewtonInfo._fields_} for i in range(self.n)]
