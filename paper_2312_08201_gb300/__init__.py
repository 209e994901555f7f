"""Python binding of liblyap (argument marshalling only).

Every computation runs in the CUDA library ``liblyap.so`` (built in-tree by
``paper_2312_08201_gb300.builder``); this module converts NumPy arrays or
torch tensors to pointers, sizes and streams and back. There is no CPU
fallback: without the compiled library (or without a GPU) calls raise.

Problem (paper §1, eqs. (Ljap jdba 1), (formA), transposed convention):
    A(v) = A0 - U diag(v) V^T,   A(v)^T X + X A(v) = -G G^T,   f(v) = trace(E X(v)).
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblyap.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "lyap.h")
TESTING_HEADER = os.path.join(os.path.dirname(HERE), "include", "lyap_testing.h")

OK = 0
PENDING = 1
EINVAL = -1
ENOMEM = -2
EUNSTABLE_SEED = -3
ECUDA = -4
ESOLVER = -5
ENOCONV = -6
EBREAKDOWN = -7
EDEVICE_TIMEOUT = -8
ENOTFOUND = -9
ENONFINITE = -10
ECANCELLED = -11
MEM_HOST = 0
MEM_DEVICE = 1
FP64 = 0
BF16_IR = 2
INJECT_ALLOC_FAIL = 0x1
INJECT_FORCE_MAXIT = 0x2
INJECT_DEVICE_WAIT = 0x4
RESID_FF = 0
RESID_FP64 = 1
RESID_TC = 2
TEST_FF = 3  # lyap_test_apply: float-float residual kernel
TEST_TC = 4  # lyap_test_apply: integer-sliced tensor-core residual kernel


class LyapOpts(ctypes.Structure):
    _fields_ = [
        ("tol", ctypes.c_double),
        ("refine_tol", ctypes.c_double),
        ("inner_tol", ctypes.c_double),
        ("maxit", ctypes.c_int),
        ("m", ctypes.c_int),
        ("s", ctypes.c_int),
        ("pbar", ctypes.c_int),
        ("batch", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("max_refine", ctypes.c_int),
        ("hbm_budget", ctypes.c_size_t),
        ("stream", ctypes.c_void_p),
        ("inject", ctypes.c_uint),
        ("residual", ctypes.c_int),
    ]


class ResultInfo(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int),
        ("refine_steps", ctypes.c_int),
        ("status", ctypes.c_int),
        ("rel_resid", ctypes.c_double),
        ("err_est", ctypes.c_double),
    ]


class SeedStats(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int),
        ("k", ctypes.c_int),
        ("g", ctypes.c_int),
        ("real_path", ctypes.c_int),
        ("cond_Q", ctypes.c_double),
        ("f0", ctypes.c_double),
        ("max_re_lambda", ctypes.c_double),
        ("min_abs_lambda_sum", ctypes.c_double),
        ("resident_bytes", ctypes.c_size_t),
    ]


class ProfKernel(ctypes.Structure):
    _fields_ = [
        ("name", ctypes.c_char * 32),
        ("launches", ctypes.c_longlong),
        ("total_ms", ctypes.c_double),
        ("units", ctypes.c_double),
        ("flops", ctypes.c_double),
        ("bytes", ctypes.c_double),
    ]


class LyapError(RuntimeError):
    def __init__(self, code, what=""):
        lib = _LIB
        name = lib.lyap_strerror(code).decode() if lib else str(code)
        detail = lib.lyap_last_error().decode() if lib else ""
        super().__init__(f"{what}: {name} ({code}) {detail}".strip())
        self.code = code


_LIB = None
_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)

_SIGS = {
    "lyap_opts_default": (None, [ctypes.POINTER(LyapOpts)]),
    "lyap_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "lyap_last_error": (ctypes.c_char_p, []),
    "lyap_ctx_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_P)]),
    "lyap_ctx_destroy": (None, [_P]),
    "lyap_seed_factor": (
        ctypes.c_int,
        [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P, _P, ctypes.c_int,
         ctypes.POINTER(LyapOpts), ctypes.POINTER(_P), _D],
    ),
    "lyap_seed_stats_get": (ctypes.c_int, [_P, ctypes.POINTER(SeedStats)]),
    "lyap_seed_free": (ctypes.c_int, [_P]),
    "lyap_param_solve": (
        ctypes.c_int,
        [_P, ctypes.c_int, _P, ctypes.c_int, ctypes.POINTER(LyapOpts), _P, ctypes.POINTER(ResultInfo)],
    ),
    "lyap_trace_EX": (
        ctypes.c_int,
        [_P, ctypes.c_int, _P, ctypes.c_int, ctypes.POINTER(LyapOpts), _P, ctypes.POINTER(ResultInfo)],
    ),
    "lyap_grad": (
        ctypes.c_int,
        [_P, ctypes.c_int, _P, ctypes.c_int, ctypes.POINTER(LyapOpts), _P, _P, ctypes.POINTER(ResultInfo)],
    ),
    "lyap_serve_create": (ctypes.c_int, [_P, ctypes.POINTER(LyapOpts), ctypes.POINTER(_P)]),
    "lyap_serve_register_seed": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_int)]),
    "lyap_serve_submit": (
        ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)]
    ),
    "lyap_serve_estimate": (
        ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]
    ),
    "lyap_serve_run": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "lyap_serve_poll": (
        ctypes.c_int, [_P, ctypes.c_uint64, _P, _P, ctypes.POINTER(ResultInfo), ctypes.POINTER(ctypes.c_double)]
    ),
    "lyap_serve_cancel": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "lyap_serve_destroy": (None, [_P]),
    "lyap_check_solution_noalloc": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _P, _P]),
    "lyap_check_explicit": (
        ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _P, _P, _P, ctypes.c_int, _P, ctypes.c_int, _P, _P]
    ),
    "lyap_proj_create": (
        ctypes.c_int,
        [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P, _P, _P, ctypes.c_double, ctypes.c_int,
         ctypes.POINTER(LyapOpts), ctypes.POINTER(_P)],
    ),
    "lyap_proj_trace_EX": (
        ctypes.c_int,
        [_P, ctypes.c_int, _P, ctypes.c_int, ctypes.POINTER(LyapOpts), ctypes.c_double, ctypes.c_int, _P, _P, _P,
         ctypes.POINTER(ResultInfo)],
    ),
    "lyap_proj_dims": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "lyap_proj_free": (ctypes.c_int, [_P]),
    "lyap_test_apply": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.c_int, ctypes.c_int, _P]),
    "lyap_test_tc_gemm": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P, _P]),
    "lyap_prof_enable": (ctypes.c_int, [ctypes.c_int]),
    "lyap_prof_read": (
        ctypes.c_int,
        [ctypes.POINTER(ProfKernel), ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_longlong)],
    ),
}


def header_functions(path: str | None = None):
    """Names of the functions declared in include/lyap.h and lyap_testing.h."""
    if path is None:
        return sorted(set(header_functions(HEADER)) | set(header_functions(TESTING_HEADER)))
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lyap_[a-zA-Z0-9_]+)\s*\(", text)))


def load(path: str = LIB_PATH):
    """Load liblyap.so (raise if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise ImportError(f"{path} not built; run paper_2312_08201_gb300.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def build(verbose: bool = False) -> str:
    from .builder import build as _b

    return _b(verbose=verbose)


def default_opts(**kw) -> LyapOpts:
    lib = load()
    o = LyapOpts()
    lib.lyap_opts_default(ctypes.byref(o))
    for key, val in kw.items():
        if key == "stream":
            val = ctypes.c_void_p(val)
        setattr(o, key, val)
    return o


def _check(code, what):
    if code != OK:
        raise LyapError(code, what)


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _host_f64(a, order="F"):
    return np.require(np.asarray(a, dtype=np.float64), requirements=[order, "A", "W"] if order == "F" else ["C"])


def _current_stream_ptr(dev_tensor):
    import torch

    return torch.cuda.current_stream(dev_tensor.device).cuda_stream


class Context:
    """A CUDA device, its stream and library handles."""

    def __init__(self, device: int = 0):
        lib = load()
        h = _P()
        _check(lib.lyap_ctx_create(device, ctypes.byref(h)), "lyap_ctx_create")
        self.h = h
        self.device = device

    def close(self):
        if self.h:
            for seed in list(getattr(self, "_seeds", [])):
                seed.free()
            load().lyap_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Seed:
    """A factored seed A0 (device-resident) for a family A(v) = A0 - U diag(v) V^T."""

    def __init__(self, ctx: Context, A0, U, V, G, E=None, **opts):
        lib = load()
        self.ctx = ctx
        n = int(A0.shape[0])
        k = int(U.shape[1])
        g = int(G.shape[1])
        o = default_opts(**opts)
        h = _P()
        cond = ctypes.c_double()
        if _is_torch(A0) and A0.is_cuda:
            # device inputs: column-major float64 = transpose of a contiguous row-major tensor
            import torch

            arrs = [t.detach().to(torch.float64).t().contiguous() for t in (A0, U, V, G)]
            e = E.detach().double().t().contiguous() if E is not None else None
            o.stream = _current_stream_ptr(A0)
            ptrs = [ctypes.c_void_p(a.data_ptr()) for a in arrs]
            code = lib.lyap_seed_factor(ctx.h, n, k, g, *ptrs, ctypes.c_void_p(e.data_ptr()) if e is not None else None,
                                        MEM_DEVICE, ctypes.byref(o), ctypes.byref(h), ctypes.byref(cond))
        else:
            arrs = [_host_f64(a) for a in (A0, U, V, G)]
            e = _host_f64(E) if E is not None else None
            ptrs = [a.ctypes.data_as(ctypes.c_void_p) for a in arrs]
            code = lib.lyap_seed_factor(ctx.h, n, k, g, *ptrs, e.ctypes.data_as(ctypes.c_void_p) if e is not None else None,
                                        MEM_HOST, ctypes.byref(o), ctypes.byref(h), ctypes.byref(cond))
        _check(code, "lyap_seed_factor")
        self.h = h
        import weakref

        if not hasattr(ctx, "_seeds"):
            ctx._seeds = weakref.WeakSet()
        ctx._seeds.add(self)
        self.n, self.k, self.g = n, k, g
        self.cond_Q = cond.value

    def stats(self) -> dict:
        s = SeedStats()
        _check(load().lyap_seed_stats_get(self.h, ctypes.byref(s)), "lyap_seed_stats_get")
        return {f: getattr(s, f) for f, _ in SeedStats._fields_}

    def free(self):
        if getattr(self, "h", None):
            load().lyap_seed_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    # ------------------------------------------------------------------ calls
    def _prep_v(self, v, o):
        if _is_torch(v) and v.is_cuda:
            import torch

            vt = v.detach().to(torch.float64).contiguous()
            o.stream = _current_stream_ptr(vt)
            return vt, MEM_DEVICE, ctypes.c_void_p(vt.data_ptr()), int(vt.shape[0])
        va = np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(-1, self.k))
        return va, MEM_HOST, va.ctypes.data_as(ctypes.c_void_p), int(va.shape[0])

    def _out(self, like, mem, shape):
        if mem == MEM_DEVICE:
            import torch

            t = torch.empty(shape, dtype=torch.float64, device=like.device)
            return t, ctypes.c_void_p(t.data_ptr())
        a = np.empty(shape, dtype=np.float64)
        return a, a.ctypes.data_as(ctypes.c_void_p)

    def trace_EX(self, v, return_info: bool = False, **opts):
        """f(v) = trace(E X(v)) for each row of v (nv x k)."""
        lib = load()
        o = default_opts(**opts)
        keep, mem, vp, nv = self._prep_v(v, o)
        out, op = self._out(keep, mem, (nv,))
        info = (ResultInfo * max(nv, 1))()
        _check(lib.lyap_trace_EX(self.h, nv, vp, mem, ctypes.byref(o), op, info), "lyap_trace_EX")
        return (out, _infos(info, nv)) if return_info else out

    def grad(self, v, return_info: bool = False, **opts):
        """(f(v), df/dv) for each row of v."""
        lib = load()
        o = default_opts(**opts)
        keep, mem, vp, nv = self._prep_v(v, o)
        f, fp = self._out(keep, mem, (nv,))
        g, gp = self._out(keep, mem, (nv, self.k))
        info = (ResultInfo * max(nv, 1))()
        _check(lib.lyap_grad(self.h, nv, vp, mem, ctypes.byref(o), fp, gp, info), "lyap_grad")
        return (f, g, _infos(info, nv)) if return_info else (f, g)

    def param_solve(self, v, **opts):
        """Capacitance solutions W'(v): complex array (nv, k, n) (column t = W'[:, t])."""
        lib = load()
        o = default_opts(**opts)
        keep, mem, vp, nv = self._prep_v(v, o)
        w, wp = self._out(keep, mem, (nv, self.k, self.n, 2))
        info = (ResultInfo * max(nv, 1))()
        _check(lib.lyap_param_solve(self.h, nv, vp, mem, ctypes.byref(o), wp, info), "lyap_param_solve")
        if mem == MEM_HOST:
            return w[..., 0] + 1j * w[..., 1], _infos(info, nv)
        return w, _infos(info, nv)


class Projection:
    """The projection framework of §2.2 (lyap_proj_*): one extended Krylov
    space EK_m(A0^T, [X0 U, V]) for every v, grown on demand; each v is
    accepted once its backward error meets eps (Algorithm 1)."""

    def __init__(self, ctx: Context, A0, U, V, G=None, E=None, XBr=None, fX0=0.0, **opts):
        lib = load()
        self.ctx = ctx
        n, k = int(A0.shape[0]), int(U.shape[1])
        g = int(G.shape[1]) if G is not None else 0
        o = default_opts(**opts)
        arrs = [_host_f64(a) for a in (A0, U, V)]
        ga = _host_f64(G) if G is not None else None
        ea = _host_f64(E) if E is not None else None
        xa = _host_f64(XBr) if XBr is not None else None
        ptr = (lambda a: a.ctypes.data_as(ctypes.c_void_p) if a is not None else None)
        h = _P()
        _check(lib.lyap_proj_create(ctx.h, n, k, g, *[ptr(a) for a in arrs], ptr(ga), ptr(ea), ptr(xa), float(fX0),
                                    MEM_HOST, ctypes.byref(o), ctypes.byref(h)), "lyap_proj_create")
        self.h = h
        self.n, self.k = n, k

    def trace_EX(self, v, eps=1e-10, m_max=200, return_info=False, **opts):
        """f(v) per row of v; with return_info also (delta, blocks, infos)."""
        lib = load()
        o = default_opts(**opts)
        va = np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(-1, self.k))
        nv = va.shape[0]
        f = np.empty(nv)
        dl = np.empty(nv)
        mb = np.empty(nv, dtype=np.int32)
        info = (ResultInfo * max(nv, 1))()
        _check(lib.lyap_proj_trace_EX(self.h, nv, va.ctypes.data_as(ctypes.c_void_p), MEM_HOST, ctypes.byref(o),
                                      float(eps), int(m_max), f.ctypes.data_as(ctypes.c_void_p),
                                      dl.ctypes.data_as(ctypes.c_void_p), mb.ctypes.data_as(ctypes.c_void_p), info),
               "lyap_proj_trace_EX")
        return (f, dl, mb, _infos(info, nv)) if return_info else f

    def dims(self):
        b, d = ctypes.c_int(), ctypes.c_int()
        _check(load().lyap_proj_dims(self.h, ctypes.byref(b), ctypes.byref(d)), "lyap_proj_dims")
        return b.value, d.value

    def free(self):
        if getattr(self, "h", None):
            load().lyap_proj_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def check_explicit(seed, v, W, A0, U, V, G, E=None):
    """lyap_check_explicit on host arrays: v (nv, k); W the complex (nv, k, n)
    solutions of Seed.param_solve. Returns (backward errors, traces)."""
    lib = load()
    va = np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(-1, seed.k))
    nv = va.shape[0]
    Wc = np.ascontiguousarray(np.asarray(W, dtype=np.complex128).reshape(nv, seed.k, seed.n))
    mats = [_host_f64(a) for a in (A0, U, V, G)]
    ea = _host_f64(E) if E is not None else None
    be = np.empty(nv)
    tr = np.empty(nv)
    ptr = (lambda a: a.ctypes.data_as(ctypes.c_void_p) if a is not None else None)
    _check(lib.lyap_check_explicit(seed.h, nv, ptr(va), ptr(Wc), *[ptr(a) for a in mats], int(mats[3].shape[1]),
                                   ptr(ea), MEM_HOST, ptr(be), ptr(tr)), "lyap_check_explicit")
    return be, tr


class Server:
    """Continuous-batching server over registered seeds (lyap_serve_*)."""

    def __init__(self, ctx: Context, **opts):
        self.lib = load()
        o = default_opts(**opts)
        h = _P()
        _check(self.lib.lyap_serve_create(ctx.h, ctypes.byref(o), ctypes.byref(h)), "lyap_serve_create")
        self.h = h
        self.k = {}

    def register(self, seed: "Seed") -> int:
        sid = ctypes.c_int()
        _check(self.lib.lyap_serve_register_seed(self.h, seed.h, ctypes.byref(sid)), "lyap_serve_register_seed")
        self.k[sid.value] = seed.k
        return sid.value

    def estimate(self, seed_id: int, nv: int, want_grad: bool = False) -> int:
        """Device bytes admission charges for a request of nv vectors."""
        b = ctypes.c_size_t()
        _check(self.lib.lyap_serve_estimate(self.h, seed_id, nv, 1 if want_grad else 0, ctypes.byref(b)),
               "lyap_serve_estimate")
        return b.value

    def submit(self, seed_id: int, v, want_grad: bool = False) -> int:
        va = np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(-1, self.k[seed_id]))
        t = ctypes.c_uint64()
        _check(self.lib.lyap_serve_submit(self.h, seed_id, va.shape[0], va.ctypes.data_as(ctypes.c_void_p),
                                          1 if want_grad else 0, ctypes.byref(t)), "lyap_serve_submit")
        return t.value

    def run(self, max_ms: int = 0) -> bool:
        busy = ctypes.c_int()
        _check(self.lib.lyap_serve_run(self.h, max_ms, ctypes.byref(busy)), "lyap_serve_run")
        return bool(busy.value)

    def poll(self, ticket: int, nv: int, k: int, want_grad: bool = False):
        """None while pending; else dict(f, g, info, latency_s) (raises on a failed request)."""
        f = np.empty(nv)
        g = np.empty((nv, k)) if want_grad else None
        info = (ResultInfo * nv)()
        lat = ctypes.c_double()
        code = self.lib.lyap_serve_poll(self.h, ticket, f.ctypes.data_as(ctypes.c_void_p),
                                        g.ctypes.data_as(ctypes.c_void_p) if g is not None else None, info,
                                        ctypes.byref(lat))
        if code == PENDING:
            return None
        _check(code, "lyap_serve_poll")
        return dict(f=f, g=g, info=_infos(info, nv), latency_s=lat.value)

    def cancel(self, ticket: int) -> int:
        return self.lib.lyap_serve_cancel(self.h, ticket)

    def close(self):
        if getattr(self, "h", None):
            self.lib.lyap_serve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def prof_enable(on: bool = True):
    """Start (clear) or stop the library's per-kernel event timing."""
    _check(load().lyap_prof_enable(1 if on else 0), "lyap_prof_enable")


def prof_read():
    """(per-kernel records, library kernel launches since prof_enable)."""
    arr = (ProfKernel * 32)()
    cnt = ctypes.c_int()
    launches = ctypes.c_longlong()
    _check(load().lyap_prof_read(arr, 32, ctypes.byref(cnt), ctypes.byref(launches)), "lyap_prof_read")
    recs = {
        arr[i].name.decode(): dict(launches=arr[i].launches, total_ms=arr[i].total_ms, units=arr[i].units,
                                   flops=arr[i].flops, bytes=arr[i].bytes)
        for i in range(cnt.value)
    }
    return recs, launches.value


def check_solution_noalloc(seed, v, w, trace_out, resid_out, stream=None):
    """lyap_check_solution_noalloc on torch CUDA tensors: v (nv, k) float64,
    w (nv, k, n, 2) float64 as returned by Seed.param_solve for device v,
    trace_out and resid_out (nv,) float64. Marshals pointers only."""
    import torch

    nv = int(v.shape[0])
    if stream is None:
        stream = torch.cuda.current_stream(v.device).cuda_stream
    code = load().lyap_check_solution_noalloc(
        seed.h, nv, ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(w.data_ptr()),
        ctypes.c_void_p(trace_out.data_ptr()), ctypes.c_void_p(resid_out.data_ptr()), ctypes.c_void_p(stream))
    _check(code, "lyap_check_solution_noalloc")


def test_apply(seed, v, w, precision=FP64, adjoint=False):
    """lyap_test_apply on torch CUDA tensors (v: (nsys, k), w: (nsys, k, n, 2))."""
    import torch

    out = torch.empty_like(w)
    code = load().lyap_test_apply(seed.h, int(v.shape[0]), ctypes.c_void_p(v.data_ptr()),
                                  ctypes.c_void_p(w.data_ptr()), precision, 1 if adjoint else 0,
                                  ctypes.c_void_p(out.data_ptr()))
    _check(code, "lyap_test_apply")
    return out


def test_tc_gemm(A, B):
    """lyap_test_tc_gemm on torch CUDA float32 tensors: returns B @ A^T (N x M)."""
    import torch

    A = A.contiguous()
    B = B.contiguous()
    D = torch.empty((B.shape[0], A.shape[0]), dtype=torch.float32, device=A.device)
    code = load().lyap_test_tc_gemm(int(A.shape[0]), int(B.shape[0]), int(A.shape[1]), ctypes.c_void_p(A.data_ptr()),
                                    ctypes.c_void_p(B.data_ptr()), ctypes.c_void_p(D.data_ptr()))
    _check(code, "lyap_test_tc_gemm")
    return D


def _infos(info, nv):
    return [
        dict(iters=info[i].iters, refine_steps=info[i].refine_steps, status=info[i].status,
             rel_resid=info[i].rel_resid, err_est=info[i].err_est)
        for i in range(nv)
    ]


def trace_ex_function():
    """torch.autograd.Function ``TraceEX``: ``f = TraceEX.apply(v, seed, opts)``.

    ``v`` is an (nv, k) tensor on the seed's GPU (device path: no copy through
    the host) or on the CPU (host path); ``f`` is float64 on ``v``'s device.
    When ``v`` requires a gradient the forward pass calls lyap_grad, which
    adds one adjoint capacitance solve per v (df/dv_i = v_i^-2 <Z_i, W'_i>,
    the adjoint of eq. (SMW_linearsystem)); backward returns
    ``grad_out[:, None] * df/dv`` in ``v``'s dtype and device. ``opts`` is a
    dict of lyap_opts fields (e.g. ``{"precision": BF16_IR}``)."""
    import torch

    class TraceEX(torch.autograd.Function):
        @staticmethod
        def forward(ctx, v, seed, opts=None):
            opts = dict(opts or {})
            if v.dim() != 2 or v.shape[1] != seed.k:
                raise ValueError(f"v must have shape (nv, {seed.k})")
            vd = v.detach().to(torch.float64)
            vin = vd.contiguous() if vd.is_cuda else vd.cpu().numpy()
            ctx.v_dtype, ctx.v_device = v.dtype, v.device
            if ctx.needs_input_grad[0]:
                f, g = seed.grad(vin, **opts)
                ctx.save_for_backward(torch.as_tensor(g).to(device=v.device, dtype=torch.float64))
            else:
                f = seed.trace_EX(vin, **opts)
            return torch.as_tensor(f).to(device=v.device, dtype=torch.float64)

        @staticmethod
        def backward(ctx, grad_out):
            (g,) = ctx.saved_tensors
            gv = grad_out.to(device=g.device, dtype=torch.float64)[:, None] * g
            return gv.to(device=ctx.v_device, dtype=ctx.v_dtype), None, None

    return TraceEX
