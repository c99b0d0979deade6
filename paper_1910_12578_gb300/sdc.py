"""Python binding of libsdc (include/sdc.h): argument marshalling only.

Every step of the SDC hot path runs in the library's CUDA kernels; PyTorch
supplies device memory and the CUDA stream.  There is no CPU fallback: without
the compiled library, or without a GPU, these calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import workloads as W

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsdc.so")

SDC_OK, SDC_ERR_INVALID_ARG, SDC_ERR_CUDA, SDC_ERR_OOM, SDC_ERR_NEWTON_NOCONV, SDC_ERR_NONPHYSICAL, \
    SDC_ERR_TIMEOUT, SDC_ERR_TOO_LARGE = range(8)
STATIC_SCRATCH_BYTES = 48 << 20
PREC_FP64, PREC_FP32_JAC, PREC_FP32X2_JAC = 0, 1, 2

# entry points declared in include/sdc.h
EXPORTS = ["sdc_init_box", "sdc_advective_term", "sdc_node_integral", "sdc_react_newton", "sdc_step",
           "sdc_step_profile", "sdc_launches_per_step", "sdc_cfl_dt", "sdc_sizes", "sdc_destroy",
           "sdc_status_string", "sdc_step_static", "sdc_selftest_math", "sdc_selftest_pow", "sdc_autotune",
           "sdc_set_variants",
           "sdc_step_backward", "sdc_set_rates", "sdc_advective_term_vjp", "sdc_step_strang"]


class SdcError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__("%s: %s (status %d)" % (what, _status_string(status), status))


class Box(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("dx", C.c_double * 3)]


class Network(C.Structure):
    _fields_ = [("nspec", C.c_int), ("nreac", C.c_int), ("rate_law", C.c_int),
                ("mass", C.POINTER(C.c_double)), ("a", C.POINTER(C.c_double)), ("nu", C.POINTER(C.c_double)),
                ("Q", C.POINTER(C.c_double)), ("reac", C.POINTER(C.c_int)), ("cnt", C.POINTER(C.c_int)),
                ("prod", C.POINTER(C.c_int))]


class Params(C.Structure):
    _fields_ = [("gamma", C.c_double), ("n_nodes", C.c_int), ("n_iters", C.c_int), ("limiter", C.c_int),
                ("prec", C.c_int), ("newton_rtol", C.c_double), ("newton_maxit", C.c_int), ("node_type", C.c_int),
                ("space_order", C.c_int)]


NODE_TYPES = {"lobatto": 0, "radau": 1}


class Stats(C.Structure):
    _fields_ = [("newton_iters_total", C.c_longlong), ("newton_solves", C.c_longlong),
                ("n_fail", C.c_longlong), ("hist", C.c_longlong * 64)]

    def as_dict(self):
        return {"newton_iters_total": self.newton_iters_total, "newton_solves": self.newton_solves,
                "n_fail": self.n_fail, "hist": list(self.hist)}


MAX_VARIANTS = 8   # SDC_MAX_VARIANTS of sdc.h


class Tuning(C.Structure):
    _fields_ = [("stencil_variants", C.c_int), ("newton_variants", C.c_int), ("stencil_choice", C.c_int),
                ("newton_choice", C.c_int), ("ms_stencil", C.c_float * MAX_VARIANTS),
                ("ms_newton", C.c_float * MAX_VARIANTS)]

    def as_dict(self):
        return {"stencil_variants": self.stencil_variants, "newton_variants": self.newton_variants,
                "stencil_choice": self.stencil_choice, "newton_choice": self.newton_choice,
                "ms_stencil": list(self.ms_stencil)[:self.stencil_variants],
                "ms_newton": list(self.ms_newton)[:self.newton_variants]}


class Profile(C.Structure):
    _fields_ = [("launches_stencil", C.c_int), ("launches_newton", C.c_int), ("launches_other", C.c_int),
                ("ms_stencil", C.c_float), ("ms_newton", C.c_float), ("ms_other", C.c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load(path: str = LIB_PATH):
    """Load libsdc.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libsdc.so is missing at %s: build it with __graft_entry__.build() "
                           "(no CPU fallback exists)" % path)
    L = C.CDLL(path)
    vp = C.c_void_p
    dp = C.c_void_p
    L.sdc_init_box.argtypes = [C.POINTER(Box), C.c_int, C.POINTER(Network), C.POINTER(Params), vp,
                               C.POINTER(vp)]
    L.sdc_advective_term.argtypes = [vp, dp, dp]
    L.sdc_node_integral.argtypes = [vp, dp, dp, C.c_double, C.c_int, dp]
    L.sdc_react_newton.argtypes = [vp, dp, C.c_double, dp, dp, vp, vp, C.POINTER(Stats)]
    L.sdc_step.argtypes = [vp, dp, C.c_double, C.POINTER(Stats)]
    L.sdc_cfl_dt.argtypes = [vp, dp, C.c_double, C.POINTER(C.c_double)]
    L.sdc_step_profile.argtypes = [vp, dp, C.c_double, C.POINTER(Stats), C.POINTER(Profile)]
    L.sdc_launches_per_step.argtypes = [vp, C.POINTER(C.c_int)]
    L.sdc_selftest_math.argtypes = [dp, C.c_longlong, dp, dp, vp]
    L.sdc_selftest_pow.argtypes = [dp, dp, C.c_longlong, dp, vp]
    L.sdc_autotune.argtypes = [vp, dp, C.c_double, C.POINTER(Tuning)]
    L.sdc_step_backward.argtypes = [vp, dp, C.c_double, dp, dp, dp]
    L.sdc_set_rates.argtypes = [vp, C.POINTER(C.c_double)]
    L.sdc_advective_term_vjp.argtypes = [vp, dp, dp, dp, C.c_int]
    L.sdc_step_strang.argtypes = [vp, dp, C.c_double, C.POINTER(Stats)]
    L.sdc_set_variants.argtypes = [vp, C.c_int, C.c_int]
    L.sdc_step_static.argtypes = [C.POINTER(Box), C.c_int, C.POINTER(Network), C.POINTER(Params), vp, dp,
                                  C.c_double, C.POINTER(Stats)]
    L.sdc_sizes.argtypes = [vp, C.POINTER(C.c_longlong), C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.sdc_destroy.argtypes = [vp]
    L.sdc_destroy.restype = None
    L.sdc_status_string.argtypes = [C.c_int]
    L.sdc_status_string.restype = C.c_char_p
    for name in ("sdc_init_box", "sdc_advective_term", "sdc_node_integral", "sdc_react_newton", "sdc_step",
                 "sdc_cfl_dt", "sdc_sizes", "sdc_step_profile", "sdc_launches_per_step", "sdc_step_static", "sdc_selftest_math", "sdc_selftest_pow", "sdc_autotune",
                 "sdc_set_variants", "sdc_step_backward", "sdc_set_rates", "sdc_advective_term_vjp",
                 "sdc_step_strang"):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _status_string(s):
    try:
        return load().sdc_status_string(int(s)).decode()
    except Exception:  # noqa: BLE001 - only used to format an error message
        return "status %d" % s


def _ptr(t):
    """Device pointer of a contiguous CUDA float64 tensor."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError("expected a contiguous CUDA float64 tensor")
    return C.c_void_p(t.data_ptr())


class Context:
    """A libsdc context over one or several periodic boxes sharing a network.

    problems: a workloads.Problem or a list of them (same dim, network and SDC
    parameters; boxes are concatenated in order)."""

    def __init__(self, problems, prec: int = PREC_FP64, stream=None):
        import torch
        L = load()
        if not isinstance(problems, (list, tuple)):
            problems = [problems]
        P0 = problems[0]
        self.problems = list(problems)
        self.dim = P0.dim
        self.nvar = P0.nvar
        self.nw = P0.net.nspec + 1
        self.ntot = sum(p.nzones for p in problems)
        boxes = (Box * len(problems))()
        for i, p in enumerate(problems):
            boxes[i].dim = p.dim
            for d in range(3):
                boxes[i].n[d] = int(p.n[d])
                boxes[i].dx[d] = float(p.dx[d])
        net = P0.net
        self._keep = [np.ascontiguousarray(net.mass, dtype=np.float64), np.ascontiguousarray(net.a, dtype=np.float64),
                      np.ascontiguousarray(net.nu, dtype=np.float64), np.ascontiguousarray(net.Q, dtype=np.float64),
                      np.ascontiguousarray(net.reac, dtype=np.int32).ravel(),
                      np.ascontiguousarray(net.cnt, dtype=np.int32).ravel(),
                      np.ascontiguousarray(net.prod, dtype=np.int32)]
        m, a, nu, Q, reac, cnt, prod = self._keep
        nw = Network(net.nspec, net.nreac, net.rate_law,
                     m.ctypes.data_as(C.POINTER(C.c_double)), a.ctypes.data_as(C.POINTER(C.c_double)),
                     nu.ctypes.data_as(C.POINTER(C.c_double)), Q.ctypes.data_as(C.POINTER(C.c_double)),
                     reac.ctypes.data_as(C.POINTER(C.c_int)), cnt.ctypes.data_as(C.POINTER(C.c_int)),
                     prod.ctypes.data_as(C.POINTER(C.c_int)))
        prm = Params(P0.gamma, P0.n_nodes, P0.n_iters, P0.limiter, int(prec), P0.newton_rtol, P0.newton_maxit,
                     NODE_TYPES[P0.nodes], int(P0.space_order))
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._h = C.c_void_p()
        s = L.sdc_init_box(boxes, len(problems), C.byref(nw), C.byref(prm), C.c_void_p(self.stream.cuda_stream),
                           C.byref(self._h))
        if s != SDC_OK:
            raise SdcError(s, "sdc_init_box")
        self.L = L

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self.L.sdc_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass

    def _check(self, s, what, allow_noconv=False):
        if s == SDC_OK or (allow_noconv and s == SDC_ERR_NEWTON_NOCONV):
            return s
        raise SdcError(s, what)

    # ------------------------------------------------------------ entry points
    def advective_term(self, U, A):
        return self._check(self.L.sdc_advective_term(self._h, _ptr(U), _ptr(A)), "sdc_advective_term")

    def node_integral(self, A_nodes, R_nodes, dt, m, I):
        return self._check(self.L.sdc_node_integral(self._h, _ptr(A_nodes), _ptr(R_nodes), float(dt), int(m),
                                                    _ptr(I)), "sdc_node_integral")

    def react_newton(self, rhs, dt_m, U_inout, R_out, zone_status=None, zone_iters=None, stats=True):
        import torch
        zs = C.c_void_p(zone_status.data_ptr()) if zone_status is not None else None
        zi = C.c_void_p(zone_iters.data_ptr()) if zone_iters is not None else None
        for t in (zone_status, zone_iters):
            if t is not None and (t.dtype != torch.int32 or not t.is_cuda):
                raise TypeError("zone arrays must be CUDA int32")
        st = Stats() if stats else None
        s = self.L.sdc_react_newton(self._h, _ptr(rhs), float(dt_m), _ptr(U_inout), _ptr(R_out), zs, zi,
                                    C.byref(st) if st is not None else None)
        self._check(s, "sdc_react_newton", allow_noconv=True)
        return st

    def step(self, U, dt, stats=True):
        st = Stats() if stats else None
        s = self.L.sdc_step(self._h, _ptr(U), float(dt), C.byref(st) if st is not None else None)
        self._check(s, "sdc_step", allow_noconv=True)
        return st

    def step_strang(self, U, dt, stats=True):
        """One Strang-split step (reactions dt/2, advection dt, reactions dt/2) of U in place."""
        st = Stats() if stats else None
        s = self.L.sdc_step_strang(self._h, _ptr(U), float(dt), C.byref(st) if st is not None else None)
        self._check(s, "sdc_step_strang", allow_noconv=True)
        return st

    def step_profile(self, U, dt):
        """One eagerly launched step (same kernels and results as step) with
        per-class CUDA-event times; returns (Stats, Profile)."""
        st = Stats()
        pr = Profile()
        s = self.L.sdc_step_profile(self._h, _ptr(U), float(dt), C.byref(st), C.byref(pr))
        self._check(s, "sdc_step_profile", allow_noconv=True)
        return st, pr

    def autotune(self, U, dt):
        """Pick the stencil tile shape and Newton variant by timing one step of
        each on a scratch copy of U; returns the Tuning record."""
        t = Tuning()
        self._check(self.L.sdc_autotune(self._h, _ptr(U), float(dt), C.byref(t)), "sdc_autotune")
        return t

    def set_variants(self, stencil_variant, newton_variant):
        self._check(self.L.sdc_set_variants(self._h, int(stencil_variant), int(newton_variant)), "sdc_set_variants")

    def step_backward(self, U_n, dt, gU_np1, gU_n, g_a=None):
        """Adjoint of one step from its checkpoint U_n: gU_n = J^T gU_np1,
        g_a += (dU^{n+1}/da)^T gU_np1 (g_a: CUDA float64 [nreac] or None)."""
        ga = _ptr(g_a) if g_a is not None else None
        self._check(self.L.sdc_step_backward(self._h, _ptr(U_n), float(dt), _ptr(gU_np1), _ptr(gU_n), ga),
                    "sdc_step_backward")

    def advective_term_vjp(self, U, Abar, Ubar, mode=0):
        """Ubar += (dA/dU)^T Abar at U (mode 0: reverse sweep per face; 1: forward-mode duals)."""
        self._check(self.L.sdc_advective_term_vjp(self._h, _ptr(U), _ptr(Abar), _ptr(Ubar), int(mode)),
                    "sdc_advective_term_vjp")

    def set_rates(self, a):
        """Replace the rate prefactors a_j (host values)."""
        arr = np.ascontiguousarray(np.asarray(a, dtype=np.float64).ravel())
        self._check(self.L.sdc_set_rates(self._h, arr.ctypes.data_as(C.POINTER(C.c_double))), "sdc_set_rates")

    def launches_per_step(self):
        n = C.c_int()
        self._check(self.L.sdc_launches_per_step(self._h, C.byref(n)), "sdc_launches_per_step")
        return n.value

    def cfl_dt(self, U, cfl):
        out = C.c_double()
        self._check(self.L.sdc_cfl_dt(self._h, _ptr(U), float(cfl), C.byref(out)), "sdc_cfl_dt")
        return out.value


def _marshal(problems, prec):
    """Box array, network and parameter structs (plus the arrays they point into)."""
    if not isinstance(problems, (list, tuple)):
        problems = [problems]
    boxes = (Box * len(problems))()
    for i, p in enumerate(problems):
        boxes[i].dim = p.dim
        for d in range(3):
            boxes[i].n[d] = int(p.n[d])
            boxes[i].dx[d] = float(p.dx[d])
    P0 = problems[0]
    net = P0.net
    keep = [np.ascontiguousarray(net.mass, dtype=np.float64), np.ascontiguousarray(net.a, dtype=np.float64),
            np.ascontiguousarray(net.nu, dtype=np.float64), np.ascontiguousarray(net.Q, dtype=np.float64),
            np.ascontiguousarray(net.reac, dtype=np.int32).ravel(),
            np.ascontiguousarray(net.cnt, dtype=np.int32).ravel(), np.ascontiguousarray(net.prod, dtype=np.int32)]
    m, a, nu, Q, reac, cnt, prod = keep
    nw = Network(net.nspec, net.nreac, net.rate_law,
                 m.ctypes.data_as(C.POINTER(C.c_double)), a.ctypes.data_as(C.POINTER(C.c_double)),
                 nu.ctypes.data_as(C.POINTER(C.c_double)), Q.ctypes.data_as(C.POINTER(C.c_double)),
                 reac.ctypes.data_as(C.POINTER(C.c_int)), cnt.ctypes.data_as(C.POINTER(C.c_int)),
                 prod.ctypes.data_as(C.POINTER(C.c_int)))
    prm = Params(P0.gamma, P0.n_nodes, P0.n_iters, P0.limiter, int(prec), P0.newton_rtol, P0.newton_maxit,
                 NODE_TYPES[P0.nodes], int(P0.space_order))
    return boxes, len(problems), nw, prm, keep


def step_static(problems, U, dt, prec=PREC_FP64, stream=None, stats=True):
    """One SDC step through sdc_step_static: no device allocation by the
    library (its workspace is a fixed 48 MiB device array shared by all calls
    in the process; calls that overlap on the GPU race)."""
    import torch
    L = load()
    boxes, nbox, nw, prm, keep = _marshal(problems, prec)
    stream = stream if stream is not None else torch.cuda.current_stream()
    st = Stats() if stats else None
    s = L.sdc_step_static(boxes, nbox, C.byref(nw), C.byref(prm), C.c_void_p(stream.cuda_stream), _ptr(U),
                          float(dt), C.byref(st) if st is not None else None)
    del keep
    if s not in (SDC_OK, SDC_ERR_NEWTON_NOCONV):
        raise SdcError(s, "sdc_step_static")
    return st


def selftest_math(x):
    """The library's Newton-Raphson reciprocal and square root of x (CUDA float64)."""
    import torch
    r = torch.empty_like(x)
    q = torch.empty_like(x)
    s = load().sdc_selftest_math(_ptr(x), x.numel(), _ptr(r), _ptr(q),
                                 C.c_void_p(torch.cuda.current_stream().cuda_stream))
    if s != SDC_OK:
        raise SdcError(s, "sdc_selftest_math")
    return r, q


def selftest_pow(T, nu):
    """The library's power-law rate factor T^nu (CUDA float64 tensors of one size)."""
    import torch
    out = torch.empty_like(T)
    s = load().sdc_selftest_pow(_ptr(T), _ptr(nu), T.numel(), _ptr(out),
                                C.c_void_p(torch.cuda.current_stream().cuda_stream))
    if s != SDC_OK:
        raise SdcError(s, "sdc_selftest_pow")
    return out


def init_box(problems, prec=PREC_FP64, stream=None) -> Context:
    return Context(problems, prec=prec, stream=stream)


def _autograd_function():
    import torch

    class SDCStep(torch.autograd.Function):
        """One SDC step as a differentiable op: forward = sdc_step on a copy of U
        with rate prefactors a; backward = sdc_step_backward from the saved input
        state (a per-step checkpoint), giving dL/dU and dL/da."""

        @staticmethod
        def forward(fctx, U, a, context, dt):
            context.set_rates(a.detach().cpu().numpy())
            Un = U.detach().contiguous().clone()
            out = Un.clone()
            context.step(out, dt, stats=False)
            fctx.save_for_backward(Un, a.detach())
            fctx.context = context
            fctx.dt = dt
            return out

        @staticmethod
        def backward(fctx, gU):
            Un, a = fctx.saved_tensors
            context = fctx.context
            context.set_rates(a.cpu().numpy())
            gUn = torch.empty_like(Un)
            ga = torch.zeros(a.numel(), dtype=torch.float64, device=Un.device)
            context.step_backward(Un, fctx.dt, gU.contiguous(), gUn, ga)
            return gUn, ga.to(a.device), None, None

    return SDCStep


_SDCStep = None


def sdc_step_fn(U, a, context, dt):
    """Differentiable SDC step: U [nvar][Ntot] (CUDA float64), a [nreac] rate
    prefactors (float64 tensor, gradients flow to it)."""
    global _SDCStep
    if _SDCStep is None:
        _SDCStep = _autograd_function()
    return _SDCStep.apply(U, a, context, dt)
