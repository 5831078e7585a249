"""ceedbp: GB300-native matrix-free bake-off operators (BP1/BP3/BP5/BP6) and Jacobi-PCG.

Thin Python binding over the C ABI of ``libceedbp.so`` (declared in
``include/ceedbp.h``).  Every step of the operator and the solver runs in the
library's CUDA kernels; this module only marshals arguments.  PyTorch supplies
device memory and the CUDA stream.  There is no CPU fallback: importing the
binding without the built library, or calling it without a CUDA device, raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libceedbp.so")

OK, EINVAL, ENOMEM, ECUDA, ENOCONV, EBREAKDOWN, EUNSUPPORTED = range(7)
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOCONV", 5: "EBREAKDOWN", 6: "EUNSUPPORTED"}
ARITH_FP64, ARITH_DF64 = 0, 1
GEOM_STORED, GEOM_RECOMPUTE = 0, 1
MIXED_NONE, MIXED_FP32, MIXED_BF16, MIXED_FP32_TC = 0, 1, 2, 3


class CeedbpError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("bp", ctypes.c_int), ("order", ctypes.c_int), ("nquad", ctypes.c_int),
                ("nelem", ctypes.c_int64), ("nglobal", ctypes.c_int64), ("arith", ctypes.c_int),
                ("geom", ctypes.c_int)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxit", ctypes.c_int), ("fixed_iters", ctypes.c_int),
                ("chunk", ctypes.c_int), ("use_graph", ctypes.c_int), ("x0_nonzero", ctypes.c_int),
                ("profile", ctypes.c_int), ("mixed", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("inner_maxit", ctypes.c_int), ("outer_maxit", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int * 3), ("rel_res", ctypes.c_double * 3),
                ("res_norm", ctypes.c_double * 3), ("b_norm", ctypes.c_double * 3),
                ("device_ms", ctypes.c_double), ("kernel_ms", ctypes.c_double * 3), ("status", ctypes.c_int),
                ("outer_iters", ctypes.c_int)]

    def as_dict(self, ncomp: int) -> dict:
        return {"iters": list(self.iters[:ncomp]), "rel_res": list(self.rel_res[:ncomp]),
                "res_norm": list(self.res_norm[:ncomp]), "b_norm": list(self.b_norm[:ncomp]),
                "device_ms": self.device_ms, "kernel_ms": list(self.kernel_ms),
                "status": STATUS_NAMES.get(self.status, self.status), "outer_iters": self.outer_iters}


_P = ctypes.c_void_p
_SIGS = {
    "ceedbp_mesh_box": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                       _P, _P, _P, ctypes.POINTER(ctypes.c_int64)]),
    "ceedbp_setup": (ctypes.c_int, [ctypes.POINTER(Params), _P, _P, _P, _P, _P, ctypes.POINTER(_P)]),
    "ceedbp_apply": (ctypes.c_int, [_P, _P, _P]),
    "ceedbp_mass": (ctypes.c_int, [_P, _P, _P]),
    "ceedbp_jacobi": (ctypes.c_int, [_P, _P]),
    "ceedbp_prepare_mixed": (ctypes.c_int, [_P, ctypes.c_int]),
    "ceedbp_set_kappa": (ctypes.c_int, [_P, _P]),
    "ceedbp_misfit": (ctypes.c_int, [_P, _P, _P, _P, ctypes.POINTER(ctypes.c_double)]),
    "ceedbp_kappa_gradient": (ctypes.c_int, [_P, _P, _P, _P]),
    "ceedbp_solve": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveInfo)]),
    "ceedbp_apply_noalloc": (ctypes.c_int, [_P, _P, _P, _P]),
    "ceedbp_destroy": (ctypes.c_int, [_P]),
    "ceedbp_tile_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int)]),
    "ceedbp_bk_apply": (ctypes.c_int, [_P, _P, _P]),
    "ceedbp_set_helmholtz": (ctypes.c_int, [_P, ctypes.c_double]),
    "ceedbp_set_tile": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "ceedbp_check": (ctypes.c_int, [_P]),
    "ceedbp_fma_peak": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]),
    "ceedbp_mma_peak": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "ceedbp_set_wait_limit": (ctypes.c_int, [_P, ctypes.c_int]),
    "ceedbp_batch_setup": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(Params), ctypes.POINTER(_P),
                                          ctypes.POINTER(_P), ctypes.POINTER(_P), _P, ctypes.POINTER(_P)]),
    "ceedbp_batch_solve": (ctypes.c_int, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(SolveOpts),
                                          ctypes.POINTER(SolveInfo)]),
    "ceedbp_batch_destroy": (ctypes.c_int, [_P]),
    "ceedbp_batch_last_error": (ctypes.c_char_p, [_P]),
    "ceedbp_last_error": (ctypes.c_char_p, [_P]),
}

_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libceedbp.so (built by ``__graft_entry__.build()``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"ceedbp library not built: {path} is missing (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int, ctx=None):
    if status != OK:
        msg = load_library().ceedbp_last_error(ctx)
        raise CeedbpError(status, msg.decode() if msg else "")


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def mesh_box(Ex: int, Ey: int, Ez: int, order: int, amp: float = 0.05):
    """Deformed-box mesh from the library (coords [E, p1^3, 3], l2g [E, p1^3], dirichlet [n_g])."""
    lib = load_library()
    p1 = order + 1
    E = Ex * Ey * Ez
    ng = ctypes.c_int64(0)
    _check(lib.ceedbp_mesh_box(Ex, Ey, Ez, order, amp, None, None, None, ctypes.byref(ng)))
    coords = np.empty((E, p1 ** 3, 3), dtype=np.float64)
    l2g = np.empty((E, p1 ** 3), dtype=np.int64)
    dirichlet = np.empty(ng.value, dtype=np.uint8)
    _check(lib.ceedbp_mesh_box(Ex, Ey, Ez, order, amp, _ptr(coords), _ptr(l2g), _ptr(dirichlet), None))
    return coords, l2g, dirichlet


def fma_peak(fp64: bool = True):
    """Measured FMA throughput of the current CUDA device: (TFLOP/s, SM count) (ceedbp_fma_peak)."""
    lib = load_library()
    tf, sms = ctypes.c_double(0.0), ctypes.c_int(0)
    _check(lib.ceedbp_fma_peak(1 if fp64 else 0, ctypes.byref(tf), ctypes.byref(sms)))
    return tf.value, sms.value


def mma_peak(kind: int) -> float:
    """Measured mma.sync throughput in TFLOP/s: kind 0 FP64 m8n8k4, 1 TF32 m16n8k8, 2 BF16 m16n8k16."""
    lib = load_library()
    tf = ctypes.c_double(0.0)
    _check(lib.ceedbp_mma_peak(int(kind), ctypes.byref(tf)))
    return tf.value


class Operator:
    """One bake-off problem on the GPU: ceedbp_setup / apply / mass / solve / destroy."""

    def __init__(self, bp: int, order: int, coords: np.ndarray, l2g: np.ndarray, dirichlet: np.ndarray | None,
                 kappa: np.ndarray | None = None, stream=None, device=None, arith: int = 0,
                 geom: int = 0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("ceedbp needs a CUDA device; there is no CPU path")
        self.lib = load_library()
        self.device = torch.device("cuda") if device is None else torch.device(device)
        # a dedicated stream: CUDA graphs cannot be captured on the legacy default stream
        self.stream = torch.cuda.Stream(self.device) if stream is None else stream
        self.bp, self.order = bp, order
        self.ncomp = 3 if bp in (2, 4, 6) else 1
        coords = np.ascontiguousarray(coords, dtype=np.float64)
        l2g = np.ascontiguousarray(l2g, dtype=np.int64)
        self.nelem = coords.shape[0]
        p1 = order + 1
        if coords.shape != (self.nelem, p1 ** 3, 3) or l2g.shape != (self.nelem, p1 ** 3):
            raise ValueError(f"coords must be [E, {p1 ** 3}, 3] and l2g [E, {p1 ** 3}] for order {order}")
        self.nglobal = int(dirichlet.shape[0]) if dirichlet is not None else int(l2g.max()) + 1
        q = order + 1 if bp in (5, 6) else order + 2
        if kappa is not None and np.asarray(kappa).size != self.nelem * q ** 3:
            raise ValueError(f"kappa must hold E * {q ** 3} values")
        dirichlet = None if dirichlet is None else np.ascontiguousarray(dirichlet, dtype=np.uint8)
        kappa = None if kappa is None else np.ascontiguousarray(kappa, dtype=np.float64)
        self.arith, self.geom = arith, geom
        prm = Params(bp, order, 0, self.nelem, self.nglobal, arith, geom)
        ctx = ctypes.c_void_p()
        cur = torch.cuda.current_stream(self.device)
        self.stream.wait_stream(cur)
        st = self.lib.ceedbp_setup(ctypes.byref(prm), _ptr(coords), _ptr(l2g), _ptr(dirichlet), _ptr(kappa),
                                   ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(ctx))
        _check(st, None)
        self.ctx = ctx

    @classmethod
    def box(cls, bp: int, Ex: int, Ey: int, Ez: int, order: int, amp: float = 0.05, kappa=None, **kw):
        coords, l2g, dirichlet = mesh_box(Ex, Ey, Ez, order, amp)
        op = cls(bp, order, coords, l2g, dirichlet, kappa=kappa, **kw)
        op.dims = (Ex, Ey, Ez)
        op.coords = coords
        return op

    def _vec(self, v):
        import torch
        if not (v.is_cuda and v.dtype == torch.float64 and v.is_contiguous()):
            raise ValueError("vectors must be contiguous float64 CUDA tensors")
        if v.numel() != self.nglobal * self.ncomp:
            raise ValueError(f"vector has {v.numel()} entries, expected {self.nglobal * self.ncomp}")
        return ctypes.c_void_p(v.data_ptr())

    def empty(self):
        import torch
        shape = (self.nglobal,) if self.ncomp == 1 else (self.nglobal, 3)
        return torch.empty(shape, dtype=torch.float64, device=self.device)

    def _enter(self):
        import torch
        cur = torch.cuda.current_stream(self.device)
        if cur.cuda_stream != self.stream.cuda_stream:
            self.stream.wait_stream(cur)
        return cur

    def _leave(self, cur):
        if cur.cuda_stream != self.stream.cuda_stream:
            cur.wait_stream(self.stream)

    def _call(self, fn, *args):
        cur = self._enter()
        try:
            st = fn(self.ctx, *args)
        finally:
            self._leave(cur)
        return st

    def apply(self, u, out=None):
        w = self.empty() if out is None else out
        _check(self._call(self.lib.ceedbp_apply, self._vec(u), self._vec(w)), self.ctx)
        return w

    def apply_noalloc(self, u, out=None):
        """ceedbp_apply_noalloc: same result as apply(), scratch in the library's static
        device array (no allocation), on this operator's stream."""
        w = self.empty() if out is None else out
        st = self._call(lambda ctx, a, b: self.lib.ceedbp_apply_noalloc(ctx, a, b, ctypes.c_void_p(self.stream.cuda_stream)),
                        self._vec(u), self._vec(w))
        _check(st, None)  # the message is the calling thread's (ceedbp_last_error(NULL))
        return w

    def check(self):
        """ceedbp_check: synchronise the operator's stream; raise CeedbpError(ECUDA) if a pair-path
        kernel gave up a bounded staging wait since the last check or solve."""
        _check(self.lib.ceedbp_check(self.ctx), self.ctx)

    def set_wait_limit(self, polls: int):
        """Polls of the staged pair schedule's first bounded wait (0: give up at once; < 0: default)."""
        _check(self.lib.ceedbp_set_wait_limit(self.ctx, int(polls)), self.ctx)

    def bk_apply(self, uL, out=None):
        """ceedbp_bk_apply: element-local w^e = A^e u^e (or B^e u^e), uL of shape [E, p1^3] or
        [E, p1^3, 3]; no gather-scatter, no Dirichlet mask."""
        import torch
        p3 = (self.order + 1) ** 3
        shape = (self.nelem, p3) if self.ncomp == 1 else (self.nelem, p3, 3)
        if not (uL.is_cuda and uL.dtype == torch.float64 and uL.is_contiguous()) or tuple(uL.shape) != shape:
            raise ValueError(f"uL must be a contiguous float64 CUDA tensor of shape {shape}")
        w = torch.empty(shape, dtype=torch.float64, device=self.device) if out is None else out
        if tuple(w.shape) != shape or not w.is_contiguous() or w.dtype != torch.float64:
            raise ValueError(f"out must be a contiguous float64 CUDA tensor of shape {shape}")
        _check(self._call(self.lib.ceedbp_bk_apply, ctypes.c_void_p(uL.data_ptr()), ctypes.c_void_p(w.data_ptr())),
               self.ctx)
        return w

    def mass(self, u, out=None):
        w = self.empty() if out is None else out
        _check(self._call(self.lib.ceedbp_mass, self._vec(u), self._vec(w)), self.ctx)
        return w

    def jacobi(self):
        import torch
        d = torch.empty(self.nglobal, dtype=torch.float64, device=self.device)
        _check(self._call(self.lib.ceedbp_jacobi, ctypes.c_void_p(d.data_ptr())), self.ctx)
        return d

    def _ptr_t(self, t, numel=None):
        import torch
        if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
            raise ValueError("expected a contiguous float64 CUDA tensor")
        if numel is not None and t.numel() != numel:
            raise ValueError(f"tensor has {t.numel()} entries, expected {numel}")
        return ctypes.c_void_p(t.data_ptr())

    @property
    def nquad(self) -> int:
        return self.order + 1 if self.bp in (5, 6) else self.order + 2

    def set_kappa(self, kappa):
        """kappa: float64 CUDA tensor [E, q^3] at the quadrature points."""
        _check(self._call(self.lib.ceedbp_set_kappa, self._ptr_t(kappa, self.nelem * self.nquad ** 3)), self.ctx)

    def misfit(self, u, u_star, rhs=None):
        """J = 1/2 (u - u*)^T B (u - u*) and the adjoint RHS M B (u - u*)."""
        rhs = self.empty() if rhs is None else rhs
        J = ctypes.c_double(0.0)
        _check(self._call(self.lib.ceedbp_misfit, self._vec(u), self._vec(u_star), self._vec(rhs),
                          ctypes.byref(J)), self.ctx)
        return rhs, J.value

    def kappa_gradient(self, u, lam, out=None):
        import torch
        g = out if out is not None else torch.empty((self.nelem, self.nquad ** 3), dtype=torch.float64,
                                                     device=self.device)
        _check(self._call(self.lib.ceedbp_kappa_gradient, self._vec(u), self._vec(lam),
                          self._ptr_t(g, self.nelem * self.nquad ** 3)), self.ctx)
        return g

    def tile_info(self):
        """(elements per block, schedule, elements per sequence) chosen by the setup autotuner for the
        pair kernel; schedule 0 = G ring, 1 = G staged by a bulk copy, 2 = pipelined sequences,
        3 = even-odd octets in pipelined sequences (BP5, odd orders 3..11)."""
        eb, st, seq = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        _check(self.lib.ceedbp_tile_info(self.ctx, ctypes.byref(eb), ctypes.byref(st), ctypes.byref(seq)),
               self.ctx)
        return eb.value, st.value, seq.value

    def set_helmholtz(self, beta: float):
        """Use H = A + beta B (Eq. (17)) in apply, bk_apply and solve; beta = 0 restores A."""
        _check(self._call(self.lib.ceedbp_set_helmholtz, ctypes.c_double(beta)), self.ctx)

    def set_tile(self, elems_per_block: int, schedule: int, seq: int = 1):
        """Pin the pair kernel's shape to one the autotuner times (see tile_info)."""
        _check(self.lib.ceedbp_set_tile(self.ctx, elems_per_block, schedule, seq), self.ctx)

    def prepare_mixed(self, precision: int):
        _check(self._call(self.lib.ceedbp_prepare_mixed, precision), self.ctx)

    def solve(self, b, x=None, tol: float = 1e-8, maxit: int = 10000, fixed_iters: int = 0, chunk: int = 32,
              use_graph: bool = True, x0=False, raise_on_noconv: bool = True, profile: bool = False,
              mixed: int = 0, inner_tol: float = 0.0, inner_maxit: int = 0, outer_maxit: int = 0):
        x = self.empty() if x is None else x
        opts = SolveOpts(tol, maxit, fixed_iters, chunk, int(use_graph), int(bool(x0)), int(profile),
                         int(mixed), float(inner_tol), int(inner_maxit), int(outer_maxit))
        info = SolveInfo()
        st = self._call(self.lib.ceedbp_solve, self._vec(b), self._vec(x), ctypes.byref(opts), ctypes.byref(info))
        if st != OK and (raise_on_noconv or st != ENOCONV):
            _check(st, self.ctx)
        return x, info.as_dict(self.ncomp)

    def close(self):
        if getattr(self, "ctx", None) is not None and self.ctx.value:
            self.lib.ceedbp_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kappa_misfit(kappa, op: "Operator", b, u_star, tol: float = 1e-10):
    """J(kappa) = 1/2 ||u(kappa) - u*||_B^2 with A(kappa) u = b, differentiable in kappa.

    The backward pass returns dJ/dkappa from one adjoint solve and the fused
    gradient kernel (ceedbp_kappa_gradient)."""
    import torch

    class _KappaMisfit(torch.autograd.Function):
        @staticmethod
        def forward(ctx, k):
            op.set_kappa(k.detach().contiguous())
            u, _ = op.solve(b, tol=tol)
            rhs, J = op.misfit(u, u_star)
            lam, _ = op.solve(rhs, tol=tol)
            ctx.save_for_backward(op.kappa_gradient(u, lam))
            return torch.tensor(J, dtype=torch.float64, device=k.device)

        @staticmethod
        def backward(ctx, grad_J):
            (g,) = ctx.saved_tensors
            return grad_J * g

    return _KappaMisfit.apply(kappa)


class Batch:
    """Many independent BP5 problems solved together (ceedbp_batch_setup / _solve)."""

    def __init__(self, problems, stream=None, device=None, arith: int = ARITH_FP64):
        """problems: list of (order, coords, l2g, dirichlet) as returned by mesh_box; arith: the
        arithmetic of every problem (ARITH_FP64 or ARITH_DF64)."""
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("ceedbp needs a CUDA device; there is no CPU path")
        self.lib = load_library()
        self.device = torch.device("cuda") if device is None else torch.device(device)
        self.stream = torch.cuda.Stream(self.device) if stream is None else stream
        n = len(problems)
        self._keep = []
        prm = (Params * n)()
        cp, lp, dp = (_P * n)(), (_P * n)(), (_P * n)()
        self.sizes = []
        for k, (order, coords, l2g, dirichlet) in enumerate(problems):
            coords = np.ascontiguousarray(coords, dtype=np.float64)
            l2g = np.ascontiguousarray(l2g, dtype=np.int64)
            dirichlet = np.ascontiguousarray(dirichlet, dtype=np.uint8)
            self._keep += [coords, l2g, dirichlet]
            prm[k] = Params(5, order, 0, coords.shape[0], dirichlet.shape[0], arith, GEOM_STORED)
            cp[k], lp[k], dp[k] = _ptr(coords), _ptr(l2g), _ptr(dirichlet)
            self.sizes.append((order, coords.shape[0], dirichlet.shape[0]))
        out = ctypes.c_void_p()
        torch.cuda.current_stream(self.device).synchronize()
        st = self.lib.ceedbp_batch_setup(n, prm, cp, lp, dp, ctypes.c_void_p(self.stream.cuda_stream),
                                         ctypes.byref(out))
        self._keep = []
        if st != OK:
            raise CeedbpError(st, (self.lib.ceedbp_batch_last_error(None) or b"").decode())
        self.handle = out
        self.n = n
        self.arith = arith

    def solve(self, bs, xs=None, tol: float = 1e-8, maxit: int = 10000, chunk: int = 32, use_graph: bool = True):
        import torch
        xs = [torch.empty_like(b) for b in bs] if xs is None else xs
        bp, xp = (_P * self.n)(), (_P * self.n)()
        for k in range(self.n):
            bp[k] = ctypes.c_void_p(bs[k].data_ptr())
            xp[k] = ctypes.c_void_p(xs[k].data_ptr())
        opts = SolveOpts(tol, maxit, 0, chunk, int(use_graph), 0, 0, 0, 0.0, 0, 0)
        infos = (SolveInfo * self.n)()
        cur = torch.cuda.current_stream(self.device)
        self.stream.wait_stream(cur)
        st = self.lib.ceedbp_batch_solve(self.handle, bp, xp, ctypes.byref(opts), infos)
        cur.wait_stream(self.stream)
        if st not in (OK,):
            raise CeedbpError(st, (self.lib.ceedbp_batch_last_error(self.handle) or b"").decode())
        return xs, [infos[k].as_dict(1) for k in range(self.n)]

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self.lib.ceedbp_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
