"""Python binding of the GB300 MLFMA library (argument marshalling only).

Every step of the matvec runs in the CUDA kernels of ``libmlfma.so`` behind the
C ABI declared in ``include/mlfma.h``; this module only passes pointers, sizes
and the current CUDA stream, and hands the library PyTorch's caching allocator
for its device memory.  There is no fallback: if the library is missing the
import of a plan fails with an error that says how to build it.

The functions keep the C names (``mlfma_plan_create``, ``mlfma_apply``,
``mlfma_apply_adjoint``, ``mlfma_plan_info``, ``mlfma_plan_export``,
``mlfma_direct_fp64``, ``mlfma_destroy``, ``mlfma_last_error``); ``Plan`` wraps
them for torch tensors.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

PREC_FP64 = 0
PREC_FP32 = 1
PREC_FP32_BF16X3 = 2
PREC_FP32_TF32X3 = 3
_PREC = {"fp64": PREC_FP64, "fp32": PREC_FP32, "bf16x3": PREC_FP32_BF16X3, "tf32x3": PREC_FP32_TF32X3}
MAX_LEVELS = 22

EXPORT = dict(PERM=0, KEYS=1, BOX_KEY=2, BOX_BEGIN=3, BOX_END=4, BOX_PARENT=5, BOX_LEAF=6, V_OFFSETS=7,
              V_SOURCES=8, NEAR_OFFSETS=9, NEAR_SOURCES=10, F=11, G=12, NEAR_PHI=13, TRANSLATION=14,
              OPERATOR_SAMPLES=15)
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "OUT_OF_MEMORY", 3: "CUDA", 4: "TIMEOUT", 5: "UNSUPPORTED"}

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class Options(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_size_t), ("precision", ctypes.c_int), ("leaf_edge", ctypes.c_double),
                ("max_depth", ctypes.c_int), ("digit_margin", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", ctypes.c_void_p), ("disable_graphs", ctypes.c_int),
                ("autotune", ctypes.c_int), ("recompute_signatures", ctypes.c_int), ("test_fail_waits", ctypes.c_int),
                ("dense_samples", ctypes.c_int), ("sampled_operators", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nlev", ctypes.c_int), ("top", ctypes.c_int), ("precision", ctypes.c_int),
                ("k", ctypes.c_double), ("leaf_edge", ctypes.c_double), ("root_edge", ctypes.c_double),
                ("root_corner", ctypes.c_double * 3), ("nbox", ctypes.c_int64 * (MAX_LEVELS + 1)),
                ("nleaf", ctypes.c_int64 * (MAX_LEVELS + 1)), ("L", ctypes.c_int * (MAX_LEVELS + 1)),
                ("K", ctypes.c_int64 * (MAX_LEVELS + 1)), ("nv", ctypes.c_int64 * (MAX_LEVELS + 1)),
                ("near_pairs", ctypes.c_int64), ("device_bytes", ctypes.c_int64), ("setup_ms", ctypes.c_double),
                ("n_geom", ctypes.c_int), ("tile_bytes", ctypes.c_int * 3), ("recompute_signatures", ctypes.c_int),
                ("dense", ctypes.c_int * (MAX_LEVELS + 1)), ("sampled_operators", ctypes.c_int),
                ("sampled", ctypes.c_int * (MAX_LEVELS + 1))]


STAGES = ["PERMUTE", "P2P", "C2M", "M2M", "M2L", "L2L", "L2O"]


class Timings(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * len(STAGES)), ("launches", ctypes.c_int64 * len(STAGES)),
                ("m2l_ms", ctypes.c_double * (MAX_LEVELS + 1)), ("applies", ctypes.c_int64)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("restarts", ctypes.c_int), ("matvecs", ctypes.c_int),
                ("converged", ctypes.c_int), ("rel_residual", ctypes.c_double)]


class MLFMAError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Loads libmlfma.so; raises if it is missing (no CPU fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if build_if_missing:
            _build.build()
        else:
            raise RuntimeError("libmlfma.so is not built: run `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(_build.LIB)
    vp, i64, ci, cd = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    lib.mlfma_options_init.argtypes = [ctypes.POINTER(Options)]
    lib.mlfma_options_init.restype = None
    lib.mlfma_plan_create.argtypes = [vp, i64, cd, ci, ci, ctypes.POINTER(Options), ctypes.POINTER(vp)]
    lib.mlfma_plan_create.restype = ci
    lib.mlfma_plan_create_batched.argtypes = [vp, vp, ci, cd, ci, ci, ctypes.POINTER(Options), ctypes.POINTER(vp)]
    lib.mlfma_plan_create_batched.restype = ci
    lib.mlfma_apply.argtypes = [vp, vp, vp, ci]
    lib.mlfma_apply.restype = ci
    lib.mlfma_apply_adjoint.argtypes = [vp, vp, vp, ci]
    lib.mlfma_apply_adjoint.restype = ci
    lib.mlfma_apply_grad.argtypes = [vp, vp, vp, vp, ci]
    lib.mlfma_apply_grad.restype = ci
    lib.mlfma_apply_vjp.argtypes = [vp, vp, vp, vp, vp, vp, ci]
    lib.mlfma_apply_vjp.restype = ci
    lib.mlfma_plan_info.argtypes = [vp, ctypes.POINTER(Info)]
    lib.mlfma_plan_info.restype = ci
    lib.mlfma_plan_export.argtypes = [vp, ci, ci, vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
    lib.mlfma_plan_export.restype = ci
    lib.mlfma_direct_fp64.argtypes = [vp, i64, vp, cd, vp, i64, vp, vp]
    lib.mlfma_direct_fp64.restype = ci
    lib.mlfma_plan_profile.argtypes = [vp, ci]
    lib.mlfma_plan_profile.restype = ci
    lib.mlfma_plan_timings.argtypes = [vp, ctypes.POINTER(Timings), ci]
    lib.mlfma_plan_timings.restype = ci
    lib.mlfma_apply_near_noalloc.argtypes = [vp, vp, vp]
    lib.mlfma_apply_near_noalloc.restype = ci
    lib.mlfma_solve_gmres.argtypes = [vp, vp, vp, cd, cd, cd, ci, ci, ctypes.POINTER(SolveInfo)]
    lib.mlfma_solve_gmres.restype = ci
    lib.mlfma_destroy.argtypes = [vp]
    lib.mlfma_destroy.restype = None
    lib.mlfma_last_error.argtypes = []
    lib.mlfma_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def mlfma_last_error() -> str:
    return load().mlfma_last_error().decode()


def _check(st):
    if st != 0:
        raise MLFMAError(st, mlfma_last_error())


def _ptr(x):
    """Address of a torch tensor or numpy array (must be contiguous, no lazy conjugation)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if (hasattr(x, "is_conj") and x.is_conj()) or (hasattr(x, "is_neg") and x.is_neg()):
            raise ValueError("tensor is a lazy conjugate/negative view; call resolve_conj() first")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    return int(x)


def mlfma_options_init() -> Options:
    o = Options()
    load().mlfma_options_init(ctypes.byref(o))
    return o


def mlfma_plan_create(points, n, k, digits, leaf_max, options=None):
    """C call: returns the opaque plan handle (int)."""
    h = ctypes.c_void_p()
    _check(load().mlfma_plan_create(_ptr(points), int(n), float(k), int(digits), int(leaf_max),
                                    ctypes.byref(options) if options is not None else None, ctypes.byref(h)))
    return h.value


def mlfma_plan_create_batched(points, offsets, n_geom, k, digits, leaf_max, options=None):
    """C call: one plan for n_geom independent geometries; offsets is a host int64 array."""
    h = ctypes.c_void_p()
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    _check(load().mlfma_plan_create_batched(_ptr(points), off.ctypes.data, int(n_geom), float(k), int(digits),
                                            int(leaf_max), ctypes.byref(options) if options is not None else None,
                                            ctypes.byref(h)))
    return h.value


def mlfma_apply(plan, q, phi, nrhs):
    _check(load().mlfma_apply(plan, _ptr(q), _ptr(phi), int(nrhs)))


def mlfma_apply_adjoint(plan, r, g, nrhs):
    _check(load().mlfma_apply_adjoint(plan, _ptr(r), _ptr(g), int(nrhs)))


def mlfma_apply_grad(plan, q, phi, grad, nrhs):
    _check(load().mlfma_apply_grad(plan, _ptr(q), _ptr(phi), _ptr(grad), int(nrhs)))


def mlfma_apply_vjp(plan, q, g, gphi, grad_q, grad_r, nrhs):
    _check(load().mlfma_apply_vjp(plan, _ptr(q), _ptr(g), _ptr(gphi), _ptr(grad_q), _ptr(grad_r), int(nrhs)))


def mlfma_plan_info(plan) -> Info:
    info = Info()
    _check(load().mlfma_plan_info(plan, ctypes.byref(info)))
    return info


def mlfma_plan_export(plan, item, level, dst=None):
    need = ctypes.c_size_t()
    if dst is None:
        _check(load().mlfma_plan_export(plan, int(item), int(level), None, 0, ctypes.byref(need)))
        return need.value
    nbytes = dst.numel() * dst.element_size() if hasattr(dst, "numel") else dst.nbytes
    _check(load().mlfma_plan_export(plan, int(item), int(level), _ptr(dst), nbytes, ctypes.byref(need)))
    return need.value


def mlfma_direct_fp64(points, n, q, k, targets, nt, phi, stream=None):
    _check(load().mlfma_direct_fp64(_ptr(points), int(n), _ptr(q), float(k), _ptr(targets), int(nt), _ptr(phi),
                                    stream))


def mlfma_plan_profile(plan, enable):
    _check(load().mlfma_plan_profile(plan, int(bool(enable))))


def mlfma_plan_timings(plan, reset=True) -> Timings:
    t = Timings()
    _check(load().mlfma_plan_timings(plan, ctypes.byref(t), int(bool(reset))))
    return t


def mlfma_apply_near_noalloc(plan, q, phi):
    """Near-field part of A q into phi (device tensors), allocating nothing."""
    _check(load().mlfma_apply_near_noalloc(plan, _ptr(q), _ptr(phi)))


def mlfma_solve_gmres(plan, b, x, sigma, tol, restart, max_iter) -> SolveInfo:
    info = SolveInfo()
    sigma = complex(sigma)
    _check(load().mlfma_solve_gmres(plan, _ptr(b), _ptr(x), sigma.real, sigma.imag, float(tol), int(restart),
                                    int(max_iter), ctypes.byref(info)))
    return info


def mlfma_destroy(plan):
    if plan:
        load().mlfma_destroy(plan)


# ---------------------------------------------------------------------------
# torch-facing wrapper
# ---------------------------------------------------------------------------
class _TorchAllocator:
    """Routes the library's device allocations through PyTorch's caching allocator."""

    def __init__(self, device):
        import torch
        self.torch = torch
        self.device = device

        def _alloc(size, stream, ctx):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(size), device=self.device,
                                                              stream=int(stream or 0)))
            except Exception:
                return None

        def _free(ptr, stream, ctx):
            try:
                torch.cuda.caching_allocator_delete(int(ptr))
            except Exception:
                pass
        self.alloc = ALLOC_FN(_alloc)
        self.free = FREE_FN(_free)


class Plan:
    """An MLFMA plan for one point set: ``phi = plan.apply(q)``.

    points    [n, 3] float64 (torch tensor on a CUDA device, or host array)
    k         wavenumber; digits: requested accuracy; leaf_max: 0 = level-uniform tree
    precision "fp32" (complex64 data), "fp64" (complex128 data), "tf32x3" or "bf16x3" (complex64
              data, the theta maps of the large level pairs on the tensor cores as split-TF32 /
              split-BF16 GEMMs)
    dense_samples  tensor-core precisions, opt-in: level pairs whose child grid has at most this many
              samples run as dense maps (0: never; mlfma_options.dense_samples)
    sampled_operators  oversampling s (3-32) of the sampled translation operators at levels with boxes
              of a wavelength or more, interpolated in M2L (0: full tables; mlfma_options.sampled_operators)
    offsets   concatenated geometries: offsets[g] .. offsets[g + 1] are geometry g's points (one
              batched plan; the matrix is block diagonal)
    graphs    replay the apply as a captured CUDA graph (default) or launch the kernels each time
    autotune  time candidate interpolation tile budgets at creation and keep the fastest
    recompute_signatures  reverse mode: False keeps grad phi of the forward charges for the backward
              pass, True recomputes it there (mlfma_options.recompute_signatures)
    test_fail_waits  test hook: every bounded device wait gives up at once (MLFMA_ERR_TIMEOUT path)
    allocator a custom (alloc, free) pair of ctypes callbacks (ALLOC_FN, FREE_FN) instead of
              PyTorch's caching allocator

    Methods: apply (A q), adjoint (A^H r), apply_grad (A q and its gradient at the points),
    vjp (reverse mode of the matvec), solve ((sigma I + A) x = b by restarted GMRES), info, export,
    profile, timings, close.
    """

    def __init__(self, points, k, digits=3, leaf_max=0, precision="fp32", leaf_edge=0.0, max_depth=12,
                 digit_margin=-1, stream=None, use_torch_allocator=True, offsets=None, graphs=True, autotune=False,
                 recompute_signatures=False, test_fail_waits=False, allocator=None, dense_samples=0,
                 sampled_operators=0):
        import torch
        self.torch = torch
        load()
        if hasattr(points, "device") and points.device.type == "cuda":
            self.device = points.device
        else:
            self.device = torch.device("cuda", torch.cuda.current_device())
        if hasattr(points, "dtype") and hasattr(points, "data_ptr"):
            pts = points.to(torch.float64).contiguous()
        else:
            pts = np.ascontiguousarray(points, dtype=np.float64)
        self.n = int(pts.shape[0])
        self.k = float(k)
        self.precision = precision
        self.cdtype = torch.complex128 if precision == "fp64" else torch.complex64
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            o = mlfma_options_init()
            o.precision = _PREC[precision]
            o.leaf_edge = float(leaf_edge)
            o.max_depth = int(max_depth)
            o.digit_margin = int(digit_margin)
            o.stream = self.stream.cuda_stream
            o.disable_graphs = 0 if graphs else 1
            o.autotune = 1 if autotune else 0
            o.recompute_signatures = 1 if recompute_signatures else 0
            o.test_fail_waits = 1 if test_fail_waits else 0
            o.dense_samples = int(dense_samples)
            o.sampled_operators = int(sampled_operators)
            self._alloc = None
            if allocator is not None:
                self._alloc = allocator
                o.alloc, o.free = allocator
            elif use_torch_allocator:
                self._alloc = _TorchAllocator(self.device)
                o.alloc = self._alloc.alloc
                o.free = self._alloc.free
            if offsets is None:
                self.handle = mlfma_plan_create(pts, self.n, self.k, digits, leaf_max, o)
            else:
                off = np.asarray(offsets, dtype=np.int64)
                if off[-1] != self.n:
                    raise ValueError("offsets[-1] must equal the number of points")
                self.handle = mlfma_plan_create_batched(pts, off, off.shape[0] - 1, self.k, digits, leaf_max, o)
        self._points = pts
        self.recompute_signatures = bool(recompute_signatures)

    def _vec(self, x, name):
        t = self.torch
        if not isinstance(x, t.Tensor):
            x = t.as_tensor(np.asarray(x))
        if x.dtype != self.cdtype:
            raise TypeError(f"{name} must be {self.cdtype} for precision {self.precision}")
        if x.shape[-1] != self.n or x.dim() > 2:
            raise ValueError(f"{name} must be [n] or [nrhs, n] with n = {self.n}")
        # lazy conjugate / negative views keep unconjugated storage: materialise them
        return x.resolve_conj().resolve_neg().contiguous()

    def apply(self, q, out=None, adjoint=False):
        q = self._vec(q, "q")
        nrhs = 1 if q.dim() == 1 else q.shape[0]
        if out is None:
            out = self.torch.empty_like(q)
        with self.torch.cuda.device(self.device):
            (mlfma_apply_adjoint if adjoint else mlfma_apply)(self.handle, q, out, nrhs)
        return out

    def adjoint(self, r, out=None):
        return self.apply(r, out, adjoint=True)

    def apply_grad(self, q, want_phi=True):
        """(phi, grad) with grad[..., i, :] = gradient of phi_i with respect to r_i."""
        q = self._vec(q, "q")
        nrhs = 1 if q.dim() == 1 else q.shape[0]
        phi = self.torch.empty_like(q) if want_phi else None
        grad = self.torch.empty(tuple(q.shape) + (3,), dtype=q.dtype, device=q.device)
        with self.torch.cuda.device(self.device):
            mlfma_apply_grad(self.handle, q, phi, grad, nrhs)
        return phi, grad

    def vjp(self, q, g, gphi=None, want_q=True, want_r=True):
        """Reverse mode of phi = A(r) q: (grad_q, grad_r) for the upstream gradient g (PyTorch's
        convention); gphi = grad phi of q from apply_grad, or None to recompute it."""
        t = self.torch
        q = self._vec(q, "q")
        g = self._vec(g, "g")
        nrhs = 1 if q.dim() == 1 else q.shape[0]
        if g.shape != q.shape:
            raise ValueError("g must have the shape of q")
        if gphi is not None:
            gphi = gphi.contiguous()
            if tuple(gphi.shape) != tuple(q.shape) + (3,) or gphi.dtype != self.cdtype:
                raise ValueError("gphi must be [..., n, 3] of the plan's complex type")
        gq = t.empty_like(q) if want_q else None
        gr = t.empty((self.n, 3), dtype=t.float64, device=q.device) if want_r else None
        with t.cuda.device(self.device):
            mlfma_apply_vjp(self.handle, q, g, gphi, gq, gr, nrhs)
        return gq, gr

    def solve(self, b, sigma=0.0, tol=1e-3, restart=30, max_iter=300, x0=None):
        """x with (sigma I + A) x = b by restarted GMRES on the device; returns (x, info dict)."""
        b = self._vec(b, "b")
        if b.dim() != 1:
            raise ValueError("solve takes one right-hand side [n]")
        x = self.torch.zeros_like(b) if x0 is None else self._vec(x0, "x0").clone()
        with self.torch.cuda.device(self.device):
            i = mlfma_solve_gmres(self.handle, b, x, sigma, tol, restart, max_iter)
        return x, dict(iterations=i.iterations, restarts=i.restarts, matvecs=i.matvecs, converged=bool(i.converged),
                       rel_residual=i.rel_residual)

    def info(self) -> dict:
        i = mlfma_plan_info(self.handle)
        nl = i.nlev
        return dict(n=i.n, nlev=nl, top=i.top, precision=i.precision, k=i.k, leaf_edge=i.leaf_edge,
                    root_edge=i.root_edge, root_corner=list(i.root_corner),
                    nbox=list(i.nbox[:nl + 1]), nleaf=list(i.nleaf[:nl + 1]), L=list(i.L[:nl + 1]),
                    K=list(i.K[:nl + 1]), nv=list(i.nv[:nl + 1]), near_pairs=i.near_pairs,
                    device_bytes=i.device_bytes, setup_ms=i.setup_ms, n_geom=i.n_geom,
                    tile_bytes=list(i.tile_bytes), recompute_signatures=bool(i.recompute_signatures),
                    dense=list(i.dense[:nl + 1]), sampled_operators=i.sampled_operators,
                    sampled=list(i.sampled[:nl + 1]))

    def export(self, item, level=0):
        """Copies a tree/list/signature array to a host numpy array."""
        it = EXPORT[item] if isinstance(item, str) else int(item)
        nbytes = mlfma_plan_export(self.handle, it, level)
        buf = np.empty(nbytes, dtype=np.uint8)
        mlfma_plan_export(self.handle, it, level, buf)
        name = item if isinstance(item, str) else [k for k, v in EXPORT.items() if v == it][0]
        if name in ("KEYS", "BOX_KEY"):
            return buf.view(np.uint64)
        if name == "BOX_LEAF":
            return buf.view(np.uint8)
        if name in ("F", "G", "NEAR_PHI", "TRANSLATION", "OPERATOR_SAMPLES"):
            return buf.view(np.complex128 if self.precision == "fp64" else np.complex64)
        return buf.view(np.int32)

    def profile(self, enable=True):
        """Start/stop recording CUDA events around every apply stage."""
        mlfma_plan_profile(self.handle, enable)

    def timings(self, reset=True) -> dict:
        t = mlfma_plan_timings(self.handle, reset)
        return dict(ms={s: t.ms[i] for i, s in enumerate(STAGES)},
                    launches={s: t.launches[i] for i, s in enumerate(STAGES)},
                    m2l_ms=list(t.m2l_ms), applies=t.applies)

    def close(self):
        if getattr(self, "handle", None):
            mlfma_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def direct_fp64(points, q, k, targets, stream=None):
    """Exact FP64 sum on the GPU at ``targets`` (torch CUDA tensors)."""
    import torch
    pts = points.to(torch.float64).contiguous()
    qq = q.to(torch.complex128).contiguous()
    tg = targets.to(torch.int64).contiguous()
    out = torch.empty(tg.shape[0], dtype=torch.complex128, device=pts.device)
    s = stream if stream is not None else torch.cuda.current_stream(pts.device)
    mlfma_direct_fp64(pts, pts.shape[0], qq, k, tg, tg.shape[0], out, s.cuda_stream)
    return out


# ---------------------------------------------------------------------------
# autograd
# ---------------------------------------------------------------------------
def _function():
    import torch

    class MLFMAFunction(torch.autograd.Function):
        """phi = A(r) q with gradients for the complex charges q and the positions r.

        forward: mlfma_apply_grad (phi and grad phi, kept for the backward pass) or, for plans
        created with recompute_signatures, mlfma_apply (grad phi is recomputed in the backward).
        backward: mlfma_apply_vjp with the upstream gradient (PyTorch's convention), which forms
        q.grad = A^H g and r.grad = Re[conj(g) grad phi + q grad psi], psi = A conj(g), in the
        library's kernels.  The tree of the plan is kept fixed.
        """

        @staticmethod
        def forward(ctx, q, points, plan):
            keep = points is not None and points.requires_grad and not plan.recompute_signatures
            if keep:
                phi, gphi = plan.apply_grad(q)
            else:
                phi, gphi = plan.apply(q), None
            ctx.plan = plan
            ctx.rdtype = points.dtype if points is not None else None
            ctx.has_gphi = gphi is not None
            ctx.save_for_backward(q, gphi if gphi is not None else q.new_zeros(0))
            return phi

        @staticmethod
        def backward(ctx, g):
            q, gphi = ctx.saved_tensors
            want_q, want_r = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
            if not (want_q or want_r):
                return None, None, None
            gq, gr = ctx.plan.vjp(q, g.contiguous(), gphi if ctx.has_gphi else None, want_q=want_q, want_r=want_r)
            if gr is not None and gr.dtype != ctx.rdtype:
                gr = gr.to(ctx.rdtype)              # the positions' own dtype (the library writes FP64)
            return gq, gr, None

    return MLFMAFunction


_MLFMAFunction = None


def mlfma(q, points, plan):
    """Differentiable matvec: phi = A(points) q through ``plan`` (built on ``points``)."""
    global _MLFMAFunction
    if _MLFMAFunction is None:
        _MLFMAFunction = _function()
    return _MLFMAFunction.apply(q, points, plan)
